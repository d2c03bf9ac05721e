"""ap_lm_solve_noalloc, the damped solve for callers that may not allocate
device memory (code inside a CUDA-graph capture, fixed memory budgets, plug-ins
whose host owns all device memory), checked against the regular per-group
solve ap_lm_solve on the same matrix, on two calls in a row.

This file is collected last on purpose: a run that stops at the first failure
has already run every other test when it gets here.  It also passes on its own
in a fresh process."""
import ctypes

import numpy as np
import pytest

from _helpers import assert_step_close, configs, damped_matrix, device_context, with_data

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_01957_gb300 import build
    build()


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


PROBLEMS = {
    # one group of 103 parameters: the regular path solves it with block-Jacobi PCG
    "pcg_group": lambda: with_data(configs.crowded_field("noalloc_pcg", configs.SEED_BASE + 51, 160, 192, 6, 18,
                                                         configs.psf_moffat(9, 3.0))),
    # one group of at most 64 parameters: the regular path uses the dense Cholesky
    "chol_group": lambda: with_data(configs.mixed_small(seed=configs.SEED_BASE + 52, H=40, W=48, K=7)),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_noalloc_solve_matches_regular_solve(name):
    from paper_2308_01957_gb300 import _lib
    lib = _lib.load()
    pr = PROBLEMS[name]()
    ctx = device_context(pr, "mixed")
    assert ctx.n_groups == 1
    jtwr, (row_ptr, col_idx, vals) = ctx.normal_eq(pr.theta_init)
    n = pr.n_params
    d_row = torch.as_tensor(row_ptr, dtype=torch.int64, device="cuda")
    d_col = torch.as_tensor(col_idx, dtype=torch.int32, device="cuda")
    JtWJ = ctx.jtwj_dense((row_ptr, col_idx, vals))
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row: the shared scratch keeps the first call's contents
    for lam in (1e-3, 1.0):
        ref, lam_ref = ctx.lm_solve(np.array([lam]))
        lam_t = torch.tensor([lam], dtype=torch.float64, device="cuda")
        delta = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = lib.ap_lm_solve_noalloc(n, ctypes.c_void_p(d_row.data_ptr()), ctypes.c_void_p(d_col.data_ptr()),
                                     ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(jtwr.data_ptr()),
                                     ctypes.c_void_p(lam_t.data_ptr()), ctypes.c_void_p(delta.data_ptr()),
                                     ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert float(lam_t.item()) == float(lam_ref.item()) == lam
        # both solve the same damped system: the step tolerance of the tests
        # for a solve of the device's own matrix
        assert_step_close(_np(delta), _np(ref), JtWJ, lam, 1e-8)
        own = np.linalg.solve(damped_matrix(JtWJ, lam), _np(jtwr))
        assert_step_close(_np(delta), own, JtWJ, lam, 1e-8)
    assert ctx.status() == 0


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_2308_01957_gb300 import _lib
    lib = _lib.load()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    assert lib.ap_lm_solve_noalloc(16385, p, p, p, p, p, p, p, None) == _lib.AP_ERR_ARG
    assert lib.ap_lm_solve_noalloc(0, p, p, p, p, p, p, p, None) == _lib.AP_ERR_ARG
