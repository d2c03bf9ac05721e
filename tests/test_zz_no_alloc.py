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


def _call_noalloc(lib, n, row_ptr, col_idx, vals, b, lam):
    """One ap_lm_solve_noalloc call on host-built CSR arrays; returns
    (rc, status, lambda after, delta)."""
    d_row = torch.as_tensor(np.asarray(row_ptr, np.int64), device="cuda")
    d_col = torch.as_tensor(np.asarray(col_idx, np.int32), device="cuda")
    d_val = torch.as_tensor(np.asarray(vals, np.float64), device="cuda")
    d_b = torch.as_tensor(np.asarray(b, np.float64), device="cuda")
    lam_t = torch.tensor([lam], dtype=torch.float64, device="cuda")
    delta = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.ap_lm_solve_noalloc(n, ctypes.c_void_p(d_row.data_ptr()), ctypes.c_void_p(d_col.data_ptr()),
                                 ctypes.c_void_p(d_val.data_ptr()), ctypes.c_void_p(d_b.data_ptr()),
                                 ctypes.c_void_p(lam_t.data_ptr()), ctypes.c_void_p(delta.data_ptr()),
                                 ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return rc, int(status.item()), float(lam_t.item()), _np(delta)


def test_noalloc_indefinite_matrix_ends_not_spd():
    """A matrix with a negative diagonal block stays indefinite under every
    damping the retries reach (its damping diagonal is the floor): each try
    meets a non-positive curvature, lambda goes up x10 nine times (the first
    try and 8 retries), and the step is zero."""
    from paper_2308_01957_gb300 import _lib
    lib = _lib.load()
    # 4 x 4: a positive 2 x 2 block and a negative 2 x 2 block, stored in full
    A = np.array([[4.0, 1.0, 0.0, 0.0], [1.0, 3.0, 0.0, 0.0], [0.0, 0.0, -2.0, 0.5], [0.0, 0.0, 0.5, -1.0]])
    rows, cols = np.nonzero(A)
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=4))])
    lam0 = 1e-3
    for _ in range(2):   # two calls in a row share the scratch
        rc, status, lam, delta = _call_noalloc(lib, 4, row_ptr, cols, A[rows, cols], [1.0, 1.0, 1.0, 1.0], lam0)
        assert rc == 0 and status == _lib.AP_ERR_NOT_SPD
        assert np.all(delta == 0.0)
        assert lam == pytest.approx(lam0 * 10.0 ** 9, rel=1e-12)


def test_noalloc_ill_conditioned_matrix_times_out():
    """The 1-D Laplacian of 16384 points with a tiny damping has condition
    number ~1e8: Jacobi-preconditioned CG needs far more than the 4000
    iterations the kernel allows, so it stops with AP_ERR_TIMEOUT (lambda
    unchanged, the last iterate returned)."""
    from paper_2308_01957_gb300 import _lib
    lib = _lib.load()
    n = 16384
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[1:] - 1, i[:-1] + 1])
    vals = np.concatenate([np.full(n, 2.0), np.full(n - 1, -1.0), np.full(n - 1, -1.0)])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))])
    # every eigenmode present (an eigenvector alone would converge at once)
    b = np.random.default_rng(3).standard_normal(n)
    rc, status, lam, delta = _call_noalloc(lib, n, row_ptr, cols, vals, b, 1e-12)
    assert rc == 0 and status == _lib.AP_ERR_TIMEOUT
    assert lam == 1e-12
    assert np.all(np.isfinite(delta))


def test_noalloc_repeated_entries_add():
    """Entries repeated at one position add up, on the diagonal as in the
    product: a matrix stored with its diagonal split into two entries gives
    the step of the matrix stored once."""
    from paper_2308_01957_gb300 import _lib
    lib = _lib.load()
    A = np.array([[4.0, 1.0, 0.0], [1.0, 3.0, 0.5], [0.0, 0.5, 2.0]])
    b = np.array([1.0, -2.0, 0.5])
    rows, cols = np.nonzero(A)
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=3))])
    _, s1, _, d1 = _call_noalloc(lib, 3, row_ptr, cols, A[rows, cols], b, 1e-2)
    # the same matrix with every diagonal value stored as two halves
    r2, c2, v2 = [], [], []
    for r in range(3):
        for c in range(3):
            if A[r, c] == 0.0:
                continue
            if r == c:
                r2 += [r, r]; c2 += [c, c]; v2 += [A[r, c] / 2, A[r, c] / 2]
            else:
                r2.append(r); c2.append(c); v2.append(A[r, c])
    rp2 = np.concatenate([[0], np.cumsum(np.bincount(r2, minlength=3))])
    _, s2, _, d2 = _call_noalloc(lib, 3, rp2, c2, v2, b, 1e-2)
    assert s1 == s2 == 0
    M = A + 1e-2 * np.diag(np.diag(A))
    np.testing.assert_allclose(d1, np.linalg.solve(M, b), rtol=1e-9)
    np.testing.assert_allclose(d2, d1, rtol=1e-12)
