"""Shared helpers for the parity tests: problems with oracle-made data, GPU
contexts, and the tolerance rules written in one place."""
import functools
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import astrophot_oracle as O  # noqa: E402
from synthetic import configs  # noqa: E402
from synthetic.problem import attach_data  # noqa: E402

# Tolerances (the stated errors of the path against the FP64 oracle)
TOL_MODEL = 1e-5      # model image: |m_gpu - m| <= TOL_MODEL * max|m|            (mixed)
TOL_CHI2 = 1e-6       # chi^2: relative                                        (mixed)
TOL_GRAD = 1e-4       # gradient and LM step components                        (mixed)
TOL_F64 = 1e-10       # model and chi^2 in the float64 form


def with_data(pr):
    """Attach data/variance made from the oracle's noise-free model at theta_true."""
    attach_data(pr, O.model_images(pr, pr.theta_true))
    return pr


@functools.lru_cache(maxsize=None)
def problem(name, **kw):
    kw = dict(kw)
    if name == "mixed":
        return with_data(configs.mixed_small(**kw))
    if name == "single_sersic":
        return with_data(configs.single_sersic(**kw))
    if name == "cutouts":
        return with_data(configs.cutouts(**kw))
    if name == "crowded":
        return with_data(configs.crowded_field(**kw))
    if name == "field_1k":
        return with_data(configs.field_1k())
    raise KeyError(name)


def grad_scale(pr, theta):
    """Per-component scale 2 sum_p |J_pk| |w_p r_p| of the gradient sum: a
    component that cancels to near zero is compared against the size of the
    terms it sums."""
    s = np.zeros(pr.n_params)
    for J, (r, w) in zip(O.jacobian(pr, theta), O.residuals(pr, theta)):
        s += 2.0 * (abs(J).T @ np.abs(w * r))
    return s


def assert_grad_close(g_gpu, g_ref, scale, tol):
    err = np.abs(g_gpu - g_ref)
    bound = tol * np.maximum(np.abs(g_ref), scale)
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"gradient components {bad[:10]}: gpu {g_gpu[bad[:10]]} ref {g_ref[bad[:10]]} bound {bound[bad[:10]]}"


def damped_matrix(JtWJ, lam):
    d = np.diag(JtWJ).copy()
    dmax = d.max() if d.size else 0.0
    d = np.maximum(d, O.DIAG_FLOOR * dmax if dmax > 0 else 1.0)
    return JtWJ + lam * np.diag(d)


EPS_JACOBIAN_F32 = 2e-6   # relative error of float32 Jacobian columns (float32 profile math, K^2-tap sums)


def assert_step_close(delta, ref, JtWJ, lam, tol, f32_jacobian=False):
    """LM step parity.  With M = J^T W J + lambda D (the damped matrix):
    (1) the error in the energy norm, ||d - d_ref||_M <= tol ||d_ref||_M -- the
        norm in which a step changes the model and chi^2;
    (2) per component |d_k - d_ref_k| <= tol_k max(|d_ref_k|, ||d_ref||_M / sqrt(M_kk)):
        a component is compared with itself or, when it is small, with the
        size the whole step has in that parameter's units.  tol_k = tol, except
        for a float32 Jacobian, whose relative error EPS_JACOBIAN_F32 is
        amplified along near-degenerate directions (Sersic n, Re, Ie) by the
        condition number kappa of the Jacobi-scaled M: there
        tol_k = max(tol, EPS_JACOBIAN_F32 * kappa)."""
    M = damped_matrix(JtWJ, lam)
    e = ref - delta
    en = float(np.sqrt(max(ref @ M @ ref, 0.0)))
    err_m = float(np.sqrt(max(e @ M @ e, 0.0)))
    assert err_m <= tol * en, ("energy-norm error", err_m / en)
    dg = np.sqrt(np.maximum(np.diag(M), 1e-300))
    tol_c = tol
    if f32_jacobian:
        ev = np.linalg.eigvalsh(M / np.outer(dg, dg))
        kappa = ev.max() / max(ev.min(), 1e-300)
        tol_c = max(tol, EPS_JACOBIAN_F32 * kappa)
    bound = tol_c * np.maximum(np.abs(ref), en / dg)
    bad = np.nonzero(np.abs(e) > bound)[0]
    assert bad.size == 0, (tol_c, bad[:8], delta[bad[:8]], ref[bad[:8]], bound[bad[:8]])


def device_context(pr, precision="mixed", tile=None, quad_order=None, jcol="auto"):
    import torch
    from paper_2308_01957_gb300 import api
    ctx = api.Context(precision=precision, quad_order=quad_order or pr.quad_order, device=0, tile=tile, jcol=jcol)
    imgs = api.to_device_images(pr.images)
    ctx.set_problem(imgs, pr.sources, pr.n_params)
    return ctx
