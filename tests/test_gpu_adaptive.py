"""Parity of the adaptive pixel integration (Sec. "Pixel Integration") on the
GPU, through the C ABI, with the oracle's same scheme.

Each sample's level is a decision taken by comparing floating-point values
with a budget; where the oracle finds a decision within a small margin of its
threshold (`near`), the GPU may take the other branch, and both results are
then valid: the levels must agree everywhere else, the values must agree to
the path's tolerance where the levels agree and to twice the budget where they
do not."""
import math

import numpy as np
import pytest

from _helpers import O, TOL_CHI2, TOL_MODEL, configs, device_context, problem, with_data
from synthetic.problem import (EXPONENTIAL, GAUSSIAN, MOFFAT, SERSIC, SKY_FLAT, SKY_PLANE, ImageSpec, Problem,
                               SourceSpec)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_01957_gb300 import build
    build()


NEAR_ABS = {"mixed": 5e-5, "f64": 1e-12}
TOL_VAL = {"mixed": TOL_MODEL, "f64": 1e-10}
ROT = 1.07 * np.array([[math.cos(0.35), -math.sin(0.35)], [math.sin(0.35), math.cos(0.35)]])


def _single(type_, params, H=24, W=28):
    im = ImageSpec(H=H, W=W, A=ROT, origin=np.array([0.4, -0.3]), psf=None, group=0)
    pidx = np.full(8, -1, dtype=np.int64)
    pidx[: len(params)] = range(len(params))
    src = SourceSpec(type_, 0, (0, W, 0, H), False, pidx, np.zeros(8))
    pr = Problem(f"single_{type_}", [im], [src], len(params), np.asarray(params, float), np.asarray(params, float),
                 quad_order=3, noise=[np.random.default_rng(7).normal(0, 1, (H, W)).astype(np.float32)],
                 var_floor=[1.0])
    return with_data(pr)


SINGLES = {
    "sersic_cusp": (SERSIC, [13.2, 11.7, 0.6, 0.7, 3.5, 2.0, 6.0]),
    "sersic_half": (SERSIC, [12.1, 12.9, 0.8, 2.2, 0.6, 3.0, 4.0]),
    "exponential": (EXPONENTIAL, [14.3, 10.6, 0.5, -0.4, 2.5, 5.0]),
    "gaussian": (GAUSSIAN, [12.8, 12.2, 0.7, 0.3, 1.1, 300.0]),
    "moffat": (MOFFAT, [13.6, 11.4, 1.0, 0.0, 3.0, 1.6, 500.0]),
}


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _check(pr, precision, tol, theta=None):
    theta = pr.theta_init if theta is None else theta
    ctx = device_context(pr, precision)
    res = ctx.eval_adaptive(theta, tol=tol, model=True, levels=True, counts=True)
    assert ctx.status() == 0
    n, off = ctx.adaptive_layout()
    lev_gpu = _np(res["levels"]).astype(np.int64)
    layers = O.model_layers_adaptive(pr, theta, tol, 0.01, NEAR_ABS[precision])
    bound = 0.0          # summed |difference| the level mismatches allow
    n_mis = 0
    hist = np.zeros(4, dtype=np.int64)
    for L in layers:
        for k, (box, vals, lev, near) in L["sources"].items():
            src = pr.sources[k]
            if src.type in (SKY_FLAT, SKY_PLANE) or vals.size == 0:
                assert off[k] == -1
                continue
            g = lev_gpu[off[k]: off[k] + vals.size].reshape(vals.shape)
            hist += np.bincount(g.ravel(), minlength=4)[:4]
            mis = g != lev
            assert not (mis & ~near).any(), (k, np.argwhere(mis & ~near)[:5], g[mis & ~near][:5], lev[mis & ~near][:5])
            R, C = np.meshgrid(np.arange(box[0], box[1]), np.arange(box[2], box[3]), indexing="ij")
            e = tol * abs(O.rect_values(pr, src, theta, R, C, 0.0, 0.0, 1.0, 1).sum()) / vals.size
            bound += 2.0 * e * mis.sum()
            n_mis += int(mis.sum())
    assert hist.sum() == n
    cnt = res["counts"]
    np.testing.assert_array_equal(cnt[:4], hist)
    for im_k, (L, m_gpu) in enumerate(zip(layers, res["model"])):
        m_ref = L["m"]
        peak = np.abs(m_ref).max()
        err = np.abs(_np(m_gpu) - m_ref).max()
        assert err <= TOL_VAL[precision] * peak + bound, (im_k, err, peak, bound)
    c_ref = np.zeros(pr.n_groups)
    for im, L in zip(pr.images, layers):
        r = np.asarray(im.data, dtype=np.float64) - L["m"]
        c_ref[im.group] += float((O.weights(im) * r * r).sum())
    c_gpu = _np(res["chi2"])
    rtol = (TOL_CHI2 if precision == "mixed" else 1e-10) if n_mis == 0 else 1e-3
    np.testing.assert_allclose(c_gpu, c_ref, rtol=rtol)
    return res, layers


@pytest.mark.parametrize("case", list(SINGLES))
@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_adaptive_single_source(case, precision):
    type_, params = SINGLES[case]
    pr = _single(type_, params)
    res, layers = _check(pr, precision, 0.01, theta=pr.theta_true)
    if case == "sersic_cusp":
        assert res["counts"][3] > 0 and res["counts"][4] > 0     # the cusp reaches the deepest level


@pytest.mark.parametrize("precision,tol", [("mixed", 0.01), ("f64", 0.01), ("mixed", 1e-3)])
def test_adaptive_with_psf_and_sky(precision, tol):
    """Several sources, PSF convolution of the galaxies, a plane sky, a
    rotated pixel grid, two images in two groups."""
    pr = problem("mixed", seed=configs.SEED_BASE + 22, H=37, W=41, K=9, n_images=2, groups=2, psf_star=False)
    res, _ = _check(pr, precision, tol)
    assert res["counts"][1] > 0 and res["counts"][2] + res["counts"][3] > 0


def test_adaptive_field_crop_many_tiles():
    """A 192 x 192 crop of the 1024 x 1024 benchmark field (its source density,
    25 x 25 PSF): many render tiles, ragged edges, every level used."""
    import bench
    pr = with_data(bench.crop_problem(configs.field_1k(), [0], 0, 0, 192, 192))
    res, _ = _check(pr, "mixed", 0.01)
    assert (res["counts"][:4] > 0).all()


@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_adaptive_limits(precision):
    """A budget too large to refine anything is the midpoint rule (the fixed
    order-1 render); a zero budget sends (nearly) every pixel to the deepest
    level, where the scheme is composite order 7 on 125 x 125 pieces."""
    pr = _single(*SINGLES["gaussian"], H=12, W=13)
    ctx = device_context(pr, precision)
    big = ctx.eval_adaptive(pr.theta_true, tol=1e30, model=True, levels=True, counts=True)
    assert (_np(big["levels"]) == 0).all()
    ctx1 = device_context(pr, precision, quad_order=1)
    mid = ctx1.render(pr.theta_true)[0]
    rtol = 1e-6 if precision == "mixed" else 1e-13
    np.testing.assert_allclose(_np(big["model"][0]), _np(mid), rtol=rtol, atol=rtol * float(mid.abs().max()))
    zero, _ = _check(pr, precision, 0.0, theta=pr.theta_true)
    # in float the criteria of the faintest pixels can round to exactly 0 and
    # stop there (the parity check above accepts those as rounding-level ties)
    assert zero["counts"][3] >= (0.99 if precision == "f64" else 0.8) * zero["counts"][:4].sum()


def test_adaptive_rejects_bad_budget():
    from paper_2308_01957_gb300._lib import ApError
    pr = _single(*SINGLES["gaussian"], H=8, W=8)
    ctx = device_context(pr, "mixed")
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(ApError):
            ctx.eval_adaptive(pr.theta_true, tol=bad)


def test_adaptive_refuses_psf_star():
    """The adaptive scheme covers the analytic profiles; a problem holding a
    PSF star is refused with AP_ERR_ARG before any work."""
    from paper_2308_01957_gb300 import _lib
    pr = problem("mixed", seed=configs.SEED_BASE + 23, H=30, W=33, K=5)
    assert any(s.type == O.PSF_STAR for s in pr.sources)
    ctx = device_context(pr, "mixed")
    with pytest.raises(_lib.ApError) as e:
        ctx.eval_adaptive(pr.theta_init, tol=0.01)
    assert e.value.code == _lib.AP_ERR_ARG
