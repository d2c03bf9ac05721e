"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every comparison runs the library and the oracle on the same seeded inputs.
Mixed precision is held to the stated errors (model 1e-5 of the peak pixel,
chi^2 1e-6 relative, gradient and LM step 1e-4); the float64 form to 1e-10."""
import math

import numpy as np
import pytest

from _helpers import (O, TOL_CHI2, TOL_F64, TOL_GRAD, TOL_MODEL, assert_grad_close, assert_step_close, configs,
                      damped_matrix, device_context, grad_scale, problem, step_envelope, with_data)

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


CASES = {
    "mixed_rot": dict(name="mixed", seed=configs.SEED_BASE + 21, H=45, W=70, K=7),
    "mixed_multi": dict(name="mixed", seed=configs.SEED_BASE + 22, H=37, W=41, K=9, n_images=3, groups=2),
    "mixed_nopsf": dict(name="mixed", seed=configs.SEED_BASE + 23, H=33, W=29, K=0, mask_frac=0.1),
    "mixed_q1": dict(name="mixed", seed=configs.SEED_BASE + 24, H=40, W=52, K=5, quad_order=1),
    "mixed_q5": dict(name="mixed", seed=configs.SEED_BASE + 25, H=40, W=52, K=11, quad_order=5),
    "mixed_q7_axis": dict(name="mixed", seed=configs.SEED_BASE + 26, H=35, W=35, K=3, quad_order=7, rotate=False),
    "single_sersic": dict(name="single_sersic"),
}


def get_case(key):
    kw = dict(CASES[key])
    return problem(kw.pop("name"), **kw)


@pytest.mark.parametrize("key", list(CASES))
@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_model_parity(key, precision):
    pr = get_case(key)
    ctx = device_context(pr, precision)
    for theta in (pr.theta_true, pr.theta_init):
        ref = O.model_images(pr, theta)
        got = [_np(t) for t in ctx.render(theta)]
        for a, b in zip(got, ref):
            peak = np.abs(b).max()
            tol = TOL_MODEL if precision == "mixed" else TOL_F64
            assert np.abs(a - b).max() <= tol * peak, (np.abs(a - b).max() / peak)
    assert ctx.status() == 0


@pytest.mark.parametrize("key", list(CASES))
@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_chi2_and_gradient_parity(key, precision):
    pr = get_case(key)
    ctx = device_context(pr, precision)
    tol_c = TOL_CHI2 if precision == "mixed" else TOL_F64
    tol_g = TOL_GRAD if precision == "mixed" else 1e-8
    for theta in (pr.theta_true, pr.theta_init):
        c_ref = O.chi2(pr, theta)
        g_ref = O.gradient(pr, theta)
        c, g = ctx.eval(theta)
        c, g = _np(c), _np(g)
        np.testing.assert_allclose(c, c_ref, rtol=tol_c, atol=0)
        assert_grad_close(g, g_ref, grad_scale(pr, theta), tol_g)
    assert ctx.status() == 0


def test_chi2_deterministic():
    pr = get_case("mixed_multi")
    ctx = device_context(pr, "mixed")
    c1, g1 = ctx.eval(pr.theta_init)
    c2, g2 = ctx.eval(pr.theta_init)
    assert torch.equal(c1, c2) and torch.equal(g1, g2)


@pytest.mark.parametrize("key", ["mixed_rot", "mixed_multi", "mixed_nopsf", "single_sersic"])
@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_normal_equations_parity(key, precision):
    pr = get_case(key)
    ctx = device_context(pr, precision)
    theta = pr.theta_init
    JtWJ_ref, JtWr_ref = O.normal_equations(pr, theta)
    jtwr, csr = ctx.normal_eq(theta)
    JtWJ = ctx.jtwj_dense(csr)
    d = np.sqrt(np.maximum(np.diag(JtWJ_ref), 1e-300))
    scale = np.outer(d, d)
    tol = TOL_GRAD if precision == "mixed" else 1e-9
    err = np.abs(JtWJ - JtWJ_ref) / scale
    assert err.max() <= tol, err.max()
    assert_grad_close(_np(jtwr), JtWr_ref, grad_scale(pr, theta) / 2, tol)
    assert ctx.status() == 0


def _normal_eq_checks(pr, ctx, tol=TOL_GRAD):
    theta = pr.theta_init
    JtWJ_ref, JtWr_ref = O.normal_equations(pr, theta)
    jtwr, csr = ctx.normal_eq(theta)
    JtWJ = ctx.jtwj_dense(csr)
    d = np.sqrt(np.maximum(np.diag(JtWJ_ref), 1e-300))
    err = np.abs(JtWJ - JtWJ_ref) / np.outer(d, d)
    assert err.max() <= tol, err.max()
    assert_grad_close(_np(jtwr), JtWr_ref, grad_scale(pr, theta) / 2, tol)
    lam = 1e-3
    delta, _ = ctx.lm_solve(np.full(pr.n_groups, lam))
    pg = pr.param_group()
    for g in range(pr.n_groups):
        idx = np.nonzero(pg == g)[0]
        ref, _, _ = O.damped_step(JtWJ_ref[np.ix_(idx, idx)], JtWr_ref[idx], lam)
        assert_step_close(_np(delta)[idx], ref, JtWJ_ref[np.ix_(idx, idx)], lam, TOL_GRAD, f32_jacobian=True,
                          envelope=lambda: step_envelope(pr, theta, lam, idx), label=f"{pr.name} group {g}")
    assert ctx.status() == 0
    return JtWJ


@pytest.mark.parametrize("key", ["mixed_rot", "mixed_multi", "mixed_q5", "single_sersic"])
def test_normal_equations_fft_mode(key):
    """The FFT mode of the Jacobian-column convolution (64^2 overlap-save
    blocks) held to the direct mode's tolerances against the oracle."""
    pr = get_case(key)
    ctx = device_context(pr, "mixed", jcol="fft")
    assert ctx.jcol_mode()[0] == "fft"
    _normal_eq_checks(pr, ctx)


def test_fft_mode_large_psf_many_blocks():
    """A 51 x 51 PSF (128^2 blocks, 78 outputs per side) on supports that
    span several blocks: FFT mode against the oracle and against the direct
    mode on the device."""
    pr = with_data(configs.crowded_field("fft_k51", configs.SEED_BASE + 71, 150, 170, 3, 8,
                                         configs.psf_moffat(51, 4.0)))
    fft = device_context(pr, "mixed", jcol="fft")
    direct = device_context(pr, "mixed", jcol="direct")
    assert fft.jcol_mode()[0] == "fft" and direct.jcol_mode()[0] == "direct"
    A = _normal_eq_checks(pr, fft)
    _, csr = direct.normal_eq(pr.theta_init)
    B = direct.jtwj_dense(csr)
    d = np.sqrt(np.maximum(np.diag(B), 1e-300))
    # a float32 transform's rounding is relative to the norm of the whole
    # block (2 log2 128 = 14 butterfly levels each way), not to each output
    # as in the direct sum: 2.5e-5 of the entry scale (1.4e-5 observed)
    assert (np.abs(A - B) / np.outer(d, d)).max() <= 2.5e-5


@pytest.mark.parametrize("key", ["mixed_rot", "mixed_multi", "single_sersic"])
@pytest.mark.parametrize("precision", ["mixed", "f64"])
@pytest.mark.parametrize("lam", [1e-3, 1.0])
def test_lm_step_parity(key, precision, lam):
    """One damped step delta from the same (theta, lambda), per group."""
    pr = get_case(key)
    ctx = device_context(pr, precision)
    theta = pr.theta_init
    JtWJ_ref, JtWr_ref = O.normal_equations(pr, theta)
    pg = pr.param_group()
    ctx.normal_eq(theta)
    delta, lam_out = ctx.lm_solve(np.full(pr.n_groups, lam))
    delta = _np(delta)
    tol = TOL_GRAD if precision == "mixed" else 1e-8
    for g in range(pr.n_groups):
        idx = np.nonzero(pg == g)[0]
        sub = JtWJ_ref[np.ix_(idx, idx)]
        ref, _, ok = O.damped_step(sub, JtWr_ref[idx], lam)
        assert ok
        assert_step_close(delta[idx], ref, sub, lam, tol, f32_jacobian=precision == "mixed",
                          envelope=lambda: step_envelope(pr, theta, lam, idx), label=f"{key} {precision} lam {lam} g {g}")
    assert ctx.status() == 0


@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_lm_iterate_matches_oracle_schedule(precision):
    """Five device LM iterations (CUDA graph) against five oracle iterations:
    the accept/reject pattern and the final chi^2 agree."""
    pr = get_case("single_sersic")
    ctx = device_context(pr, precision)
    th_ref, lam_ref, hist = O.lm_iterate(pr, pr.theta_init, np.array([1e-3]), 5)
    th, lam, chi2, log = ctx.lm_iterate(pr.theta_init, np.array([1e-3]), 5, log=True)
    acc_ref = [bool(h[2][0]) for h in hist]
    acc = [bool(r[0, 3]) for r in log]
    assert acc == acc_ref
    c_ref = O.chi2(pr, th_ref)[0]
    assert abs(_np(chi2)[0] - c_ref) <= 1e-4 * c_ref
    np.testing.assert_allclose(_np(th), th_ref, rtol=1e-3, atol=1e-3)
    assert ctx.status() == 0


def test_batched_cutouts_dense_cholesky():
    """Independent cutouts in one launch: chi^2 per group, gradient and the
    per-group dense Cholesky step (workload shape of the batched config,
    reduced in count and size)."""
    pr = with_data(configs.cutouts(n_cut=6, side_lo=40, side_hi=90, max_src=4, name="cutouts_small"))
    ctx = device_context(pr, "mixed")
    theta = pr.theta_init
    c, g = ctx.eval(theta)
    np.testing.assert_allclose(_np(c), O.chi2(pr, theta), rtol=TOL_CHI2)
    assert_grad_close(_np(g), O.gradient(pr, theta), grad_scale(pr, theta), TOL_GRAD)
    JtWJ_ref, JtWr_ref = O.normal_equations(pr, theta)
    ctx.normal_eq(theta)
    lam = np.full(pr.n_groups, 1e-2)
    delta, _ = ctx.lm_solve(lam)
    pg = pr.param_group()
    for gi in range(pr.n_groups):
        idx = np.nonzero(pg == gi)[0]
        sub = JtWJ_ref[np.ix_(idx, idx)]
        ref, _, _ = O.damped_step(sub, JtWr_ref[idx], lam[gi])
        assert_step_close(_np(delta)[idx], ref, sub, lam[gi], TOL_GRAD, f32_jacobian=True,
                          envelope=lambda: step_envelope(pr, theta, lam[gi], idx), label=f"cutouts_small g {gi}")


def test_pcg_group_matches_dense_solve():
    """A group larger than 64 parameters goes through block-Jacobi PCG: it
    solves the device's own damped matrix to 1e-8, and the step matches the
    oracle's dense solve to the LM step tolerance."""
    pr = with_data(configs.crowded_field("crowded_small", configs.SEED_BASE + 31, 160, 192, 6, 18,
                                         configs.psf_moffat(9, 3.0)))
    assert pr.n_params > 64
    ctx = device_context(pr, "mixed")
    theta = pr.theta_init
    JtWJ_ref, JtWr_ref = O.normal_equations(pr, theta)
    jtwr, csr = ctx.normal_eq(theta)
    JtWJ_dev = ctx.jtwj_dense(csr)
    for lam in (1e-3, 1.0):
        delta, _ = ctx.lm_solve(np.array([lam]))
        _, _, cg = ctx.state()
        assert 0 < cg[0] < 4000
        own = np.linalg.solve(damped_matrix(JtWJ_dev, lam), _np(jtwr))
        assert_step_close(_np(delta), own, JtWJ_dev, lam, 1e-8)
        ref, _, ok = O.damped_step(JtWJ_ref, JtWr_ref, lam)
        assert_step_close(_np(delta), ref, JtWJ_ref, lam, TOL_GRAD, f32_jacobian=True,
                          envelope=lambda: step_envelope(pr, theta, lam, np.arange(pr.n_params)),
                          label=f"crowded_small lam {lam}")
    assert ctx.status() == 0


def test_autograd_function_and_fd():
    from paper_2308_01957_gb300 import api
    pr = get_case("mixed_multi")
    ctx = device_context(pr, "f64")
    th = torch.tensor(pr.theta_init, dtype=torch.float64, device="cuda", requires_grad=True)
    c = api.chi2(th, ctx)
    w = torch.arange(1, pr.n_groups + 1, dtype=torch.float64, device="cuda")
    (c * w).sum().backward()
    _, g = ctx.eval(pr.theta_init)
    pg = pr.param_group()
    expect = _np(g) * np.where(pg >= 0, np.arange(1, pr.n_groups + 1)[np.maximum(pg, 0)], 0)
    np.testing.assert_allclose(_np(th.grad), expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())
    # central differences of the device chi^2 (float64 form)
    gd = _np(g)
    for k in range(pr.n_params):
        h = 1e-6 * max(1.0, abs(pr.theta_init[k]))
        tp, tm = pr.theta_init.copy(), pr.theta_init.copy()
        tp[k] += h
        tm[k] -= h
        fd = (_np(ctx.eval(tp, grad=False)[0]).sum() - _np(ctx.eval(tm, grad=False)[0]).sum()) / (2 * h)
        assert abs(fd - gd[k]) <= 1e-5 * max(abs(gd[k]), 1e-3 * np.abs(gd).max()), (k, fd, gd[k])


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def _tiny(H, W, K, sources_fn, mask=None):
    from synthetic.problem import ImageSpec, Problem
    rng = np.random.default_rng(H * 1000 + W)
    psf = None if K == 0 else configs.psf_moffat(K, 2.0)
    im = ImageSpec(H=H, W=W, A=np.eye(2), origin=np.zeros(2), psf=psf, mask=mask, group=0)
    srcs, theta = sources_fn(W, H)
    pr = Problem("tiny", [im], srcs, len(theta), np.asarray(theta, float), np.asarray(theta, float) * 1.01,
                 noise=[rng.standard_normal((H, W)).astype(np.float32)], var_floor=[1.0])
    return with_data(pr)


def _sersic_and_sky(W, H):
    from synthetic.problem import SERSIC, SKY_FLAT, SourceSpec
    p = np.full(8, -1)
    p[:7] = range(7)
    q = np.full(8, -1)
    q[0] = 7
    return ([SourceSpec(SERSIC, 0, (0, W, 0, H), True, p, np.zeros(8)),
             SourceSpec(SKY_FLAT, 0, (0, W, 0, H), False, q, np.zeros(8))],
            [W / 2.0 - 0.3, H / 2.0 + 0.2, 0.6, 0.3, 1.7, 2.5, 5.0, 0.8])


@pytest.mark.parametrize("H,W,K", [(1, 1, 0), (1, 1, 3), (1, 37, 5), (29, 1, 3), (17, 16, 1), (5, 6, 31)])
def test_edge_shapes(H, W, K):
    pr = _tiny(H, W, K, _sersic_and_sky)
    ctx = device_context(pr, "mixed")
    ref = O.model_images(pr, pr.theta_init)[0]
    got = _np(ctx.render(pr.theta_init)[0])
    assert np.abs(got - ref).max() <= TOL_MODEL * np.abs(ref).max()
    c, g = ctx.eval(pr.theta_init)
    assert abs(_np(c)[0] - O.chi2(pr, pr.theta_init)[0]) <= chi2_bound(pr, pr.theta_init)
    assert_grad_close(_np(g), O.gradient(pr, pr.theta_init), grad_scale(pr, pr.theta_init), TOL_GRAD)


def chi2_bound(pr, theta):
    """TOL_CHI2 relative, or -- on images of a handful of pixels, where nothing
    averages -- the change 2 sum w |r| |dm| that a float32 model error of
    |dm| <= 1e-6 |m| causes, whichever is larger."""
    c = O.chi2(pr, theta).sum()
    prop = 0.0
    for im, m in zip(pr.images, O.model_images(pr, theta)):
        w = O.weights(im)
        prop += np.sum(2.0 * w * np.abs(im.data - m) * 1e-6 * np.abs(m))
    return max(TOL_CHI2 * c, prop)


def test_fully_masked_image_has_zero_chi2():
    pr = _tiny(20, 24, 5, _sersic_and_sky, mask=np.ones((20, 24), np.uint8))
    ctx = device_context(pr, "mixed")
    c, g = ctx.eval(pr.theta_init)
    assert _np(c)[0] == 0.0 and np.all(_np(g) == 0.0)


def test_window_outside_image_is_skipped():
    from synthetic.problem import SERSIC, SourceSpec

    def srcs(W, H):
        s, th = _sersic_and_sky(W, H)
        p = np.full(8, -1)
        p[:7] = range(8, 15)
        s.append(SourceSpec(SERSIC, 0, (W + 5, W + 30, 0, H), True, p, np.zeros(8)))
        return s, th + [W + 15.0, H / 2, 0.5, 0.1, 2.0, 3.0, 4.0]
    pr = _tiny(24, 30, 7, srcs)
    ctx = device_context(pr, "mixed")
    c, g = ctx.eval(pr.theta_init)
    np.testing.assert_allclose(_np(c), O.chi2(pr, pr.theta_init), rtol=TOL_CHI2)
    assert np.all(_np(g)[8:] == 0.0)


def test_nonfinite_variance_sets_status():
    pr = _tiny(16, 16, 3, _sersic_and_sky)
    from paper_2308_01957_gb300 import api
    imgs = api.to_device_images(pr.images)
    imgs[0].variance[3, 4] = float("nan")
    ctx = api.Context("mixed", 3)
    ctx.set_problem(imgs, pr.sources, pr.n_params)
    ctx.eval(pr.theta_init)
    assert ctx.status() == 4   # AP_ERR_NONFINITE
    assert ctx.status() == 0   # cleared on read


def test_bad_descriptor_rejected():
    from paper_2308_01957_gb300 import api, _lib
    pr = _tiny(16, 16, 3, _sersic_and_sky)
    imgs = api.to_device_images(pr.images)
    imgs[0].psf = torch.ones((4, 4), dtype=torch.float32, device="cuda")  # even PSF
    ctx = api.Context("mixed", 3)
    with pytest.raises(_lib.ApError) as e:
        ctx.set_problem(imgs, pr.sources, pr.n_params)
    assert e.value.code == 1 and "odd" in str(e.value)


# ---------------------------------------------------------------------------
# the 1024 x 1024 field at full size
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def field():
    return problem("field_1k")


def test_field_1k_full_size(field):
    pr = field
    ctx = device_context(pr, "mixed")
    theta = pr.theta_init
    m = _np(ctx.render(theta)[0])
    rng = np.random.default_rng(0)
    pix = [tuple(x) for x in rng.integers(0, 1024, size=(40, 2))]
    # brightest pixels too: galaxy centres
    for s in pr.sources[:10]:
        x0, x1, y0, y1 = s.win
        pix.append(((y0 + y1) // 2, (x0 + x1) // 2))
    ref = O.model_at(pr, theta, 0, pix)
    peak = m.max()
    got = np.array([m[i, j] for i, j in pix])
    assert np.abs(got - ref).max() <= TOL_MODEL * peak
    c, g = ctx.eval(theta)
    c_ref = O.chi2(pr, theta)
    np.testing.assert_allclose(_np(c), c_ref, rtol=TOL_CHI2)
    g_ref = O.gradient(pr, theta)
    assert_grad_close(_np(g), g_ref, grad_scale(pr, theta), TOL_GRAD)
    assert ctx.status() == 0


def test_grid_pcg_large_group():
    """A group of more than 2048 parameters is solved by the cooperative
    grid-wide PCG: it solves the device's own damped matrix to 1e-8 and
    matches the oracle's dense step to the LM step tolerance."""
    pr = with_data(configs.crowded_field("crowded_grid", configs.SEED_BASE + 41, 384, 384, 60, 560,
                                         configs.psf_moffat(9, 3.0)))
    assert pr.n_params > 2048
    ctx = device_context(pr, "mixed")
    theta = pr.theta_init
    jtwr, csr = ctx.normal_eq(theta)
    JtWJ_dev = ctx.jtwj_dense(csr)
    lam = 1e-2
    delta, _ = ctx.lm_solve(np.array([lam]))
    _, _, cg = ctx.state()
    assert 0 < cg[0] < 4000
    own = np.linalg.solve(damped_matrix(JtWJ_dev, lam), _np(jtwr))
    assert_step_close(_np(delta), own, JtWJ_dev, lam, 1e-8)
    JtWJ_ref, JtWr_ref = O.normal_equations(pr, theta)
    ref = np.linalg.solve(damped_matrix(JtWJ_ref, lam), JtWr_ref)
    assert_step_close(_np(delta), ref, JtWJ_ref, lam, TOL_GRAD, f32_jacobian=True,
                      envelope=lambda: step_envelope(pr, theta, lam, np.arange(pr.n_params)), label="crowded_grid")
    # the same solve inside a graph-captured LM iteration
    th, lam_out, chi2, log = ctx.lm_iterate(theta, np.array([lam]), 1, log=True)
    assert np.isfinite(_np(chi2)).all()
    assert ctx.status() == 0


def _merge_groups(problems):
    """Independent problems side by side as the groups of one problem."""
    from synthetic.problem import Problem, SourceSpec
    images, sources, tt, ti, noise, floors = [], [], [], [], [], []
    for g, pr in enumerate(problems):
        i0, p0 = len(images), len(tt)
        for im in pr.images:
            im.group = g
            images.append(im)
        for s in pr.sources:
            pidx = s.pidx.copy()
            pidx[pidx >= 0] += p0
            sources.append(SourceSpec(s.type, s.image + i0, s.win, s.psf_convolve, pidx, s.pfix.copy()))
        tt.extend(pr.theta_true)
        ti.extend(pr.theta_init)
        noise.extend(pr.noise)
        floors.extend(pr.var_floor)
    return Problem("merged", images, sources, len(tt), np.asarray(tt), np.asarray(ti), noise=noise, var_floor=floors)


def _check_group_solves(pr, lam, distributed):
    """Every group's damped step against a float64 solve of the device's own
    matrix (1e-8: the solver's error alone) and the oracle's step (TOL_GRAD).
    `distributed`: whether the solve must have run the distributed PCG (its
    launches are timed under their own name)."""
    ctx = device_context(pr, "mixed")
    theta = pr.theta_init
    jtwr, csr = ctx.normal_eq(theta)
    JtWJ_dev = ctx.jtwj_dense(csr)
    JtWJ_ref, JtWr_ref = O.normal_equations(pr, theta)
    ctx.set_timing(True)
    ctx.get_timing()
    delta, _ = ctx.lm_solve(lam)
    assert ("lm_solve_dist" in ctx.get_timing()) == distributed
    ctx.set_timing(False)
    _, _, cg = ctx.state()
    pg = pr.param_group()
    for g in range(pr.n_groups):
        idx = np.nonzero(pg == g)[0]
        assert 0 < cg[g] < 4000
        own = np.linalg.solve(damped_matrix(JtWJ_dev[np.ix_(idx, idx)], lam[g]), _np(jtwr)[idx])
        assert_step_close(_np(delta)[idx], own, JtWJ_dev[np.ix_(idx, idx)], lam[g], 1e-8)
        ref, _, _ = O.damped_step(JtWJ_ref[np.ix_(idx, idx)], JtWr_ref[idx], lam[g])
        assert_step_close(_np(delta)[idx], ref, JtWJ_ref[np.ix_(idx, idx)], lam[g], TOL_GRAD, f32_jacobian=True,
                          envelope=lambda: step_envelope(pr, theta, lam[g], idx), label=f"{pr.name} group {g}")
    assert ctx.status() == 0


def test_pcg_groups_in_clusters():
    """A few groups of more than 64 parameters: each group's PCG is spread
    over the CTAs of one thread-block cluster, all groups in one launch."""
    parts = [with_data(configs.crowded_field(f"g{k}", configs.SEED_BASE + 60 + k, 96, 112, 3, 16,
                                             configs.psf_moffat(7, 3.0))) for k in range(5)]
    assert all(p.n_params > 64 for p in parts)
    _check_group_solves(_merge_groups(parts), np.array([1e-3, 1e-2, 1e-1, 1.0, 3e-3]), True)


def test_many_pcg_groups_one_cta_each():
    """Forty groups of 65 parameters, enough to fill the GPU: each group's
    PCG runs in one CTA (the batched path for many medium groups)."""
    parts = [with_data(configs.crowded_field(f"h{k}", configs.SEED_BASE + 100 + k, 64, 72, 2, 16,
                                             configs.psf_moffat(7, 3.0))) for k in range(40)]
    assert all(p.n_params > 64 for p in parts)
    lam = np.geomspace(1e-4, 10.0, len(parts))
    _check_group_solves(_merge_groups(parts), lam, False)


def _multiband(tag, seed, side, n_sersic, n_star):
    """A small joint fit: 4 bands of one epoch, each galaxy's shape shared
    with a flux per band (10 parameters), each star's position shared with a
    flux per band (6): preconditioner blocks of whole objects, past 8."""
    return with_data(configs.joint(seed=configs.SEED_BASE + seed, n_band=4, n_epoch=1, side=side, n_sersic=n_sersic,
                                   n_star=n_star, K=9, name=tag))


def test_pcg_object_blocks_in_a_cluster():
    """Block-Jacobi PCG whose blocks are whole multi-band objects (10 and 6
    parameters) in one group spread over a thread-block cluster."""
    pr = _multiband("mb_cluster", 120, 96, 6, 12)
    assert pr.n_params > 64
    _check_group_solves(pr, np.array([1e-4]), True)


def test_pcg_object_blocks_one_cta_each():
    """The same object blocks in the one-CTA PCG of many medium groups."""
    parts = [_multiband(f"mb{k}", 130 + k, 48, 3, 5) for k in range(40)]
    assert all(p.n_params > 64 for p in parts)
    lam = np.geomspace(1e-5, 1.0, len(parts))
    _check_group_solves(_merge_groups(parts), lam, False)


def _lm_paths(pr, lam0, n, precision="mixed"):
    """The same n LM iterations three ways: n calls of one iteration (every
    iteration evaluates the model at theta), one call of n (later iterations
    reuse an accepted trial's model), and one iteration + lm_continue(n - 1)."""
    ctx = device_context(pr, precision)
    lam = np.full(pr.n_groups, lam0)
    th, lm = pr.theta_init, lam
    logs = []
    for _ in range(n):
        th, lm, c_a, lg = ctx.lm_iterate(th, lm, 1, log=True)
        logs.append(lg[0])
    a = (_np(th), _np(c_a), np.array(logs))
    th_b, _, c_b, log_b = ctx.lm_iterate(pr.theta_init, lam, n, log=True)
    b = (_np(th_b), _np(c_b), log_b)
    _, _, _, log_c0 = ctx.lm_iterate(pr.theta_init, lam, 1, log=True)
    th_c, _, c_c, log_c1 = ctx.lm_continue(n - 1, log=True)
    c = (_np(th_c), _np(c_c), np.concatenate([log_c0, log_c1]))
    assert ctx.status() == 0
    return ctx, a, b, c


def _same_trajectory(a, b):
    (th_a, c_a, log_a), (th_b, c_b, log_b) = a, b
    np.testing.assert_array_equal(log_a[:, :, 3], log_b[:, :, 3])          # accept / reject per iteration
    np.testing.assert_allclose(log_b[:, :, :2], log_a[:, :, :2], rtol=1e-12)  # chi^2 before and at the trial
    np.testing.assert_allclose(c_b, c_a, rtol=1e-12)
    np.testing.assert_allclose(th_b, th_a, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("key", ["mixed_multi", "cutouts"])
def test_lm_reuses_accepted_trial(key):
    """An accepted trial's model, residual and chi^2 serve as the next
    iteration's current point: the trajectory is the one that evaluates the
    model at theta in every iteration, with accepts and rejects both taken."""
    if key == "cutouts":
        pr = with_data(configs.cutouts(n_cut=6, side_lo=40, side_hi=90, max_src=4, name="cutouts_small"))
    else:
        pr = get_case(key)
    _, a, b, c = _lm_paths(pr, 1e-9, 8)
    flags = a[2][:, :, 3]
    assert flags.max() == 1.0 and flags.min() == 0.0, flags
    _same_trajectory(a, b)
    _same_trajectory(a, c)


def test_lm_continue_after_other_evaluations():
    """ap_eval / ap_normal_eq between LM calls overwrite the forward buffers:
    the continued fit then evaluates at its theta again."""
    pr = get_case("mixed_rot")
    ctx, a, _, _ = _lm_paths(pr, 1e-3, 4, "f64")
    lam = np.full(pr.n_groups, 1e-3)
    ctx.lm_iterate(pr.theta_init, lam, 2)
    ctx.eval(pr.theta_true)
    ctx.normal_eq(pr.theta_init * (1.0 + 1e-3))
    th, _, c, log = ctx.lm_continue(2, log=True)
    np.testing.assert_array_equal(log[:, :, 3], a[2][2:, :, 3])
    np.testing.assert_allclose(_np(c), a[1], rtol=1e-12)
    np.testing.assert_allclose(_np(th), a[0], rtol=1e-10, atol=1e-12)


def test_lm_continue_needs_a_started_fit():
    from paper_2308_01957_gb300._lib import ApError
    pr = get_case("single_sersic")
    ctx = device_context(pr, "mixed")
    with pytest.raises(ApError):
        ctx.lm_continue(1)


# Every correlation tile variant, forced, against the oracle: the autotuner
# may pick any of them on another problem or GPU.  The PSF sizes reach a
# register-window specialisation (K = 5: 2 chunks of 4 taps; K = 25: 7) and
# the generic tile code (K = 35: 9 chunks); the image spans several tiles of
# every variant with ragged edges.
VARIANT_KS = (5, 25, 35)


@pytest.fixture(scope="module")
def variant_table():
    from paper_2308_01957_gb300 import api
    ctx = api.Context("mixed", 3, device=0)
    _, shapes, _ = ctx.conv_variant()
    ctx.close()
    return shapes


@pytest.mark.parametrize("K", VARIANT_KS)
@pytest.mark.parametrize("variant", range(7))
def test_forced_tile_variant_parity(variant, K, variant_table):
    assert len(variant_table) == 7
    pr = problem("mixed", seed=configs.SEED_BASE + 40 + K, H=75, W=141, K=K)
    from paper_2308_01957_gb300 import api
    ctx = api.Context("mixed", pr.quad_order, device=0, jcol="direct", conv_variant=variant)
    ctx.set_problem(api.to_device_images(pr.images), pr.sources, pr.n_params)
    assert ctx.conv_variant()[0] == variant
    theta = pr.theta_init
    ref = O.model_images(pr, theta)
    got = [_np(t) for t in ctx.render(theta)]
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() <= TOL_MODEL * np.abs(b).max()
    c, g = ctx.eval(theta)
    np.testing.assert_allclose(_np(c), O.chi2(pr, theta), rtol=TOL_CHI2, atol=0)
    assert_grad_close(_np(g), O.gradient(pr, theta), grad_scale(pr, theta), TOL_GRAD)
    JtWJ_ref, JtWr_ref = O.normal_equations(pr, theta)
    jtwr, csr = ctx.normal_eq(theta)
    JtWJ = ctx.jtwj_dense(csr)
    d = np.sqrt(np.maximum(np.diag(JtWJ_ref), 1e-300))
    assert (np.abs(JtWJ - JtWJ_ref) / np.outer(d, d)).max() <= TOL_GRAD
    assert_grad_close(_np(jtwr), JtWr_ref, grad_scale(pr, theta) / 2, TOL_GRAD)
    assert ctx.status() == 0


# small crowded fields whose tiles span the column classes of the Gram
# kernels: (H, W, Sersics, stars, seed offset), tiles per class
TILE_FIELDS = {
    "sparse": (128, 192, 6, 30, 80),   # 36 tiles of at most 32 columns, 60 of 33-64
    "graded": (96, 160, 12, 20, 72),   # 22 of 33-64, 38 of 65-96
    "packed": (64, 96, 16, 12, 83),    # 7 of 65-96, 16 of 97-128, 1 past 128
    "dense": (64, 72, 40, 12, 71),     # 20 of 219-288
}


@pytest.mark.parametrize("tc_min", [1, 257, 0])
@pytest.mark.parametrize("field", list(TILE_FIELDS))
def test_jtwj_every_tile_column_class(field, tc_min):
    """J^T W J for tiles of every column class: the tensor-core kernel's
    forms for up to 32, 64 and 128 columns, and the warp-MMA kernel with one
    and with two shared-memory column blocks (past 96 columns); entry by entry
    against the oracle, and the damped step; every tile it can on the
    tensor-core kernel (tc_min 1), every tile on the warp-MMA kernel (257),
    and the threshold the planner times (0)."""
    from paper_2308_01957_gb300 import api
    H, W, ns, nm, seed = TILE_FIELDS[field]
    pr = with_data(configs.crowded_field(f"{field}_tiles", configs.SEED_BASE + seed, H, W, ns, nm,
                                         configs.psf_moffat(5, 2.5)))
    ctx = api.Context("mixed", pr.quad_order, device=0, gram_tc_min=tc_min)
    ctx.set_problem(api.to_device_images(pr.images), pr.sources, pr.n_params)
    _normal_eq_checks(pr, ctx)


def test_jtwj_pairs_over_many_tiles():
    """The per-pair sums over tiles in each of their three forms: a 768^2
    field (2304 tiles) whose sky meets every tile (sky x sky: one CTA per
    entry past 2048 tiles), large galaxies meeting hundreds of tiles (one warp
    per entry) and stars meeting a few (one warp per pair); J^T W J entry by
    entry against the oracle, and the damped step."""
    from paper_2308_01957_gb300 import api
    pr = with_data(configs.crowded_field("sky_tiles", configs.SEED_BASE + 76, 768, 768, 4, 6,
                                         configs.psf_moffat(5, 2.5)))
    ctx = api.Context("mixed", pr.quad_order, device=0)
    ctx.set_problem(api.to_device_images(pr.images), pr.sources, pr.n_params)
    _normal_eq_checks(pr, ctx)


@pytest.mark.parametrize("tc_min", [1, 257])
def test_jtwj_both_gram_kernels_on_mixed_problems(tc_min):
    """The two tile-Gram kernels on the small mixed problems (rotated, several
    images and groups, every profile): J^T W J and the step against the oracle."""
    from paper_2308_01957_gb300 import api
    for key in ("mixed_rot", "mixed_multi"):
        pr = get_case(key)
        ctx = api.Context("mixed", pr.quad_order, device=0, gram_tc_min=tc_min)
        ctx.set_problem(api.to_device_images(pr.images), pr.sources, pr.n_params)
        _normal_eq_checks(pr, ctx)


# Pixel-centred sampling with the interpolated re-shift (Sec. "PSF convolution")
SHIFT_CASES = ["mixed_rot", "mixed_multi", "mixed_q5", "single_sersic"]


@pytest.mark.parametrize("key", SHIFT_CASES)
@pytest.mark.parametrize("method", ["lanczos3", "bilinear"])
@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_shifted_model_and_chi2_parity(key, method, precision):
    pr = get_case(key)
    ctx = device_context(pr, precision)
    code = {"lanczos3": O.SHIFT_LANCZOS3, "bilinear": O.SHIFT_BILINEAR}[method]
    theta = pr.theta_init
    layers = O.model_layers_shifted(pr, theta, code)
    c, models = ctx.eval_shifted(theta, method, model=True)
    tol = TOL_MODEL if precision == "mixed" else TOL_F64
    for got, L in zip(models, layers):
        ref = L["m"]
        assert np.abs(_np(got) - ref).max() <= tol * np.abs(ref).max()
    np.testing.assert_allclose(_np(c), O.chi2_shifted(pr, theta, code), rtol=TOL_CHI2 if precision == "mixed" else TOL_F64)
    # the ordinary evaluation after it is unaffected (true-centre sampling)
    c2, _ = ctx.eval(theta)
    np.testing.assert_allclose(_np(c2), O.chi2(pr, theta), rtol=TOL_CHI2 if precision == "mixed" else TOL_F64)
    assert ctx.status() == 0


def test_psf_star_every_path():
    """The PSF-star model on its own image (with a galaxy and a sky): model,
    chi^2, gradient, J^T W J and the step against the oracle."""
    pr = get_case("mixed_rot")
    assert any(s.type == O.PSF_STAR for s in pr.sources)
    ctx = device_context(pr, "mixed")
    theta = pr.theta_init
    for a, b in zip([_np(t) for t in ctx.render(theta)], O.model_images(pr, theta)):
        assert np.abs(a - b).max() <= TOL_MODEL * np.abs(b).max()
    _normal_eq_checks(pr, ctx)


# Live PSF parameters (Sec. "PSF convolution"; the PSF-extraction example)
LIVE_CASES = {
    "live_rot": dict(seed=configs.SEED_BASE + 81, H=38, W=44, K=9, live_psf=True),
    "live_multi": dict(seed=configs.SEED_BASE + 82, H=33, W=37, K=7, live_psf=True, n_images=3, groups=2),
}


@pytest.mark.parametrize("key", list(LIVE_CASES))
@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_live_psf_parity(key, precision):
    """A circular Moffat PSF whose (n, Rd) are fitted and shared with the
    image's Moffat stars: model, chi^2, gradient (including d/d(n, Rd)
    through every galaxy's convolution), J^T W J and the damped step."""
    pr = problem("mixed", **LIVE_CASES[key])
    assert all(im.psf_pidx is not None for im in pr.images)
    ctx = device_context(pr, precision)
    theta = pr.theta_init
    tol_m = TOL_MODEL if precision == "mixed" else TOL_F64
    for a, b in zip([_np(t) for t in ctx.render(theta)], O.model_images(pr, theta)):
        assert np.abs(a - b).max() <= tol_m * np.abs(b).max()
    c, g = ctx.eval(theta)
    np.testing.assert_allclose(_np(c), O.chi2(pr, theta), rtol=TOL_CHI2 if precision == "mixed" else TOL_F64)
    assert_grad_close(_np(g), O.gradient(pr, theta), grad_scale(pr, theta), TOL_GRAD if precision == "mixed" else 1e-8)
    JtWJ_ref, JtWr_ref = O.normal_equations(pr, theta)
    jtwr, csr = ctx.normal_eq(theta)
    JtWJ = ctx.jtwj_dense(csr)
    d = np.sqrt(np.maximum(np.diag(JtWJ_ref), 1e-300))
    assert (np.abs(JtWJ - JtWJ_ref) / np.outer(d, d)).max() <= (TOL_GRAD if precision == "mixed" else 1e-9)
    lam = 1e-3
    delta, _ = ctx.lm_solve(np.full(pr.n_groups, lam))
    pg = pr.param_group()
    for gi in range(pr.n_groups):
        idx = np.nonzero(pg == gi)[0]
        ref, _, _ = O.damped_step(JtWJ_ref[np.ix_(idx, idx)], JtWr_ref[idx], lam)
        if precision == "mixed":
            assert_step_close(_np(delta)[idx], ref, JtWJ_ref[np.ix_(idx, idx)], lam, TOL_GRAD, f32_jacobian=True,
                              envelope=lambda: step_envelope(pr, theta, lam, idx), label=f"{key} group {gi}")
        else:
            assert_step_close(_np(delta)[idx], ref, JtWJ_ref[np.ix_(idx, idx)], lam, 1e-8, label=f"{key} f64 g {gi}")
    assert ctx.status() == 0


def test_live_psf_lm_iterations_follow_the_oracle():
    """Three LM iterations with the live PSF in the fit: the accept pattern
    and the final chi^2 follow the oracle's."""
    pr = problem("mixed", **LIVE_CASES["live_rot"])
    ctx = device_context(pr, "f64")
    th_ref, _, hist = O.lm_iterate(pr, pr.theta_init, np.array([1e-3]), 3)
    th, lam, chi2, log = ctx.lm_iterate(pr.theta_init, np.array([1e-3]), 3, log=True)
    assert [bool(r[0, 3]) for r in log] == [bool(h[2][0]) for h in hist]
    c_ref = O.chi2(pr, th_ref)[0]
    assert abs(_np(chi2)[0] - c_ref) <= 1e-8 * c_ref
    assert ctx.status() == 0
