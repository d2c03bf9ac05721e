"""The large workloads at full size, in the configuration bench.py times.

* 256 batched cutouts: the groups are independent, so a few of them are
  cut out as problems of their own and compared with the oracle whole
  (chi^2, gradient, damped step) against the batched launch.
* 4096^2 crowded field and the 12-image joint fit: model pixels sampled one
  by one by the oracle, chi^2 checked as the weighted residual sum of the
  device model (a property that holds at any size), the mixed-precision
  gradient against directional central differences of the float64 form, and
  sampled J^T W J entries against the oracle's Jacobian columns.
"""
import numpy as np
import pytest

from _helpers import (O, TOL_CHI2, TOL_GRAD, TOL_MODEL, assert_grad_close, assert_step_close, configs,
                      device_context, grad_scale, with_data)
from synthetic.problem import Problem, SourceSpec, attach_data

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


def sub_problem(pr, groups):
    """The cutouts of the given groups as a problem of their own (parameters
    renumbered, images re-indexed)."""
    img_map = {}
    images = []
    for i, im in enumerate(pr.images):
        if im.group in groups:
            img_map[i] = len(images)
            images.append(im)
    pmap = {}
    sources = []
    for s in pr.sources:
        if s.image not in img_map:
            continue
        pidx = s.pidx.copy()
        for k in range(8):
            if pidx[k] >= 0:
                pidx[k] = pmap.setdefault(int(pidx[k]), len(pmap))
        sources.append(SourceSpec(s.type, img_map[s.image], s.win, s.psf_convolve, pidx, s.pfix.copy()))
    order = sorted(pmap, key=pmap.get)
    out = Problem("sub", images, sources, len(order), pr.theta_true[order], pr.theta_init[order],
                  noise=[pr.noise[i] for i in img_map], var_floor=[pr.var_floor[i] for i in img_map])
    return out, order


@pytest.fixture(scope="module")
def cutouts():
    pr = configs.cutouts()
    # data from the oracle, cutout by cutout (every group is independent)
    models = [None] * len(pr.images)
    for g in range(pr.n_groups):
        sub, _ = sub_problem(pr, {g})
        models[g] = O.model_images(sub, sub.theta_true)[0]
    attach_data(pr, models)
    return pr


def test_cutouts_256_full_size(cutouts):
    pr = cutouts
    ctx = device_context(pr, "mixed")
    theta = pr.theta_init
    c, g = ctx.eval(theta)
    c, g = _np(c), _np(g)
    jtwr, csr = ctx.normal_eq(theta)
    lam = np.full(pr.n_groups, 1e-2)
    delta, _ = ctx.lm_solve(lam)
    delta = _np(delta)
    rng = np.random.default_rng(7)
    for gi in sorted(rng.choice(pr.n_groups, size=6, replace=False)):
        sub, order = sub_problem(pr, {gi})
        th = theta[order]
        c_ref = O.chi2(sub, th).sum()   # the sub-problem keeps its group id
        assert abs(c[gi] - c_ref) <= TOL_CHI2 * c_ref
        assert_grad_close(g[order], O.gradient(sub, th), grad_scale(sub, th), TOL_GRAD)
        A, b = O.normal_equations(sub, th)
        ref, _, _ = O.damped_step(A, b, lam[gi])
        assert_step_close(delta[order], ref, A, lam[gi], TOL_GRAD, f32_jacobian=True)
    assert ctx.status() == 0


def _sampled_model_check(pr, ctx, theta, n_pix=24, seed=3):
    models = ctx.render(theta)
    rng = np.random.default_rng(seed)
    for ii in rng.choice(len(pr.images), size=min(3, len(pr.images)), replace=False):
        im = pr.images[ii]
        m = _np(models[ii])
        pix = [tuple(p) for p in rng.integers(0, [im.H, im.W], size=(n_pix, 2))]
        # and the brightest sampled region: a few galaxy centres on this image
        for s in [s for s in pr.sources if s.image == ii and s.type == 0][:6]:
            x0, x1, y0, y1 = s.win
            pix.append(((y0 + y1) // 2, (x0 + x1) // 2))
        ref = O.model_at(pr, theta, ii, pix)
        got = np.array([m[i, j] for i, j in pix])
        assert np.abs(got - ref).max() <= TOL_MODEL * max(m.max(), np.abs(ref).max())
    return models


def _property_checks(pr, theta):
    ctx = device_context(pr, "mixed")
    models = _sampled_model_check(pr, ctx, theta)
    c, g = ctx.eval(theta)
    # chi^2 is the weighted residual sum of the device model, per group
    ref = np.zeros(pr.n_groups)
    for im, m in zip(pr.images, models):
        var = im.variance.astype(np.float64)
        w = np.where(im.mask == 1, 0.0, 1.0 / var) if im.mask is not None else 1.0 / var
        ref[im.group] += np.sum(w * (im.data.astype(np.float64) - _np(m)) ** 2)
    np.testing.assert_allclose(_np(c), ref, rtol=TOL_CHI2)
    # mixed gradient against the float64 form and its directional derivative
    ctx64 = device_context(pr, "f64")
    c64, g64 = ctx64.eval(theta)
    g, g64 = _np(g), _np(g64)
    bound = TOL_GRAD * np.maximum(np.abs(g64), 1e-3 * np.abs(g64).max())
    ratio = np.abs(g - g64) / bound
    worst = np.argsort(ratio)[-5:]
    assert ratio.max() <= 1.0, [(int(k), g[k], g64[k], ratio[k]) for k in worst]
    rng = np.random.default_rng(11)
    for _ in range(2):
        v = rng.standard_normal(pr.n_params) * np.maximum(np.abs(theta), 1.0) * 1e-7
        fd = (_np(ctx64.eval(theta + v, grad=False)[0]).sum() - _np(ctx64.eval(theta - v, grad=False)[0]).sum()) / 2
        assert abs(fd - g64 @ v) <= 1e-4 * (np.abs(g64) @ np.abs(v))
    assert ctx.status() == 0 and ctx64.status() == 0


def _jtwj_sampled_check(pr, ctx, theta, n_rows=10, seed=5):
    """Sampled J^T W J entries (the diagonal and a random stored column of
    random rows) against the oracle's Jacobian columns of the sources that
    reference them: entry (p, q) = sum over images and pixels of w J_p J_q,
    J_p the sum of the columns of every (source, slot) that holds p.  Sky
    parameters (whole-image columns) are left out of the sample."""
    import collections
    jtwr, (row_ptr, col_idx, vals) = ctx.normal_eq(theta)
    vals = _np(vals)
    refs = collections.defaultdict(list)
    for si, s in enumerate(pr.sources):
        for k in range(8):
            if s.pidx[k] >= 0 and s.type not in (4, 5):
                refs[int(s.pidx[k])].append((si, k))
    weights = {}
    for ii, im in enumerate(pr.images):
        var = im.variance.astype(np.float64)
        weights[ii] = np.where(im.mask == 1, 0.0, 1.0 / var) if im.mask is not None else 1.0 / var
    cache = {}

    def cols(si):
        if si not in cache:
            cache[si] = O.source_jacobian(pr, pr.sources[si], theta)
        return cache[si]

    def entry(p, q):
        tot = 0.0
        for sa, ka in refs[p]:
            for sb, kb in refs[q]:
                ia = pr.sources[sa].image
                if ia != pr.sources[sb].image:
                    continue
                (a0, a1, b0, b1), Ca = cols(sa)
                (c0_, c1_, d0, d1), Cb = cols(sb)
                r0, r1, x0, x1 = max(a0, c0_), min(a1, c1_), max(b0, d0), min(b1, d1)
                if r0 >= r1 or x0 >= x1:
                    continue
                ja = Ca[ka][r0 - a0:r1 - a0, x0 - b0:x1 - b0]
                jb = Cb[kb][r0 - c0_:r1 - c0_, x0 - d0:x1 - d0]
                tot += float(np.sum(weights[ia][r0:r1, x0:x1] * ja * jb))
        return tot

    rng = np.random.default_rng(seed)
    rows = rng.choice(sorted(refs), size=min(n_rows, len(refs)), replace=False)
    checked = 0
    for p in rows:
        e0, e1 = int(row_ptr[p]), int(row_ptr[p + 1])
        cand = [e for e in range(e0, e1) if int(col_idx[e]) in refs]
        picks = {e for e in range(e0, e1) if col_idx[e] == p} | set(rng.choice(cand, size=min(2, len(cand)), replace=False).tolist())
        for e in picks:
            q = int(col_idx[e])
            ref = entry(p, q)
            scale = np.sqrt(max(entry(p, p), 0.0) * max(entry(q, q), 0.0))
            assert abs(vals[e] - ref) <= TOL_GRAD * scale, (p, q, vals[e], ref, scale)
            checked += 1
    assert checked >= n_rows


def _device_rendered_data(pr):
    """Data for the property checks: the float64 device render at the true
    parameters plus the workload's seeded noise (var = model + floor).  It is
    no oracle input: the oracle's sampled pixels depend on theta only."""
    for im in pr.images:
        im.data = np.zeros((im.H, im.W), np.float32)
        im.variance = np.ones((im.H, im.W), np.float32)
    ctx = device_context(pr, "f64")
    models = [_np(m) for m in ctx.render(pr.theta_true)]
    ctx.close()
    attach_data(pr, models)
    return pr


def test_crowded_4k_full_size():
    pr = _device_rendered_data(configs.crowded_4k())
    _property_checks(pr, pr.theta_init)
    _jtwj_sampled_check(pr, device_context(pr, "mixed"), pr.theta_init)


def test_joint_12x2k_full_size():
    pr = _device_rendered_data(configs.joint())
    _property_checks(pr, pr.theta_init)
    # shared shape parameters: entries summed over images and sources
    _jtwj_sampled_check(pr, device_context(pr, "mixed"), pr.theta_init)
