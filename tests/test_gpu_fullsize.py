"""The large workloads at full size, in the configuration bench.py times, and
crops of them small enough for the oracle.

* 256 batched cutouts: the groups are independent, so a few of them are
  cut out as problems of their own and compared with the oracle whole
  (chi^2, gradient, damped step) against the batched launch.
* 4096^2 crowded field and the 12-image joint fit, at full size: model pixels
  sampled one by one by the oracle, chi^2 checked as the weighted residual sum
  of the device model (a property that holds at any size), and sampled
  J^T W J entries against the oracle's Jacobian columns.  Their data and
  variance are seeded maps that do not come from any model (the sampled
  checks use the variance and mask only).
* Crops of the same two workloads that keep their structure (the 51 x 51
  Moffat + wing PSF, the 2 % mask and the source density of the 4096^2 field;
  two rotated, dithered images of different bands sharing shape parameters
  for the joint fit), with data from the oracle: model, chi^2, gradient,
  J^T W J and the damped step element by element against the oracle, in the
  mixed form and in the float64 form.
"""
import numpy as np
import pytest

from _helpers import (O, TOL_CHI2, TOL_F64, TOL_GRAD, TOL_MODEL, assert_grad_close, assert_step_close, configs,
                      device_context, grad_scale, step_envelope, with_data)
from synthetic.problem import ImageSpec
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
        assert_step_close(delta[order], ref, A, lam[gi], TOL_GRAD, f32_jacobian=True,
                          envelope=lambda: step_envelope(sub, th, lam[gi], np.arange(sub.n_params)),
                          label=f"cutouts_256 group {gi}")
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
    assert np.all(np.isfinite(_np(g)))
    assert ctx.status() == 0


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


def _seeded_data(pr, seed):
    """Data and variance for the full-size property checks: seeded maps made
    by the generator alone (no model, neither the library's nor the
    oracle's): variance uniform in [floor, floor + 20], data the floor plus
    Gaussian noise of that variance."""
    rng = np.random.default_rng(seed)
    for im, floor in zip(pr.images, pr.var_floor):
        var = (floor + 20.0 * rng.random((im.H, im.W))).astype(np.float32)
        im.variance = var
        im.data = (floor + np.sqrt(var) * rng.standard_normal((im.H, im.W))).astype(np.float32)
    return pr


def test_crowded_4k_full_size():
    pr = _seeded_data(configs.crowded_4k(), 17)
    _property_checks(pr, pr.theta_init)
    _jtwj_sampled_check(pr, device_context(pr, "mixed"), pr.theta_init)


def test_joint_12x2k_full_size():
    pr = _seeded_data(configs.joint(), 19)
    _property_checks(pr, pr.theta_init)
    # shared shape parameters: entries summed over images and sources
    _jtwj_sampled_check(pr, device_context(pr, "mixed"), pr.theta_init)


# ---------------------------------------------------------------------------
# crops of the large workloads against the oracle
# ---------------------------------------------------------------------------

def crop(pr, image_ids, r0, c0, H, W):
    """The workload on rows r0..r0+H and columns c0..c0+W of the given images:
    the same pixel-scale matrices, origins moved to the crop's corner, PSFs,
    masks and noise cut to the crop, every source whose window meets it (its
    window clipped), parameters renumbered with shared indices kept shared;
    one group."""
    imap, images, noise, floors = {}, [], [], []
    for i in image_ids:
        im = pr.images[i]
        A = np.asarray(im.A, float)
        o = np.asarray(im.origin, float) + A @ np.array([c0, r0], float)
        m = None if im.mask is None else im.mask[r0:r0 + H, c0:c0 + W].copy()
        imap[i] = len(images)
        images.append(ImageSpec(H=H, W=W, A=A, origin=o, psf=im.psf, mask=m, group=0))
        noise.append(pr.noise[i][r0:r0 + H, c0:c0 + W].copy())
        floors.append(pr.var_floor[i])
    pmap, srcs = {}, []
    for s in pr.sources:
        if s.image not in imap:
            continue
        x0, x1, y0, y1 = s.win
        x0, x1, y0, y1 = max(x0 - c0, 0), min(x1 - c0, W), max(y0 - r0, 0), min(y1 - r0, H)
        if x0 >= x1 or y0 >= y1:
            continue
        pidx = s.pidx.copy()
        for k in range(8):
            if pidx[k] >= 0:
                pidx[k] = pmap.setdefault(int(pidx[k]), len(pmap))
        srcs.append(SourceSpec(s.type, imap[s.image], (x0, x1, y0, y1), s.psf_convolve, pidx, s.pfix.copy()))
    order = sorted(pmap, key=pmap.get)
    return Problem(pr.name + "_crop", images, srcs, len(order), pr.theta_true[order], pr.theta_init[order],
                   quad_order=pr.quad_order, noise=noise, var_floor=floors)


def _crop_checks(pr, label):
    """Model, chi^2, gradient, J^T W J and the damped step of the crop
    against the oracle, mixed form and float64 form."""
    theta = pr.theta_init
    ref_models = O.model_images(pr, theta)
    c_ref = O.chi2(pr, theta)
    JtWJ_ref, JtWr_ref = O.normal_equations(pr, theta)
    g_ref = -2.0 * JtWr_ref    # d chi^2 / d theta = -2 J^T W r (pinned against central differences)
    gs = grad_scale(pr, theta)
    lam = 1e-3
    ref_step, _, ok = O.damped_step(JtWJ_ref, JtWr_ref, lam)
    assert ok
    d = np.sqrt(np.maximum(np.diag(JtWJ_ref), 1e-300))
    for prec in ("mixed", "f64"):
        ctx = device_context(pr, prec)
        tol_m = TOL_MODEL if prec == "mixed" else TOL_F64
        for a, b in zip([_np(t) for t in ctx.render(theta)], ref_models):
            assert np.abs(a - b).max() <= tol_m * np.abs(b).max()
        c, g = ctx.eval(theta)
        np.testing.assert_allclose(_np(c), c_ref, rtol=TOL_CHI2 if prec == "mixed" else TOL_F64)
        assert_grad_close(_np(g), g_ref, gs, TOL_GRAD if prec == "mixed" else 1e-8)
        jtwr, csr = ctx.normal_eq(theta)
        JtWJ = ctx.jtwj_dense(csr)
        assert (np.abs(JtWJ - JtWJ_ref) / np.outer(d, d)).max() <= (TOL_GRAD if prec == "mixed" else 1e-9)
        assert_grad_close(_np(jtwr), JtWr_ref, gs / 2, TOL_GRAD if prec == "mixed" else 1e-9)
        delta, _ = ctx.lm_solve(np.array([lam]))
        if prec == "mixed":
            assert_step_close(_np(delta), ref_step, JtWJ_ref, lam, TOL_GRAD, f32_jacobian=True,
                              envelope=lambda: step_envelope(pr, theta, lam, np.arange(pr.n_params)),
                              label=f"{label} mixed")
        else:
            assert_step_close(_np(delta), ref_step, JtWJ_ref, lam, 1e-8, label=f"{label} f64")
        assert ctx.status() == 0
        ctx.close()


def test_crowded_4k_crop_against_oracle():
    """384 x 384 of the 4096^2 field at its centre: the 51 x 51 Moffat + wing
    PSF, the 2 % mask and the field's source density (galaxies whose windows
    reach in from outside included, clipped)."""
    pr = with_data(crop(configs.crowded_4k(), [0], 1856, 1856, 384, 384))
    assert pr.images[0].mask is not None and pr.images[0].psf.shape == (51, 51)
    _crop_checks(pr, "crowded_4k crop 384")


def test_joint_12x2k_crop_against_oracle():
    """512 x 512 at the centre of two images of different bands and epochs
    (each rotated and dithered): galaxy shapes and star positions shared by
    both images, fluxes per band."""
    full = configs.joint()
    pr = with_data(crop(full, [0, 4], 768, 768, 512, 512))
    shared = {int(s.pidx[0]) for s in pr.sources if s.image == 0 and s.type == 0} & \
             {int(s.pidx[0]) for s in pr.sources if s.image == 1 and s.type == 0}
    assert len(shared) >= 5
    _crop_checks(pr, "joint_12x2k crop 2x512")


def test_table1_benchmark_workload_against_oracle():
    """The paper's GPU benchmark (Table 1) at full size with one Sersic (a
    window up to 512 x 512 on the 1000 x 1000 image), data from the oracle at
    the workload's order-7 rendering: chi^2, gradient, J^T W J and the step of
    the order-3 fit against the oracle."""
    import copy
    pr = configs.table1(1)
    gen = copy.copy(pr)
    gen.quad_order = pr.data_quad_order
    attach_data(pr, O.model_images(gen, pr.theta_true))
    _crop_checks(pr, "table1_1")
