"""Pins of the CPU oracle to things other than itself: closed forms, special
cases, brute force, library routines of other functions, finite differences.

Each test names what a plausible mistake in the oracle would break."""
import json
import math
import os

import numpy as np
import pytest
from scipy import special

from oracle import astrophot_oracle as O
from synthetic import configs
from synthetic.problem import (EXPONENTIAL, GAUSSIAN, MOFFAT, SERSIC, SKY_FLAT, SKY_PLANE,
                               ImageSpec, Problem, SourceSpec, attach_data)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pidx(*i):
    out = np.full(8, -1, dtype=np.int64)
    out[: len(i)] = i
    return out


def one_source_problem(type_, params, H=64, W=64, A=None, origin=None, psf=None, win=None, conv=False,
                       Q=3, pfix=None, free=None):
    A = np.eye(2) if A is None else np.asarray(A, dtype=np.float64)
    origin = np.zeros(2) if origin is None else np.asarray(origin, dtype=np.float64)
    im = ImageSpec(H=H, W=W, A=A, origin=origin, psf=psf, group=0)
    n = len(params)
    pidx = _pidx(*range(n)) if free is None else free
    src = SourceSpec(type_, 0, (0, W, 0, H) if win is None else win, conv, pidx,
                     np.zeros(8) if pfix is None else pfix)
    return Problem("t", [im], [src], n, np.asarray(params, float), np.asarray(params, float), quad_order=Q,
                   noise=[np.zeros((H, W), np.float32)], var_floor=[1.0])


# ---------------------------------------------------------------------------
# b_n
# ---------------------------------------------------------------------------

def test_bn_half_is_ln2():
    # P(1, b) = 1 - exp(-b) = 1/2  =>  b = ln 2 exactly
    assert abs(O.sersic_b(0.5) - math.log(2.0)) < 1e-14


def test_bn_exponential_by_bisection():
    # n = 1: P(2, b) = 1 - (1 + b) e^-b = 1/2, solved by plain bisection
    lo, hi = 0.5, 3.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (1.0 + mid) * math.exp(-mid) > 0.5:
            lo = mid
        else:
            hi = mid
    assert abs(O.sersic_b(1.0) - 0.5 * (lo + hi)) < 1e-13


@pytest.mark.parametrize("n", [0.36, 0.7, 1.3, 2.5, 4.0, 6.0, 8.0])
def test_bn_residual_and_high_precision(n):
    b = O.sersic_b(n)
    assert abs(special.gammainc(2 * n, b) - 0.5) < 1e-14
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    f = lambda x: mpmath.gammainc(2 * n, 0, x, regularized=True) - mpmath.mpf(1) / 2
    ref = mpmath.findroot(f, b)
    assert abs(b - float(ref)) < 1e-12 * b


def test_bn_ciotti_bertin_asymptotic():
    # Ciotti & Bertin (1999) series, accurate for large n
    for n in (4.0, 6.0, 8.0):
        cb = 2 * n - 1 / 3 + 4 / (405 * n) + 46 / (25515 * n ** 2) + 131 / (1148175 * n ** 3)
        assert abs(O.sersic_b(n) - cb) < 1e-5


@pytest.mark.parametrize("n", [0.4, 0.5, 1.0, 2.5, 5.0, 7.9])
def test_db_dn_against_finite_difference(n):
    h = 1e-5 * n
    fd = (O.sersic_b(n + h) - O.sersic_b(n - h)) / (2 * h)
    assert abs(O.sersic_db_dn(n) - fd) < 1e-7 * abs(fd)


# ---------------------------------------------------------------------------
# quadrature
# ---------------------------------------------------------------------------

def test_gauss_legendre_degree_from_paper():
    """Order-Q rule on a pixel: exact for x^a y^b up to per-axis degree 2Q-1,
    not exact at 2Q (the paper's footnote)."""
    facts = json.load(open(os.path.join(GOLDEN, "pixel_integration.json")))["facts"]
    rng = np.random.default_rng(0)
    for row in facts["gauss_legendre_orders"]:
        Q, deg = row["order"], row["exact_degree"]
        assert Q * Q == row["evaluations_per_pixel"]
        sx, sy = rng.uniform(0.5, 2.0, 2)
        im = ImageSpec(H=4, W=4, A=np.diag([sx, sy]), origin=np.array([0.3, -0.7]))
        i, j = 2, 1
        x, y, W2 = O.node_coords(im, np.array([float(i)]), np.array([float(j)]), Q)
        xa, xb = 0.3 + sx * j, 0.3 + sx * (j + 1)
        ya, yb = -0.7 + sy * i, -0.7 + sy * (i + 1)
        for a in range(deg + 1):
            b = min(deg, a)
            exact = ((xb ** (a + 1) - xa ** (a + 1)) / (a + 1)) * ((yb ** (b + 1) - ya ** (b + 1)) / (b + 1))
            quad = sx * sy * np.sum(W2 * x[0, 0] ** a * y[0, 0] ** b)
            assert abs(quad - exact) < 1e-11 * max(1.0, abs(exact))
        # degree 2Q: the centred monomial (x - xm)^(2Q) is no longer exact
        xm = 0.5 * (xa + xb)
        exact = sy * (xb - xa) ** (deg + 2) / ((deg + 2) * 2 ** (deg + 1))
        quad = sx * sy * np.sum(W2 * (x[0, 0] - xm) ** (deg + 1))
        assert abs(quad - exact) > 1e-3 * exact


def _brute(problem, src, theta, S=64):
    """Sub-pixel midpoint integration with S x S sub-samples per pixel."""
    im = problem.images[src.image]
    u = (np.arange(S) + 0.5) / S * 2.0 - 1.0      # sub-pixel centres on [-1, 1]
    r0, r1, c0, c1 = O.source_box(problem, src)
    out = np.zeros((r1 - r0, c1 - c0))
    p = O.slot_values(src, theta)
    A = np.asarray(im.A)
    for i in range(r0, r1):
        for j in range(c0, c1):
            uu = j + 0.5 + 0.5 * u[:, None]
            vv = i + 0.5 + 0.5 * u[None, :]
            x = im.origin[0] + A[0, 0] * uu + A[0, 1] * vv
            y = im.origin[1] + A[1, 0] * uu + A[1, 1] * vv
            I, _ = O.profile(src.type, p, x, y, im, False)
            out[i - r0, j - c0] = O.det_A(im) * I.mean()
    return out


def test_midpoint_fails_and_gl3_meets_budget():
    """Steep Sersic (n = 4, Re = 2 px): the midpoint is off by more than 20 %
    on the centre pixel; Q = 3 meets the per-pixel budget e = 0.01 F / N on
    every pixel but the few central ones the adaptive pass would refine, and
    Q = 7 converges towards the brute-force integral."""
    facts = json.load(open(os.path.join(GOLDEN, "pixel_integration.json")))["facts"]
    params = [8.0, 8.0, 0.8, 0.3, 4.0, 2.0, 1.0]
    pr1 = one_source_problem(SERSIC, params, H=16, W=16, Q=1)
    pr3 = one_source_problem(SERSIC, params, H=16, W=16, Q=3)
    pr7 = one_source_problem(SERSIC, params, H=16, W=16, Q=7)
    src = pr3.sources[0]
    brute = _brute(pr3, src, pr3.theta_true)
    m1 = O.render_source(pr1, src, pr1.theta_true)[1]
    m3 = O.render_source(pr3, src, pr3.theta_true)[1]
    m7 = O.render_source(pr7, src, pr7.theta_true)[1]
    c = np.unravel_index(np.argmax(brute), brute.shape)
    assert abs(m1[c] - brute[c]) / brute[c] > facts["midpoint_error_fraction_at_least"]
    budget = facts["image_accuracy_fraction"] * brute.sum() / brute.size
    bad = np.argwhere(np.abs(m3 - brute) > budget)
    assert len(bad) <= 4
    assert all(max(abs(b[0] - c[0]), abs(b[1] - c[1])) <= 1 for b in bad)
    assert np.abs(m7 - brute).max() < np.abs(m3 - brute).max()


def test_brute_force_smooth_profile_agrees_tightly():
    # a smooth, wide Gaussian on a rotated, skewed grid: Q = 3 vs 64 x 64 brute force
    A = np.array([[0.9, 0.2], [-0.3, 1.1]])
    pr = one_source_problem(GAUSSIAN, [1.0, 2.0, 0.7, 0.4, 3.0, 100.0], H=12, W=12, A=A,
                            origin=np.array([-6.0, -5.0]))
    src = pr.sources[0]
    brute = _brute(pr, src, pr.theta_true)
    m3 = O.render_source(pr, src, pr.theta_true)[1]
    assert np.abs(m3 - brute).max() < 1e-3 * brute.max()


# ---------------------------------------------------------------------------
# profiles: closed forms and special cases
# ---------------------------------------------------------------------------

def sersic_total_flux(n, Re, q, Ie):
    b = special.gammaincinv(2 * n, 0.5)
    return 2 * math.pi * n * Ie * Re * Re * q * math.exp(b) * special.gamma(2 * n) / b ** (2 * n)


@pytest.mark.parametrize("n,Re,tol", [(0.5, 6.0, 2e-9), (1.0, 6.0, 1e-6), (2.0, 4.0, 1e-6)])
def test_sersic_total_flux_closed_form(n, Re, tol):
    """Summed pixels of a Sersic on a rotated, scaled grid vs the closed form
    2 pi n Ie Re^2 q e^b Gamma(2n) / b^(2n).  The 5 x 5 pixels around the
    centre, where the cusp of n >= 1 profiles defeats any fixed-order rule, are
    integrated by 256 x 256 sub-pixel brute force (n >= 1); the rest use the oracle's
    Q = 3 rule.  The tail outside the image is bounded with the upper
    incomplete gamma.  For n = 1/2 the tolerance covers the shift b eps^2/Re^2
    of the radius regularisation."""
    q, Ie = 0.6, 3.0
    half = 190 if n < 2 else 250
    A = 1.3 * np.array([[math.cos(0.3), -math.sin(0.3)], [math.sin(0.3), math.cos(0.3)]])
    H = W = 2 * half
    origin = -A @ np.array([W / 2.0, H / 2.0])
    pr = one_source_problem(SERSIC, [0.21, -0.37, q, 1.1, n, Re, Ie], H=H, W=W, A=A, origin=origin)
    src = pr.sources[0]
    vals = O.render_source(pr, src, pr.theta_true)[1]
    uc, vc = np.linalg.solve(A, np.array([0.21, -0.37]) - origin)
    ic, jc = int(vc), int(uc)
    box = (ic - 2, ic + 3, jc - 2, jc + 3)
    S = 256
    u = (np.arange(S) + 0.5) / S
    p = O.slot_values(src, pr.theta_true)
    for i in range(box[0], box[1] if n >= 1 else box[0]):
        for j in range(box[2], box[3]):
            uu = j + u[:, None] + 0 * u[None, :]
            vv = i + u[None, :] + 0 * u[:, None]
            x = origin[0] + A[0, 0] * uu + A[0, 1] * vv
            y = origin[1] + A[1, 0] * uu + A[1, 1] * vv
            I, _ = O.profile(SERSIC, p, x, y, pr.images[0], False)
            vals[i, j] = O.det_A(pr.images[0]) * I.mean()
    tot = vals.sum()
    exact = sersic_total_flux(n, Re, q, Ie)
    # light beyond the ellipse that fits inside the image
    Rmax = 1.3 * (half - 1) * q
    b = special.gammaincinv(2 * n, 0.5)
    tail = special.gammaincc(2 * n, b * (Rmax / Re) ** (1 / n))
    assert tail < 0.1 * tol
    assert abs(tot - exact) < tol * exact


def test_sersic_half_is_gaussian():
    """Sersic n = 1/2 equals a Gaussian with sigma^2 = Re^2 / (2 ln 2) and the
    matching total flux (links the two profile formulas)."""
    rng = np.random.default_rng(1)
    x = rng.uniform(-10, 10, 200)
    y = rng.uniform(-10, 10, 200)
    im = ImageSpec(H=1, W=1, A=np.eye(2), origin=np.zeros(2))
    Re, q, PA, Ie = 3.0, 0.6, 0.8, 2.0
    Is, _ = O.profile(SERSIC, np.array([0.5, -0.2, q, PA, 0.5, Re, Ie]), x, y, im, False)
    sig = Re / math.sqrt(2 * math.log(2))
    F = sersic_total_flux(0.5, Re, q, Ie)
    Ig, _ = O.profile(GAUSSIAN, np.array([0.5, -0.2, q, PA, sig, F]), x, y, im, False)
    np.testing.assert_allclose(Is, Ig, rtol=1e-8)
    # and the Gaussian is its textbook form along the major axis
    X = np.array([1.0, 2.0, 3.0])
    Ix, _ = O.profile(GAUSSIAN, np.array([0.0, 0.0, q, 0.0, sig, F]), X, 0 * X, im, False)
    np.testing.assert_allclose(Ix, F / (2 * math.pi * sig * sig * q) * np.exp(-X ** 2 / (2 * sig * sig)), rtol=1e-14)


def test_exponential_is_sersic_n1():
    rng = np.random.default_rng(2)
    x, y = rng.uniform(-8, 8, (2, 100))
    im = ImageSpec(H=1, W=1, A=np.eye(2), origin=np.zeros(2))
    Ie, _ = O.profile(EXPONENTIAL, np.array([0.1, 0.2, 0.5, 0.3, 4.0, 2.0]), x, y, im, False)
    Is, _ = O.profile(SERSIC, np.array([0.1, 0.2, 0.5, 0.3, 1.0, 4.0, 2.0]), x, y, im, False)
    np.testing.assert_allclose(Ie, Is, rtol=1e-15)
    # e^(-b R / Re) form with b = 1.678...: the exponential profile
    b1 = O.sersic_b(1.0)
    R = np.sqrt(x * x + y * y)
    Ic, _ = O.profile(EXPONENTIAL, np.array([0.0, 0.0, 1.0, 0.0, 4.0, 2.0]), x, y, im, False)
    np.testing.assert_allclose(Ic, 2.0 * np.exp(-b1 * (R / 4.0 - 1.0)), rtol=1e-7)


@pytest.mark.parametrize("type_,params", [
    (MOFFAT, [0.3, -0.4, 0.7, 0.5, 3.5, 2.0, 50.0]),
    (GAUSSIAN, [0.3, -0.4, 0.7, 0.5, 2.0, 50.0]),
])
def test_point_source_total_flux_is_F(type_, params):
    """The Moffat and Gaussian are normalised so their integral is F.  At
    Q = 7 the quadrature error on a 2-px core is below 1e-6; the Moffat tail
    beyond the image, (1 + r^2/Rd^2)^(1-n) at r = 70, is ~2e-8."""
    H = W = 200
    origin = np.array([-100.0, -100.0])
    pr = one_source_problem(type_, params, H=H, W=W, origin=origin, Q=7)
    tot = O.render_source(pr, pr.sources[0], pr.theta_true)[1].sum()
    assert abs(tot - params[-1]) < 1e-6 * params[-1]


def test_moffat_fwhm():
    """Moffat FWHM = 2 Rd sqrt(2^(1/n) - 1) (definition of the core radius)."""
    im = ImageSpec(H=1, W=1, A=np.eye(2), origin=np.zeros(2))
    n, Rd = 3.0, 1.5 / math.sqrt(2 ** (1 / 3) - 1)
    I0, _ = O.profile(MOFFAT, np.array([0, 0, 1, 0, n, Rd, 1.0]), np.array([0.0]), np.array([0.0]), im, False)
    Ih, _ = O.profile(MOFFAT, np.array([0, 0, 1, 0, n, Rd, 1.0]), np.array([1.5]), np.array([0.0]), im, False)
    assert abs(Ih[0] / I0[0] - 0.5) < 1e-14


def test_pa_orientation():
    """PA counter-clockwise from +x: a source at PA = pi/2 has its major axis
    along +y, so it is brighter at (0, 2) than at (2, 0)."""
    im = ImageSpec(H=1, W=1, A=np.eye(2), origin=np.zeros(2))
    I, _ = O.profile(GAUSSIAN, np.array([0, 0, 0.5, math.pi / 2, 1.0, 1.0]), np.array([0.0, 2.0]),
                     np.array([2.0, 0.0]), im, False)
    assert I[0] > 100 * I[1]


def test_symmetry_pa_plus_pi_and_point_reflection():
    p = [12.0, 10.0, 0.55, 0.7, 2.2, 3.0, 4.0]
    pr = one_source_problem(SERSIC, p, H=20, W=24)
    a = O.render_source(pr, pr.sources[0], pr.theta_true)[1]
    p2 = list(p)
    p2[3] += math.pi
    b = O.render_source(pr, pr.sources[0], np.asarray(p2))[1]
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14 * a.max())
    # centred on the image centre (a pixel corner): point reflection symmetry
    np.testing.assert_allclose(a, a[::-1, ::-1], rtol=1e-11, atol=1e-13 * a.max())


def test_sky_plane_pixel_values():
    """Plane sky integrates exactly: pixel value = |det A| x plane at the centre."""
    A = np.array([[1.2, 0.1], [0.0, 0.9]])
    pr = one_source_problem(SKY_PLANE, [2.0, 0.01, -0.02], H=5, W=7, A=A, origin=np.array([3.0, 1.0]))
    m = O.render_source(pr, pr.sources[0], pr.theta_true)[1]
    im = pr.images[0]
    xc, yc = np.array([3.0, 1.0]) + A @ np.array([3.5, 2.5])
    for i in range(5):
        for j in range(7):
            x, y = np.array([3.0, 1.0]) + A @ np.array([j + 0.5, i + 0.5])
            assert abs(m[i, j] - O.det_A(im) * (2.0 + 0.01 * (x - xc) - 0.02 * (y - yc))) < 1e-13
    pf = one_source_problem(SKY_FLAT, [2.0], H=5, W=7, A=A)
    np.testing.assert_allclose(O.render_source(pf, pf.sources[0], pf.theta_true)[1], 2.0 * O.det_A(im), rtol=1e-14)


# ---------------------------------------------------------------------------
# PSF convolution
# ---------------------------------------------------------------------------

def test_convolution_orientation_delta():
    """A unit impulse at image pixel (i0, j0) convolved with an asymmetric PSF
    puts P[ty, tx] at (i0 + ty - h, j0 + tx - h): a true (flipped) convolution."""
    rng = np.random.default_rng(3)
    K, h, H, W = 5, 2, 11, 13
    P = rng.random((K, K))
    G = np.zeros((H + 2 * h, W + 2 * h))
    i0, j0 = 4, 6
    G[i0 + h, j0 + h] = 1.0
    M = O.convolve_layer(G, P, H, W)
    for ty in range(K):
        for tx in range(K):
            assert M[i0 + ty - h, j0 + tx - h] == P[ty, tx]
    assert np.count_nonzero(M) == K * K


def test_gaussian_conv_gaussian():
    """Point-sampled (Q = 1) Gaussian sigma1 convolved with a sampled Gaussian
    PSF sigma2 equals the sampled Gaussian of variance sigma1^2 + sigma2^2.
    By Poisson summation the discrete sum differs by aliasing terms of order
    exp(-2 pi^2 s1^2 s2^2 / (s1^2 + s2^2)) ~ 1e-27 here, and the PSF
    truncation at h = 8 sigma2 costs exp(-32)."""
    s1, s2, K, F = 2.5, 2.5, 41, 100.0
    H = W = 64
    c = (K - 1) / 2
    yy, xx = np.mgrid[0:K, 0:K]
    psf = np.exp(-((xx - c) ** 2 + (yy - c) ** 2) / (2 * s2 * s2))
    pr = one_source_problem(GAUSSIAN, [32.0, 32.0, 1.0, 0.0, s1, F], H=H, W=W, psf=psf, conv=True, Q=1,
                            win=(12, 52, 12, 52))
    M = O.model_layers(pr, pr.theta_true)[0]["M"]
    s2t = s1 * s1 + s2 * s2
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    ref = F / (2 * math.pi * s2t) * np.exp(-((xx - 32.0) ** 2 + (yy - 32.0) ** 2) / (2 * s2t))
    np.testing.assert_allclose(M, ref, rtol=0, atol=1e-13 * ref.max())


def test_flux_conservation_normalised_psf():
    rng = np.random.default_rng(4)
    psf = rng.random((9, 9)).astype(np.float32) + 0.1
    pr = one_source_problem(SERSIC, [30.0, 28.0, 0.7, 0.2, 1.5, 3.0, 2.0], H=60, W=60, psf=psf, conv=True,
                            win=(14, 46, 12, 44))
    L = O.model_layers(pr, pr.theta_true)[0]
    assert abs(L["M"].sum() - L["G"].sum()) < 1e-12 * L["G"].sum()


# ---------------------------------------------------------------------------
# chi^2, gradient, Jacobian, normal equations, LM
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def mixed():
    pr = configs.mixed_small(H=30, W=38, K=7)
    attach_data(pr, O.model_images(pr, pr.theta_true))
    return pr


@pytest.fixture(scope="module")
def mixed_multi():
    pr = configs.mixed_small(seed=configs.SEED_BASE + 12, H=26, W=31, K=5, n_images=3, groups=2)
    attach_data(pr, O.model_images(pr, pr.theta_true))
    return pr


def test_chi2_definition_and_mask(mixed):
    im = mixed.images[0]
    m = O.model_images(mixed, mixed.theta_init)[0]
    keep = im.mask == 0
    direct = np.sum(((im.data.astype(float) - m) ** 2 / im.variance.astype(float))[keep])
    assert abs(O.chi2(mixed, mixed.theta_init)[0] - direct) < 1e-12 * direct
    # changing a masked pixel's data changes nothing
    d0 = im.data.copy()
    i, j = np.argwhere(im.mask == 1)[0]
    im.data[i, j] += 1e6
    try:
        assert O.chi2(mixed, mixed.theta_init)[0] == pytest.approx(direct, rel=1e-14)
    finally:
        im.data[:] = d0


def test_chi2_expectation_at_truth():
    pr = configs.single_sersic()
    attach_data(pr, O.model_images(pr, pr.theta_true))
    N = pr.images[0].H * pr.images[0].W
    c = O.chi2(pr, pr.theta_true)[0]
    assert abs(c - N) < 4 * math.sqrt(2 * N)


def test_nonfinite_variance_rejected(mixed):
    im = mixed.images[0]
    v0 = im.variance.copy()
    i, j = np.argwhere(im.mask == 0)[0]
    im.variance[i, j] = 0.0
    try:
        with pytest.raises(ValueError):
            O.chi2(mixed, mixed.theta_true)
    finally:
        im.variance[:] = v0


def _fd_gradient(pr, theta, rel=1e-6):
    g = np.zeros_like(theta)
    for k in range(theta.size):
        h = rel * max(1.0, abs(theta[k]))
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        g[k] = (O.chi2(pr, tp).sum() - O.chi2(pr, tm).sum()) / (2 * h)
    return g


@pytest.mark.parametrize("which", ["mixed", "mixed_multi"])
def test_gradient_matches_central_fd(which, request):
    pr = request.getfixturevalue(which)
    th = pr.theta_init
    g = O.gradient(pr, th)
    fd = _fd_gradient(pr, th)
    scale = np.abs(g).max()
    np.testing.assert_allclose(g, fd, rtol=2e-6, atol=2e-7 * scale)


def test_jacobian_columns_match_fd(mixed):
    th = mixed.theta_init
    J = O.jacobian(mixed, th)[0].toarray()
    for k in range(th.size):
        h = 1e-6 * max(1.0, abs(th[k]))
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        col = (O.model_images(mixed, tp)[0] - O.model_images(mixed, tm)[0]).ravel() / (2 * h)
        np.testing.assert_allclose(J[:, k], col, rtol=1e-5, atol=1e-7 * max(np.abs(col).max(), 1e-30))


def test_normal_equations_properties(mixed_multi):
    pr = mixed_multi
    JtWJ, JtWr = O.normal_equations(pr, pr.theta_init)
    assert np.allclose(JtWJ, JtWJ.T, rtol=0, atol=1e-12 * np.abs(JtWJ).max())
    ev = np.linalg.eigvalsh(JtWJ)
    assert ev.min() > -1e-10 * ev.max()
    np.testing.assert_allclose(-2 * JtWr, O.gradient(pr, pr.theta_init), rtol=1e-12, atol=1e-9)
    # groups do not couple
    pg = pr.param_group()
    assert np.all(JtWJ[np.ix_(pg == 0, pg == 1)] == 0)


def test_shared_parameter_chi2_is_sum_of_images(mixed_multi):
    pr = mixed_multi
    tot = O.chi2(pr, pr.theta_init)
    per = []
    for im, m in zip(pr.images, O.model_images(pr, pr.theta_init)):
        per.append((im.group, np.sum(O.weights(im) * (im.data - m) ** 2)))
    for g in range(pr.n_groups):
        assert tot[g] == pytest.approx(sum(v for gg, v in per if gg == g), rel=1e-13)


def test_cholesky_against_library():
    rng = np.random.default_rng(5)
    B = rng.standard_normal((9, 9))
    M = B @ B.T + 0.1 * np.eye(9)
    np.testing.assert_allclose(O.cholesky_lower(M), np.linalg.cholesky(M), rtol=1e-12, atol=1e-13)
    M[3, 3] = -1.0
    assert O.cholesky_lower(M) is None


def test_lm_linear_case_lands_on_least_squares():
    """With only the linear parameters free (intensities, fluxes, sky), one
    nearly undamped LM step reaches the exact weighted least-squares optimum,
    found here with a library least-squares solve on finite-difference columns."""
    base = configs.mixed_small(seed=configs.SEED_BASE + 13, H=28, W=33, K=5, mask_frac=0.0)
    attach_data(base, O.model_images(base, base.theta_true))
    linear = []
    for s in base.sources:
        slots = {SERSIC: [6], EXPONENTIAL: [5], GAUSSIAN: [5], MOFFAT: [6], SKY_FLAT: [0], SKY_PLANE: [0, 1, 2],
                 O.PSF_STAR: [2]}[s.type]
        linear += [int(s.pidx[k]) for k in slots if s.pidx[k] >= 0]
    linear = sorted(set(linear))
    # freeze the nonlinear slots at their true values by moving them to pfix
    new_index = {p: n for n, p in enumerate(linear)}
    for s in base.sources:
        for k in range(O.N_SLOTS[s.type]):
            p = int(s.pidx[k])
            if p < 0:
                continue
            if p in new_index:
                s.pidx[k] = new_index[p]
            else:
                s.pfix[k] = base.theta_true[p]
                s.pidx[k] = -1
    th0 = base.theta_init[linear]
    base.n_params = len(linear)
    base.theta_true = base.theta_true[linear]
    base.theta_init = th0
    JtWJ, JtWr = O.normal_equations(base, th0)
    delta, _, ok = O.damped_step(JtWJ, JtWr, 1e-14)
    assert ok
    # least squares on finite-difference columns (the model is linear here)
    im = base.images[0]
    m0 = O.model_images(base, th0)[0].ravel()
    cols = []
    for k in range(th0.size):
        t = th0.copy()
        t[k] += 1.0
        cols.append(O.model_images(base, t)[0].ravel() - m0)
    Jfd = np.stack(cols, 1)
    sw = np.sqrt(O.weights(im).ravel())
    sol, *_ = np.linalg.lstsq(Jfd * sw[:, None], (im.data.ravel() - m0) * sw, rcond=None)
    np.testing.assert_allclose(th0 + delta, th0 + sol, rtol=1e-8, atol=1e-10)


def test_lm_reduces_chi2_monotonically():
    pr = configs.single_sersic()
    attach_data(pr, O.model_images(pr, pr.theta_true))
    th, lam, hist = O.lm_iterate(pr, pr.theta_init, np.array([1e-3]), 6)
    best = [h[0][0] for h in hist]
    assert all(b2 <= b1 for b1, b2 in zip(best, best[1:]))
    assert O.chi2(pr, th)[0] < best[0]


def test_model_at_matches_full_render(mixed):
    pr = mixed
    m = O.model_images(pr, pr.theta_init)[0]
    pix = [(0, 0), (5, 7), (pr.images[0].H - 1, pr.images[0].W - 1), (13, 20)]
    np.testing.assert_allclose(O.model_at(pr, pr.theta_init, 0, pix), [m[i, j] for i, j in pix], rtol=1e-12,
                               atol=1e-13 * np.abs(m).max())


def test_damped_step_limits():
    """lambda -> 0: the Gauss-Newton solution of the normal equations;
    lambda -> infinity: a gradient step scaled by 1/(lambda D)."""
    rng = np.random.default_rng(6)
    B = rng.standard_normal((30, 6)) * np.array([1.0, 10.0, 0.1, 3.0, 1.0, 100.0])
    M = B.T @ B
    r = rng.standard_normal(6)
    d0, _, ok = O.damped_step(M, r, 1e-14)
    assert ok
    np.testing.assert_allclose(d0, np.linalg.solve(M, r), rtol=1e-8)
    lam = 1e8
    d1, _, _ = O.damped_step(M, r, lam)
    np.testing.assert_allclose(d1 * lam, r / np.diag(M), rtol=1e-5)


# ---------------------------------------------------------------------------
# Parameter box and LM schedule (Sec. "Optimization methods"; readings: the
# box the paper clips initial values to holds during the fit; strict accept,
# lambda / 9 on accept, lambda * 11 on reject with theta kept)
# ---------------------------------------------------------------------------

def test_param_bounds_box_by_hand():
    """The box written out slot by slot for every profile type, and a shared
    index taking the intersection of its slots' boxes.  A wrong bound (a
    Moffat n floor, the q ceiling, a radius floor on the wrong slot) fails."""
    im = ImageSpec(H=8, W=8, A=np.eye(2), origin=np.zeros(2), group=0)
    z = np.zeros(8)
    srcs = [SourceSpec(SERSIC, 0, (0, 8, 0, 8), False, _pidx(0, 1, 2, 3, 4, 5, 6), z),
            SourceSpec(EXPONENTIAL, 0, (0, 8, 0, 8), False, _pidx(7, 8, 9, 10, 11, 12), z),
            SourceSpec(GAUSSIAN, 0, (0, 8, 0, 8), False, _pidx(13, 14, 15, 16, 17, 18), z),
            SourceSpec(MOFFAT, 0, (0, 8, 0, 8), False, _pidx(19, 20, 21, 22, 23, 24, 25), z),
            SourceSpec(SKY_FLAT, 0, (0, 8, 0, 8), False, _pidx(26), z),
            SourceSpec(SKY_PLANE, 0, (0, 8, 0, 8), False, _pidx(27, 28, 29), z),
            # a second Moffat sharing its n with the Sersic n, and its q with the Gaussian sigma
            SourceSpec(MOFFAT, 0, (0, 8, 0, 8), False, _pidx(30, 31, 17, 32, 4, 33, 34), z)]
    pr = Problem("box", [im], srcs, 35, np.ones(35), np.ones(35), noise=[np.zeros((8, 8), np.float32)],
                 var_floor=[1.0])
    lo, hi = O.param_bounds(pr)
    inf = np.inf
    want = {2: (0.05, 1.0), 4: (1.05, 8.0), 5: (1e-3, inf),            # Sersic q, n (shared), Re
            9: (0.05, 1.0), 11: (1e-3, inf),                            # exponential q, Re
            15: (0.05, 1.0), 17: (0.05, 1.0),                           # Gaussian q, sigma (shared with a q)
            21: (0.05, 1.0), 23: (1.05, 50.0), 24: (1e-3, inf),         # Moffat q, n, Rd
            33: (1e-3, inf)}                                            # second Moffat Rd
    for p in range(35):
        a, b = want.get(p, (-inf, inf))
        assert lo[p] == a and hi[p] == b, (p, lo[p], hi[p], a, b)


def _flat_sky_problem(H, W, A, data, var):
    im = ImageSpec(H=H, W=W, A=np.asarray(A, float), origin=np.zeros(2), group=0)
    src = SourceSpec(SKY_FLAT, 0, (0, W, 0, H), False, _pidx(0), np.zeros(8))
    pr = Problem("sky", [im], [src], 1, np.zeros(1), np.zeros(1), noise=[np.zeros((H, W), np.float32)],
                 var_floor=[1.0])
    im.data = np.asarray(data, np.float32)
    im.variance = np.asarray(var, np.float32)
    return pr


def test_lm_schedule_accept_by_hand():
    """Flat sky S on pixels of area a = |det A| = 4: the model is a S, so
    J^T W J = a^2 sum w, J^T W r = a sum w (d - a S), D = diag(J^T W J) and the
    damped step is the Gauss-Newton step (S* - S) shrunk by 1 / (1 + lambda),
    S* = sum w d / (a sum w).  Every step lowers chi^2 strictly: accept,
    lambda / 9.  Three iterations against that recursion by hand."""
    rng = np.random.default_rng(41)
    H, W = 5, 6
    d = rng.uniform(3.0, 9.0, (H, W)).astype(np.float32).astype(np.float64)
    v = rng.uniform(0.5, 2.0, (H, W)).astype(np.float32).astype(np.float64)
    pr = _flat_sky_problem(H, W, 2.0 * np.eye(2), d, v)
    a, w = 4.0, 1.0 / v
    s_star = np.sum(w * d) / (a * np.sum(w))
    S, lam = 0.25, 0.5
    th = np.array([S])
    lam_arr = np.array([lam])
    for _ in range(3):
        th, lam_arr, hist = O.lm_iterate(pr, th, lam_arr, 1)
        S = S + (s_star - S) / (1.0 + lam)
        lam = lam / 9.0
        assert bool(hist[0][2][0])
        assert th[0] == pytest.approx(S, rel=1e-12)
        assert lam_arr[0] == pytest.approx(lam, rel=1e-15)


def test_lm_schedule_reject_at_exact_optimum():
    """At the exact optimum the residual is zero, the step is zero and the
    trial chi^2 equals the current one: a strict-decrease rule rejects
    (theta kept, lambda * 11); an accept-on-equal rule would divide by 9."""
    H, W = 4, 4
    pr = _flat_sky_problem(H, W, 2.0 * np.eye(2), np.full((H, W), 8.0), np.full((H, W), 2.0))
    th, lam, hist = O.lm_iterate(pr, np.array([2.0]), np.array([1e-3]), 2)
    assert th[0] == 2.0
    assert not any(bool(h[2][0]) for h in hist)
    assert hist[0][0][0] == 0.0 and hist[0][1][0] == 0.0
    assert lam[0] == pytest.approx(1e-3 * 11.0 * 11.0, rel=1e-15)


def _one_free_slot(type_, true, start, slot, H=32, W=32):
    n = O.N_SLOTS[type_]
    pfix = np.zeros(8)
    pfix[:n] = true
    free = np.full(8, -1, dtype=np.int64)
    free[slot] = 0
    pr = one_source_problem(type_, [start], H=H, W=W, pfix=pfix, free=free)
    m = O.model_images(pr, np.array([true[slot]]))[0]
    pr.images[0].data = m.astype(np.float32)
    pr.images[0].variance = (np.abs(m) + 1.0).astype(np.float32)
    return pr


@pytest.mark.parametrize("type_,true,start,slot,bound", [
    (SERSIC, [16.2, 15.7, 0.7, 0.4, 9.0, 5.0, 10.0], 7.9, 4, 8.0),          # Sersic n ceiling
    (SERSIC, [16.2, 15.7, 0.7, 0.4, 0.3, 5.0, 10.0], 0.40, 4, 0.36),        # Sersic n floor
    (SERSIC, [16.2, 15.7, 1.15, 0.4, 1.5, 5.0, 10.0], 0.98, 2, 1.0),        # q ceiling
    (GAUSSIAN, [16.2, 15.7, 0.04, 0.4, 3.0, 100.0], 0.07, 2, 0.05),         # q floor
    (MOFFAT, [16.2, 15.7, 0.9, 0.4, 1.02, 2.0, 100.0], 1.10, 4, 1.05),      # Moffat n floor
    (MOFFAT, [16.2, 15.7, 0.9, 0.4, 55.0, 2.0, 100.0], 48.0, 4, 50.0),      # Moffat n ceiling
])
def test_lm_schedule_clamps_trial_to_box(type_, true, start, slot, bound):
    """Data made beyond a bound: the damped step (solved here with a library
    solve of the oracle's normal equations) leaves the box, the trial is
    clamped onto the bound, chi^2 drops, the clamped point is taken."""
    pr = _one_free_slot(type_, true, start, slot)
    lam0 = 1e-6
    JtWJ, JtWr = O.normal_equations(pr, np.array([start]))
    M = JtWJ + lam0 * np.diag(np.diag(JtWJ))
    unclamped = start + np.linalg.solve(M, JtWr)[0]
    assert (unclamped > bound) if bound > start else (unclamped < bound)
    th, lam, hist = O.lm_iterate(pr, np.array([start]), np.array([lam0]), 1)
    assert bool(hist[0][2][0]) and th[0] == bound
    assert lam[0] == pytest.approx(lam0 / 9.0, rel=1e-15)


def test_lm_schedule_groups_decide_independently():
    """Two groups in one iteration, one accepting and one rejecting: each
    group's outcome follows its own chi^2 (trial from a library solve of the
    damped system, clamped to the box), the rejecting group keeps theta and
    takes lambda * 11, the accepting one moves and takes lambda / 9."""
    pr = configs.mixed_small(seed=configs.SEED_BASE + 60, H=30, W=34, K=5, n_images=2, groups=2)
    attach_data(pr, O.model_images(pr, pr.theta_true))
    rng = np.random.default_rng(0)
    lo, hi = O.param_bounds(pr)
    th0 = np.clip(pr.theta_true * (1 + 0.3 * rng.standard_normal(pr.n_params)), lo, hi)
    lam0 = 1e-8
    c0 = O.chi2(pr, th0)
    JtWJ, JtWr = O.normal_equations(pr, th0)
    pg = pr.param_group()
    trial = th0.copy()
    for g in range(2):
        idx = np.nonzero(pg == g)[0]
        M = JtWJ[np.ix_(idx, idx)]
        D = np.maximum(np.diag(M), 1e-12 * np.diag(M).max())   # the damping diagonal's floor
        trial[idx] = np.clip(th0[idx] + np.linalg.solve(M + lam0 * np.diag(D), JtWr[idx]), lo[idx], hi[idx])
    c1 = O.chi2(pr, trial)
    acc = c1 < c0
    assert acc.tolist() == [False, True]
    th, lam, hist = O.lm_iterate(pr, th0, np.array([lam0, lam0]), 1)
    assert hist[0][2].tolist() == [False, True]
    for g in range(2):
        idx = np.nonzero(pg == g)[0]
        want = trial[idx] if acc[g] else th0[idx]
        np.testing.assert_allclose(th[idx], want, rtol=1e-9, atol=1e-12)
        assert lam[g] == pytest.approx(lam0 / 9.0 if acc[g] else lam0 * 11.0, rel=1e-15)


def test_step_envelope_bounds_jacobian_perturbations():
    """The test-side envelope (first-order bound on the step change under a
    relative change eps of every Jacobian entry) holds for random such
    changes of the oracle's Jacobian: the step recomputed from the perturbed
    normal equations moves by no more than the bound, component by component."""
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from _helpers import step_envelope
    pr = configs.mixed_small(seed=configs.SEED_BASE + 14, H=24, W=30, K=5)
    attach_data(pr, O.model_images(pr, pr.theta_true))
    th, lam, eps = pr.theta_init, 1e-3, 1e-4
    idx = np.arange(pr.n_params)
    env = step_envelope(pr, th, lam, idx, eps=eps)
    Js = O.jacobian(pr, th)
    res = O.residuals(pr, th)

    def step(Jlist):
        M = sum((J.T @ J.multiply(w[:, None])).toarray() for J, (r, w) in zip(Jlist, res))
        b = sum(J.T @ (w * r) for J, (r, w) in zip(Jlist, res))
        d = np.diag(M)
        return np.linalg.solve(M + lam * np.diag(np.maximum(d, O.DIAG_FLOOR * d.max())), b)

    d0 = step(Js)
    rng = np.random.default_rng(8)
    worst = 0.0
    for _ in range(6):
        Jp = []
        for J in Js:
            J2 = J.copy().tocsr()
            J2.data = J2.data * (1.0 + eps * rng.uniform(-1, 1, J2.data.size))
            Jp.append(J2)
        worst = max(worst, float(np.max(np.abs(step(Jp) - d0) / env)))
    # first order: second-order terms are ~eps relative smaller
    print("envelope use", worst)
    assert worst <= 1.0 + 1e-3, worst


# ---------------------------------------------------------------------------
# The psf star model (Sec. "A Zoo of Models": a PSF pixel map interpolated
# bilinearly; readings in the oracle's psf_star_profile)
# ---------------------------------------------------------------------------

def _psf_star_problem(P, xy, H=15, W=17, Q=1, A=None, origin=None, F=7.0):
    from synthetic.problem import PSF_STAR
    pr = one_source_problem(PSF_STAR, [xy[0], xy[1], F], H=H, W=W, A=A, origin=origin,
                            psf=np.asarray(P, np.float32), Q=Q)
    return pr


def test_psf_star_on_a_pixel_centre_is_the_map():
    """At a pixel centre, sampled at the pixel centres (order 1), the model is
    F times the normalised map, its centre pixel on the star's pixel."""
    rng = np.random.default_rng(31)
    P = rng.uniform(0.1, 1.0, (5, 5))
    pr = _psf_star_problem(P, (8.5, 6.5))      # pixel (6, 8) centre, A = I, origin 0
    m = O.model_images(pr, pr.theta_true)[0]
    Pn = P.astype(np.float32).astype(np.float64)
    Pn = Pn / Pn.sum()
    want = np.zeros_like(m)
    want[4:9, 6:11] = 7.0 * Pn
    np.testing.assert_allclose(m, want, rtol=1e-13, atol=1e-15)


def test_psf_star_half_pixel_shift_averages_neighbours():
    """Half a pixel to the right, each pixel centre falls half-way between two
    map pixels: bilinear interpolation gives their mean."""
    rng = np.random.default_rng(32)
    P = rng.uniform(0.1, 1.0, (5, 5))
    pr = _psf_star_problem(P, (9.0, 6.5))
    m = O.model_images(pr, pr.theta_true)[0]
    Pn = P.astype(np.float32).astype(np.float64)
    Pn = Pn / Pn.sum()
    pad = np.zeros((5, 7))
    pad[:, 1:6] = Pn
    want = np.zeros_like(m)
    want[4:9, 6:12] = 7.0 * 0.5 * (pad[:, :-1] + pad[:, 1:])
    np.testing.assert_allclose(m, want, rtol=1e-13, atol=1e-15)


def test_psf_star_delta_map_is_the_tent_surface():
    """A delta map interpolates to the tent (1 - |du|)(1 - |dv|): its pixel
    integrals are 9/16 (centre), 3/32 (edge neighbours), 1/64 (corners),
    checked by brute-force 64 x 64 sub-sampling of the oracle's surface; a
    rotated image keeps the map on its own pixel grid."""
    P = np.zeros((3, 3))
    P[1, 1] = 1.0
    for A in (np.eye(2), np.array([[0.0, -1.0], [1.0, 0.0]])):
        origin = -A @ np.array([8.0, 7.0])
        xy = origin + A @ np.array([8.5, 7.5])     # centre of pixel (7, 8)
        pr = _psf_star_problem(P, xy, A=A, origin=origin, F=1.0)
        src = pr.sources[0]
        vals = _brute(pr, src, pr.theta_true)
        want = {(0, 0): 9 / 16, (0, 1): 3 / 32, (1, 0): 3 / 32, (1, 1): 1 / 64}
        for (di, dj), v in want.items():
            for si in (-1, 1):
                for sj in (-1, 1):
                    assert abs(vals[7 + si * di, 8 + sj * dj] - v) < 2e-4, (di, dj, vals[7 + si * di, 8 + sj * dj], v)
        assert abs(vals.sum() - 1.0) < 1e-6


def test_psf_star_total_flux():
    """The bilinear surface of a normalised map integrates to one, so the
    total light is F: the order-7 rule on every pixel comes within 1e-3 of
    F (the surface's kinks at pixel centres limit the rule)."""
    rng = np.random.default_rng(33)
    P = rng.uniform(0.0, 1.0, (7, 7))
    pr = _psf_star_problem(P, (8.3, 7.1), Q=7, F=5.0)
    m = O.model_images(pr, pr.theta_true)[0]
    assert abs(m.sum() - 5.0) < 5e-3


# ---------------------------------------------------------------------------
# Pixel-centred sampling and the interpolated re-shift (Sec. "PSF convolution")
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("method", [O.SHIFT_LANCZOS3, O.SHIFT_BILINEAR])
def test_shift_by_whole_pixels_is_exact(method):
    """A shift by a whole pixel moves every value one place: the Lanczos
    kernel vanishes at the other integers, the bilinear one too."""
    rng = np.random.default_rng(41)
    img = rng.standard_normal((12, 15))
    out = O.interp_shift(img, 1.0, -1.0, method)
    want = np.zeros_like(img)
    want[:-1, 1:] = img[1:, :-1]
    np.testing.assert_allclose(out, want, atol=1e-15)


def test_bilinear_half_pixel_averages_neighbours():
    rng = np.random.default_rng(42)
    img = rng.standard_normal((9, 11))
    out = O.interp_shift(img, 0.5, 0.0, O.SHIFT_BILINEAR)
    pad = np.zeros((9, 12))
    pad[:, 1:] = img
    np.testing.assert_allclose(out, 0.5 * (pad[:, 1:] + pad[:, :-1]), atol=1e-15)


def test_lanczos_reproduces_band_limited_input():
    """A sampled sinusoid moved by 0.3 pixel against the sinusoid evaluated at
    the moved points, away from the edges.  Bilinear interpolation is exact on
    linear functions, so its error falls as the square of the frequency;
    the normalised 3-lobe Lanczos kernel is far more accurate at high
    frequencies (a few samples per period) and stays within a few 1e-3."""
    x = np.arange(128, dtype=np.float64)
    errs = {}
    for period in (8.0, 16.0, 32.0, 64.0):
        img = np.tile(np.sin(2 * np.pi * x / period), (5, 1))
        exact = np.sin(2 * np.pi * (x[16:-16] - 0.3) / period)
        for method in (O.SHIFT_LANCZOS3, O.SHIFT_BILINEAR):
            out = O.interp_shift(img, 0.3, 0.0, method)
            errs[period, method] = np.abs(out[2, 16:-16] - exact).max()
    for period in (8.0, 16.0, 32.0, 64.0):
        assert errs[period, O.SHIFT_LANCZOS3] < 6e-3
    assert errs[8.0, O.SHIFT_LANCZOS3] < 0.1 * errs[8.0, O.SHIFT_BILINEAR]
    for p1, p2 in ((8.0, 16.0), (16.0, 32.0), (32.0, 64.0)):
        r = errs[p1, O.SHIFT_BILINEAR] / errs[p2, O.SHIFT_BILINEAR]
        assert 3.5 < r < 4.5, (p1, r)


def test_shift_conserves_flux_and_commutes_with_convolution():
    """Normalised weights keep the total of an interior image; shifting then
    convolving equals convolving then shifting (both discrete convolutions),
    away from the array's edges."""
    rng = np.random.default_rng(43)
    img = np.zeros((40, 40))
    img[12:28, 10:30] = rng.random((16, 20))
    for method in (O.SHIFT_LANCZOS3, O.SHIFT_BILINEAR):
        out = O.interp_shift(img, 0.37, -0.21, method)
        assert abs(out.sum() - img.sum()) < 1e-12 * img.sum()
        P = rng.random((7, 7))
        P /= P.sum()
        pad = np.pad(img, 3)
        a = O.convolve_layer(np.pad(O.interp_shift(img, 0.37, -0.21, method), 3), P, 40, 40)
        b = O.interp_shift(O.convolve_layer(pad, P, 40, 40), 0.37, -0.21, method)
        np.testing.assert_allclose(a[8:-8, 8:-8], b[8:-8, 8:-8], atol=1e-14)


def test_shifted_model_of_a_smooth_source_matches_true_centre():
    """A well-sampled Gaussian (sigma 2.5 px): sampled at the pixel centre and
    moved back, the model agrees with the model sampled at the true centre to
    the interpolation's accuracy (Lanczos far better than bilinear)."""
    P = configs.psf_gaussian(9, 1.2)
    pr = one_source_problem(GAUSSIAN, [20.3, 17.8, 0.8, 0.5, 2.5, 500.0], H=40, W=44, psf=P, conv=True)
    ref = O.model_images(pr, pr.theta_true)[0]
    for method, tol in ((O.SHIFT_LANCZOS3, 6e-3), (O.SHIFT_BILINEAR, 5e-2)):
        m = O.model_layers_shifted(pr, pr.theta_true, method)[0]["m"]
        assert np.abs(m - ref).max() <= tol * ref.max(), (method, np.abs(m - ref).max() / ref.max())
    # a source already on a pixel centre is not moved
    pr2 = one_source_problem(GAUSSIAN, [20.5, 17.5, 0.8, 0.5, 2.5, 500.0], H=40, W=44, psf=P, conv=True)
    np.testing.assert_allclose(O.model_layers_shifted(pr2, pr2.theta_true, O.SHIFT_LANCZOS3)[0]["m"],
                               O.model_images(pr2, pr2.theta_true)[0], rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Live PSF parameters (Sec. "PSF convolution"; the PSF-extraction example:
# a Moffat PSF (n, Rd) fitted with the galaxies, shared with the stars)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def live():
    pr = configs.mixed_small(seed=configs.SEED_BASE + 15, H=30, W=34, K=7, live_psf=True, n_images=2, groups=1)
    attach_data(pr, O.model_images(pr, pr.theta_true))
    return pr


def test_live_psf_point_sampled_is_the_moffat_image():
    """Sampled at pixel centres (order 1) on an axis-aligned unit grid, the
    live PSF is the Moffat image of the generator (point-sampled, unit sum)."""
    from synthetic.problem import ImageSpec
    fwhm, beta, K = 3.0, 3.0, 11
    im = ImageSpec(H=8, W=8, A=np.eye(2), origin=np.zeros(2), psf=np.zeros((K, K), np.float32), group=0,
                   psf_pidx=np.array([-1, -1]), psf_pfix=np.array([beta, configs.moffat_rd(fwhm, beta)]))
    pr = Problem("p", [im], [], 0, np.zeros(0), np.zeros(0), quad_order=1, noise=[np.zeros((8, 8))], var_floor=[1.0])
    P, _ = O.image_psf(pr, 0, np.zeros(0))
    np.testing.assert_allclose(P, configs.psf_moffat(K, fwhm, beta).astype(np.float64), rtol=2e-7, atol=1e-9)


def test_live_psf_gradient_and_columns_match_central_differences(live):
    """d chi^2 / d(n, Rd) of the live PSF (through the convolution of every
    galaxy and the shared Moffat stars) and its Jacobian columns against
    central differences of the oracle's own chi^2 and model."""
    pr = live
    th = pr.theta_init
    g = O.gradient(pr, th)
    Js = O.jacobian(pr, th)
    for p in {int(q) for im in pr.images for q in im.psf_pidx}:
        h = 1e-6 * max(1.0, abs(th[p]))
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (O.chi2(pr, tp).sum() - O.chi2(pr, tm).sum()) / (2 * h)
        assert abs(g[p] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (p, g[p], fd)
        mp, mm = O.model_images(pr, tp), O.model_images(pr, tm)
        for J, a, b in zip(Js, mp, mm):
            col = J[:, p].toarray().ravel()
            fdc = ((a - b) / (2 * h)).ravel()
            assert np.abs(col - fdc).max() <= 1e-6 * np.abs(fdc).max()


def test_live_psf_params_belong_to_the_group_and_box(live):
    pr = live
    lo, hi = O.param_bounds(pr)
    pn, prd = (int(q) for q in pr.images[0].psf_pidx)
    assert pr.param_group()[pn] == pr.images[0].group
    assert (lo[pn], hi[pn]) == (1.05, 50.0) and lo[prd] == 1e-3
