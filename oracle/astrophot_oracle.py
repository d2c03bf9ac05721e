"""CPU FP64 oracle of the chi^2 forward-modelling path (arXiv:2308.01957).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The GPU product never calls it, and it shares no code with the GPU
path: profiles, quadrature, convolution, chi^2, Jacobian and the LM step are
written out here, plainly and slowly, in float64 with numpy/scipy primitives.

Every function cites the passage of the paper it follows.  Where the paper is
silent the reading taken is stated in the docstring or in the comment above
it.  Pins (tests/test_oracle_pins.py, tests/test_oracle_adaptive_pins.py) tie each function to
something other than itself: closed forms, special cases, brute force and
finite differences.

Problem objects are read by attribute (see synthetic/problem.py for the
layout): images with H, W, A, origin, psf, mask, group, data, variance and
sources with type, image, win, psf_convolve, pidx, pfix.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy import integrate, sparse, special

# profile codes (the interface's type codes)
SERSIC, EXPONENTIAL, GAUSSIAN, MOFFAT, SKY_FLAT, SKY_PLANE, PSF_STAR = range(7)
N_SLOTS = {SERSIC: 7, EXPONENTIAL: 6, GAUSSIAN: 6, MOFFAT: 7, SKY_FLAT: 1, SKY_PLANE: 3, PSF_STAR: 3}

# Reading: the Sersic radius is regularised as sqrt(R^2 + eps^2) so that the
# derivatives stay finite when a quadrature node lands on the centre.
EPS_REL = 1e-4


# ---------------------------------------------------------------------------
# Sersic b_n  (Sersic 1963, named in Sec. "A Zoo of Models")
# ---------------------------------------------------------------------------

def sersic_b(n: float) -> float:
    """b_n: the root of gamma(2n, b) = Gamma(2n)/2, i.e. the regularised lower
    incomplete gamma P(2n, b) = 1/2 (half the light inside R_e).  Computed with
    the library inverse of P."""
    return float(special.gammaincinv(2.0 * n, 0.5))


def sersic_db_dn(n: float) -> float:
    """d b_n / d n by implicit differentiation of P(2n, b_n) = 1/2:
    db/dn = -2 (dP/da) / (dP/dx) at a = 2n, x = b_n, with
    dP/dx = x^(a-1) e^-x / Gamma(a) and
    dP/da = (1/Gamma(a)) int_0^x ln t t^(a-1) e^-t dt - psi(a) P(a, x)."""
    a = 2.0 * n
    b = sersic_b(n)
    dPdx = math.exp((a - 1.0) * math.log(b) - b - special.gammaln(a))
    # int_0^b e^-t * t^(a-1) * ln t dt   (QUADPACK algebraic-log weight)
    val, _ = integrate.quad(lambda t: math.exp(-t), 0.0, b, weight="alg-loga", wvar=(a - 1.0, 0.0),
                            epsabs=0.0, epsrel=1e-13, limit=200)
    dPda = val / special.gamma(a) - special.digamma(a) * special.gammainc(a, b)
    return -2.0 * dPda / dPdx


# ---------------------------------------------------------------------------
# Geometry and quadrature  (Sec. "Pixel Integration"; pixel-scale matrix of
# the multi-band example; "arcsec from bottom corner" in the config example)
# ---------------------------------------------------------------------------

def gl_rule(Q: int):
    """Gauss-Legendre nodes and weights of order Q on [-1, 1] (library rule).
    An order-Q rule is exact for polynomials of degree 2Q-1 and costs Q^2
    evaluations per pixel (footnote of the pixel-integration section)."""
    u, w = leggauss(Q)
    return u, w


def det_A(im) -> float:
    A = np.asarray(im.A, dtype=np.float64)
    return abs(A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0])


def node_coords(im, rows: np.ndarray, cols: np.ndarray, Q: int):
    """World coordinates of the Q x Q Gauss-Legendre nodes of pixels rows x cols.

    Pixel (i, j) covers the unit square [j, j+1) x [i, i+1) of pixel
    coordinates; a pixel-coordinate point (u, v) sits at world position
    origin + A (u, v).  Node (a, b) of pixel (i, j) is at
    (j + 1/2 + u_a/2, i + 1/2 + u_b/2).  Returns x, y of shape
    (nr, nc, Q, Q) with axis 2 the column node and axis 3 the row node, and the
    (Q, Q) weights w_a w_b / 4 (the rule mapped to a unit interval per axis)."""
    u, w = gl_rule(Q)
    A = np.asarray(im.A, dtype=np.float64)
    o = np.asarray(im.origin, dtype=np.float64)
    uu = cols[None, :, None, None] + 0.5 + 0.5 * u[None, None, :, None]
    vv = rows[:, None, None, None] + 0.5 + 0.5 * u[None, None, None, :]
    x = o[0] + A[0, 0] * uu + A[0, 1] * vv
    y = o[1] + A[1, 0] * uu + A[1, 1] * vv
    W2 = 0.25 * w[:, None] * w[None, :]
    return x, y, W2


def image_centre(im):
    A = np.asarray(im.A, dtype=np.float64)
    o = np.asarray(im.origin, dtype=np.float64)
    return o + A @ np.array([im.W / 2.0, im.H / 2.0])


# ---------------------------------------------------------------------------
# Profiles and their analytic derivatives (Sec. "A Zoo of Models")
# ---------------------------------------------------------------------------

def slot_values(src, theta) -> np.ndarray:
    """The source's slot values: theta[pidx[k]] or the fixed value pfix[k]."""
    out = np.zeros(8)
    for k in range(N_SLOTS[src.type]):
        p = int(src.pidx[k])
        out[k] = theta[p] if p >= 0 else float(src.pfix[k])
    return out


def _ellipse(x, y, x0, y0, q, PA):
    """Elliptical radius.  X runs along the major axis at angle PA
    (counter-clockwise from the +x world axis), Y along the minor axis;
    rho^2 = X^2 + (Y/q)^2 with q = b/a.  Returns X, Y, rho^2 and the
    derivatives of rho^2 with respect to x0, y0, q, PA."""
    c, s = math.cos(PA), math.sin(PA)
    dx = x - x0
    dy = y - y0
    X = c * dx + s * dy
    Y = -s * dx + c * dy
    r2 = X * X + (Y / q) ** 2
    Yq2 = Y / (q * q)
    d_x0 = 2.0 * (X * (-c) + Yq2 * s)
    d_y0 = 2.0 * (X * (-s) + Yq2 * (-c))
    d_q = -2.0 * Y * Y / q ** 3
    d_PA = 2.0 * (X * Y + Yq2 * (-X))
    return X, Y, r2, (d_x0, d_y0, d_q, d_PA)


def profile(type_: int, p: np.ndarray, x, y, im, want_grad: bool):
    """Surface brightness I(x, y) of one source and, if asked, dI/d(slot) for
    each slot.  Readings of the named profiles (the paper prints none):

    * Sersic:  I = Ie exp(-b_n [(R/Re)^(1/n) - 1]), R = sqrt(rho^2 + eps^2)
    * exponential: the Sersic with n = 1, parameterised by Re
    * Gaussian: I = F / (2 pi sigma^2 q) exp(-rho^2 / (2 sigma^2))
    * Moffat:  I = F (n-1) / (pi Rd^2 q) (1 + rho^2/Rd^2)^(-n)
    * flat sky: I = S;  plane sky: I = S + gx (x - xc) + gy (y - yc), (xc, yc)
      the world position of the image centre.
    """
    grads = None
    if type_ in (SERSIC, EXPONENTIAL):
        if type_ == SERSIC:
            x0, y0, q, PA, n, Re, Ie = p[:7]
        else:
            x0, y0, q, PA, Re, Ie = p[:6]
            n = 1.0
        b = sersic_b(n)
        eps = EPS_REL * math.sqrt(det_A(im))
        X, Y, r2, dr2 = _ellipse(x, y, x0, y0, q, PA)
        r2 = r2 + eps * eps
        t = (r2 / (Re * Re)) ** (0.5 / n)
        e = np.exp(-b * (t - 1.0))
        I = Ie * e
        if want_grad:
            dI_dr2 = I * (-b) * t / (2.0 * n * r2)
            g = [dI_dr2 * dr2[0], dI_dr2 * dr2[1], dI_dr2 * dr2[2], dI_dr2 * dr2[3]]
            if type_ == SERSIC:
                db = sersic_db_dn(n)
                lnu = 0.5 * np.log(r2 / (Re * Re))
                g.append(I * (-db * (t - 1.0) + b * t * lnu / (n * n)))
            g.append(I * b * t / (n * Re))
            g.append(e)
            grads = g
        return I, grads
    if type_ == GAUSSIAN:
        x0, y0, q, PA, sg, F = p[:6]
        X, Y, r2, dr2 = _ellipse(x, y, x0, y0, q, PA)
        e = np.exp(-r2 / (2.0 * sg * sg)) / (2.0 * math.pi * sg * sg * q)
        I = F * e
        if want_grad:
            dI_dr2 = -I / (2.0 * sg * sg)
            grads = [dI_dr2 * dr2[0], dI_dr2 * dr2[1], dI_dr2 * dr2[2] - I / q, dI_dr2 * dr2[3],
                     I * (-2.0 / sg + r2 / sg ** 3), e]
        return I, grads
    if type_ == MOFFAT:
        x0, y0, q, PA, n, Rd, F = p[:7]
        X, Y, r2, dr2 = _ellipse(x, y, x0, y0, q, PA)
        v = 1.0 + r2 / (Rd * Rd)
        e = (n - 1.0) / (math.pi * Rd * Rd * q) * v ** (-n)
        I = F * e
        if want_grad:
            dI_dr2 = -n * I / (v * Rd * Rd)
            grads = [dI_dr2 * dr2[0], dI_dr2 * dr2[1], dI_dr2 * dr2[2] - I / q, dI_dr2 * dr2[3],
                     I * (1.0 / (n - 1.0) - np.log(v)),
                     I * (-2.0 / Rd + 2.0 * n * r2 / (v * Rd ** 3)), e]
        return I, grads
    if type_ == PSF_STAR:
        return psf_star_profile(p, x, y, im, want_grad)
    if type_ == SKY_FLAT:
        I = np.full_like(x, p[0])
        return I, ([np.ones_like(x)] if want_grad else None)
    if type_ == SKY_PLANE:
        xc, yc = image_centre(im)
        I = p[0] + p[1] * (x - xc) + p[2] * (y - yc)
        return I, ([np.ones_like(x), x - xc, y - yc] if want_grad else None)
    raise ValueError(f"unknown profile type {type_}")


def psf_star_profile(p, x, y, im, want_grad: bool):
    """The "psf star" model of Sec. "A Zoo of Models": a point source whose
    light follows a PSF pixel map, interpolated bilinearly between the map's
    pixel centres.  Readings (the paper names the model and the interpolation
    only): the map is the image's PSF image, normalised to unit sum, on the
    image's own pixel grid; its centre pixel (K-1)/2 sits on the source
    position (x0, y0); the map is zero beyond its edge.  A world point is
    taken to the image's pixel coordinates, (u, v) = A^-1 (x - origin), and
    its offset from the source's pixel position gives the continuous map index
    (X, Y) = ((K-1)/2 + du, (K-1)/2 + dv), X along the map's columns.  The
    surface brightness is F B(X, Y) / |det A| per unit world area, B the
    bilinear interpolant, so that the light per unit pixel area is F B and a
    pixel value is F times the pixel integral of B."""
    x0, y0, F = p[:3]
    if psf_is_live(im):
        raise ValueError("a PSF star needs a fixed PSF image (its map would depend on the live PSF parameters)")
    P = normalised_psf(im)
    K = P.shape[0]
    c = 0.5 * (K - 1)
    Ai = np.linalg.inv(np.asarray(im.A, dtype=np.float64))
    o = np.asarray(im.origin, dtype=np.float64)
    u = Ai[0, 0] * (x - o[0]) + Ai[0, 1] * (y - o[1])
    v = Ai[1, 0] * (x - o[0]) + Ai[1, 1] * (y - o[1])
    u0 = Ai[0, 0] * (x0 - o[0]) + Ai[0, 1] * (y0 - o[1])
    v0 = Ai[1, 0] * (x0 - o[0]) + Ai[1, 1] * (y0 - o[1])
    X = c + (u - u0)
    Y = c + (v - v0)
    bx = np.floor(X).astype(np.int64)
    by = np.floor(Y).astype(np.int64)
    tx = X - bx
    ty = Y - by

    def at(r, q):
        inside = (r >= 0) & (r < K) & (q >= 0) & (q < K)
        out = np.zeros(r.shape)
        out[inside] = P[r[inside], q[inside]]
        return out

    p00, p01 = at(by, bx), at(by, bx + 1)
    p10, p11 = at(by + 1, bx), at(by + 1, bx + 1)
    B = (1 - ty) * ((1 - tx) * p00 + tx * p01) + ty * ((1 - tx) * p10 + tx * p11)
    area = det_A(im)
    I = F * B / area
    grads = None
    if want_grad:
        dBdX = (1 - ty) * (p01 - p00) + ty * (p11 - p10)
        dBdY = (1 - tx) * (p10 - p00) + tx * (p11 - p01)
        # X = c + u - u0(x0, y0): dX/dx0 = -Ai[0, 0], dX/dy0 = -Ai[0, 1]; Y likewise with row 1
        grads = [F / area * (-Ai[0, 0] * dBdX - Ai[1, 0] * dBdY),
                 F / area * (-Ai[0, 1] * dBdX - Ai[1, 1] * dBdY),
                 B / area]
    return I, grads


# ---------------------------------------------------------------------------
# Windows and the render (Sec. "Automatic Initialization": models are only
# evaluated inside their window; Sec. "PSF convolution": galaxies are sampled
# with the PSF's reach around them, then convolved)
# ---------------------------------------------------------------------------

def psf_half(im) -> int:
    return 0 if im.psf is None else (np.asarray(im.psf).shape[0] - 1) // 2


def is_convolved(problem, src) -> bool:
    """Galaxies with psf_convolve set on an image with a PSF; a PSF star is
    the PSF itself and is never convolved."""
    return bool(src.psf_convolve) and problem.images[src.image].psf is not None and src.type != PSF_STAR


def source_box(problem, src):
    """Pixel box (r0, r1, c0, c1), half-open, on which a source is sampled.

    Reading: the window is first clipped to the image (an empty clip means
    the source is not drawn); a convolved source is then sampled on its window
    grown by the PSF half width h = (K-1)/2, clipped to the image grown by h
    (the galaxy layer); other sources on their clipped window."""
    im = problem.images[src.image]
    x0, x1, y0, y1 = src.win
    x0, x1, y0, y1 = max(x0, 0), min(x1, im.W), max(y0, 0), min(y1, im.H)
    if x0 >= x1 or y0 >= y1:
        return (0, 0, 0, 0)
    if is_convolved(problem, src):
        h = psf_half(im)
        return (max(y0 - h, -h), min(y1 + h, im.H + h), max(x0 - h, -h), min(x1 + h, im.W + h))
    return (max(y0, 0), min(y1, im.H), max(x0, 0), min(x1, im.W))


def render_source(problem, src, theta, box=None, want_grad=False):
    """Pixel-integrated source on ``box`` (default: its sampling box):
    m(i, j) = |det A| sum_ab (w_a w_b / 4) I(node_ab(i, j))  (order-Q
    Gauss-Legendre on every pixel, Q = problem.quad_order).

    Returns (box, values[nr, nc], grads[n_slots, nr, nc] or None)."""
    im = problem.images[src.image]
    sb = source_box(problem, src)
    if box is None:
        box = sb
    else:
        box = (max(box[0], sb[0]), min(box[1], sb[1]), max(box[2], sb[2]), min(box[3], sb[3]))
    r0, r1, c0, c1 = box
    nr, nc = max(r1 - r0, 0), max(c1 - c0, 0)
    ns = N_SLOTS[src.type]
    if nr == 0 or nc == 0:
        return box, np.zeros((nr, nc)), (np.zeros((ns, nr, nc)) if want_grad else None)
    x, y, W2 = node_coords(im, np.arange(r0, r1, dtype=np.float64), np.arange(c0, c1, dtype=np.float64),
                           problem.quad_order)
    p = slot_values(src, theta)
    I, g = profile(src.type, p, x, y, im, want_grad)
    area = det_A(im)
    vals = area * np.einsum("rcab,ab->rc", I, W2)
    grads = None
    if want_grad:
        grads = np.stack([area * np.einsum("rcab,ab->rc", gk, W2) for gk in g])
    return box, vals, grads


def normalised_psf(im) -> np.ndarray:
    """The PSF divided by its sum (the paper's PSFs are normalised internally
    before convolution)."""
    P = np.asarray(im.psf, dtype=np.float64)
    return P / P.sum()


# ---------------------------------------------------------------------------
# Live PSF (Sec. "PSF convolution": the PSF may itself be a model whose
# parameters are optimised during the fit; the multi-band example fits a
# Moffat PSF (n, Rd) shared with the image's Moffat stars)
# ---------------------------------------------------------------------------

def psf_is_live(im) -> bool:
    return getattr(im, "psf_pidx", None) is not None


def live_psf_params(im, theta):
    return [float(theta[int(p)]) if int(p) >= 0 else float(f) for p, f in zip(im.psf_pidx, im.psf_pfix)]


def live_psf_raw(problem, im, theta, want_grad: bool):
    """The live PSF before normalisation and its derivatives by (n, Rd).
    Reading: a circular Moffat (q = 1) of unit flux, centred on the centre of
    the map's middle pixel (K-1)/2, integrated over each map pixel with the
    problem's order-Q rule exactly like a source on the image (the map's
    pixels are the image's pixels, mapped to the world by A)."""
    K = np.asarray(im.psf).shape[0]
    c = 0.5 * (K - 1)
    n, Rd = live_psf_params(im, theta)
    u, w = gl_rule(problem.quad_order)
    A = np.asarray(im.A, dtype=np.float64)
    idx = np.arange(K, dtype=np.float64) - c
    du = idx[None, :, None, None] + 0.5 * u[None, None, :, None]     # column offset of each node (pixels)
    dv = idx[:, None, None, None] + 0.5 * u[None, None, None, :]     # row offset
    x = A[0, 0] * du + A[0, 1] * dv
    y = A[1, 0] * du + A[1, 1] * dv
    W2 = 0.25 * w[:, None] * w[None, :]
    area = det_A(im)
    I, g = profile(MOFFAT, np.array([0.0, 0.0, 1.0, 0.0, n, Rd, 1.0]), x, y, im, want_grad)
    P = area * np.einsum("rcab,ab->rc", I, W2)
    if not want_grad:
        return P, None
    return P, [area * np.einsum("rcab,ab->rc", g[4], W2), area * np.einsum("rcab,ab->rc", g[5], W2)]


def image_psf(problem, ii, theta, want_grad: bool = False):
    """The normalised PSF of image ii at theta (fixed or live), and for a
    live PSF the derivatives of the normalised PSF by (n, Rd):
    d(P/S) = (dP - (P/S) dS) / S, S = sum P."""
    im = problem.images[ii]
    if not psf_is_live(im):
        return normalised_psf(im), None
    P, g = live_psf_raw(problem, im, theta, want_grad)
    S = P.sum()
    Pn = P / S
    if not want_grad:
        return Pn, None
    return Pn, [(gk - Pn * gk.sum()) / S for gk in g]


def convolve_layer(Gpad: np.ndarray, P: np.ndarray, H: int, W: int) -> np.ndarray:
    """True 2-D convolution M = P * G on the image pixels.

    G lives on the image grown by h = (K-1)/2 on every side (Gpad[i + h, j + h]
    is image pixel (i, j)); zero beyond.  M(i, j) = sum_{ty, tx} P[ty, tx]
    G(i - (ty - h), j - (tx - h)); taps summed in a fixed order."""
    K = P.shape[0]
    h = (K - 1) // 2
    M = np.zeros((H, W))
    for ty in range(K):
        for tx in range(K):
            M += P[ty, tx] * Gpad[2 * h - ty: 2 * h - ty + H, 2 * h - tx: 2 * h - tx + W]
    return M


def model_layers(problem, theta) -> List[dict]:
    """Per image: galaxy layer G (image + PSF halo), unconvolved layer U, the
    convolved galaxies M = P * G and the model m = M + U (the sum of all
    component models on the image, Eq. chi2's m(i, theta))."""
    out = []
    for ii, im in enumerate(problem.images):
        h = psf_half(im)
        G = np.zeros((im.H + 2 * h, im.W + 2 * h))
        U = np.zeros((im.H, im.W))
        for src in problem.sources:
            if src.image != ii:
                continue
            (r0, r1, c0, c1), vals, _ = render_source(problem, src, theta)
            if vals.size == 0:
                continue
            if is_convolved(problem, src):
                G[r0 + h: r1 + h, c0 + h: c1 + h] += vals
            else:
                U[r0:r1, c0:c1] += vals
        M = convolve_layer(G, image_psf(problem, ii, theta)[0], im.H, im.W) if im.psf is not None else np.zeros_like(U)
        out.append(dict(G=G, U=U, M=M, m=M + U))
    return out


def model_images(problem, theta) -> List[np.ndarray]:
    return [L["m"] for L in model_layers(problem, theta)]


# ---------------------------------------------------------------------------
# chi^2 (Eq. likelihood and Eq. chi2; variance map and mask)
# ---------------------------------------------------------------------------

def weights(im) -> np.ndarray:
    """w = 1/sigma^2 on unmasked pixels, 0 on masked ones (mask 1 = excluded).
    A non-positive or non-finite variance on an unmasked pixel is an error."""
    var = np.asarray(im.variance, dtype=np.float64)
    keep = np.ones((im.H, im.W), dtype=bool) if im.mask is None else (np.asarray(im.mask) == 0)
    bad = keep & ~(np.isfinite(var) & (var > 0))
    if bad.any():
        raise ValueError("non-positive or non-finite variance on an unmasked pixel")
    w = np.zeros((im.H, im.W))
    w[keep] = 1.0 / var[keep]
    return w


def chi2(problem, theta) -> np.ndarray:
    """chi^2 per group: sum over the group's pixels of w (d - m)^2.

    Reading of Eq. chi2: the reported quantity drops the factor 1/2 and the
    constant C, chi^2 = sum_i (d_i - m_i)^2 / sigma_i^2."""
    out = np.zeros(problem.n_groups)
    for im, m in zip(problem.images, model_images(problem, theta)):
        r = np.asarray(im.data, dtype=np.float64) - m
        out[im.group] += np.sum(weights(im) * r * r)
    return out


# ---------------------------------------------------------------------------
# Jacobian, gradient and normal equations (Sec. "Implementation with PyTorch"
# for the gradient; Sec. "Optimization methods" for LM)
# ---------------------------------------------------------------------------

def source_jacobian(problem, src, theta):
    """Columns dm/d(slot) of one source on the image: the pixel-integrated
    profile derivatives, convolved with the normalised PSF for convolved
    sources.  Returns (box, cols[n_slots, nr, nc]) with box the image-pixel
    region the columns can reach."""
    im = problem.images[src.image]
    box, _, D = render_source(problem, src, theta, want_grad=True)
    if not is_convolved(problem, src):
        return box, D
    h = psf_half(im)
    r0, r1, c0, c1 = box
    jr0, jr1, jc0, jc1 = max(r0 - h, 0), min(r1 + h, im.H), max(c0 - h, 0), min(c1 + h, im.W)
    if jr0 >= jr1 or jc0 >= jc1:
        return (jr0, jr0, jc0, jc0), np.zeros((D.shape[0], 0, 0))
    P = image_psf(problem, src.image, theta)[0]
    # convolve each derivative image on the output box: embed it in a
    # zero layer that covers the output box grown by h
    Hs, Ws = jr1 - jr0, jc1 - jc0
    cols = []
    for k in range(D.shape[0]):
        L = np.zeros((Hs + 2 * h, Ws + 2 * h))
        L[r0 - jr0 + h: r1 - jr0 + h, c0 - jc0 + h: c1 - jc0 + h] = D[k]
        cols.append(convolve_layer(L, P, Hs, Ws))
    return (jr0, jr1, jc0, jc1), np.stack(cols)


def jacobian(problem, theta) -> List[sparse.csr_matrix]:
    """Per image, the sparse Jacobian J[pixel, theta index] = dm/dtheta.
    Slots that share a theta index (within or across sources) add up."""
    out = []
    P = problem.n_params
    for ii, im in enumerate(problem.images):
        rows, cols, vals = [], [], []
        for src in problem.sources:
            if src.image != ii:
                continue
            (r0, r1, c0, c1), C = source_jacobian(problem, src, theta)
            if C.size == 0:
                continue
            rr, cc = np.meshgrid(np.arange(r0, r1), np.arange(c0, c1), indexing="ij")
            flat = (rr * im.W + cc).ravel()
            for k in range(C.shape[0]):
                pk = int(src.pidx[k])
                if pk < 0:
                    continue
                rows.append(flat)
                cols.append(np.full(flat.size, pk))
                vals.append(C[k].ravel())
        if psf_is_live(im):
            # dm/d(n, Rd) of the live PSF: (dP/dphi) * G over the image, G the
            # galaxy layer at theta (the PSF's Moffat stars add their own
            # columns through their shared slots above)
            G = model_layers(problem, theta)[ii]["G"]
            _, dP = image_psf(problem, ii, theta, want_grad=True)
            flat = np.arange(im.H * im.W)
            for k in range(2):
                pk = int(im.psf_pidx[k])
                if pk < 0:
                    continue
                rows.append(flat)
                cols.append(np.full(flat.size, pk))
                vals.append(convolve_layer(G, dP[k], im.H, im.W).ravel())
        if rows:
            J = sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                  shape=(im.H * im.W, P)).tocsr()
        else:
            J = sparse.csr_matrix((im.H * im.W, P))
        out.append(J)
    return out


def residuals(problem, theta):
    """Per image: r = d - m (flattened) and w."""
    out = []
    for im, m in zip(problem.images, model_images(problem, theta)):
        r = (np.asarray(im.data, dtype=np.float64) - m).ravel()
        out.append((r, weights(im).ravel()))
    return out


def gradient(problem, theta) -> np.ndarray:
    """d chi^2 / d theta = -2 J^T W r (exact derivative of the chi^2 above)."""
    g = np.zeros(problem.n_params)
    for J, (r, w) in zip(jacobian(problem, theta), residuals(problem, theta)):
        g += -2.0 * (J.T @ (w * r))
    return g


def normal_equations(problem, theta):
    """J^T W J (dense, P x P) and J^T W r of the Gauss-Newton / LM model."""
    P = problem.n_params
    JtWJ = np.zeros((P, P))
    JtWr = np.zeros(P)
    for J, (r, w) in zip(jacobian(problem, theta), residuals(problem, theta)):
        WJ = sparse.diags(w) @ J
        JtWJ += (J.T @ WJ).toarray()
        JtWr += J.T @ (w * r)
    return JtWJ, JtWr


# ---------------------------------------------------------------------------
# Levenberg-Marquardt (Sec. "Optimization methods": Marquardt 1963,
# Transtrum & Sethna 2012, Gavin 2022)
# ---------------------------------------------------------------------------

LAMBDA_DOWN = 9.0     # accepted step: lambda / 9
LAMBDA_UP = 11.0      # rejected step: lambda * 11
LAMBDA_MIN, LAMBDA_MAX = 1e-12, 1e12
DIAG_FLOOR = 1e-12    # damping diagonal floor, relative to the largest diagonal
CHOL_RETRIES = 8      # failed factorisation: lambda * 10, retry


def param_bounds(problem):
    """Box bounds applied after each update (the paper clips initial values
    back to their range; reading: the same box holds during the fit).
    q in [0.05, 1]; Sersic n in [0.36, 8]; Moffat n in [1.05, 50];
    Re, Rd, sigma >= 1e-3; everything else free.  A shared index takes the
    intersection of its slots' boxes."""
    lo = np.full(problem.n_params, -np.inf)
    hi = np.full(problem.n_params, np.inf)

    def clamp(p, a, b):
        lo[p] = max(lo[p], a)
        hi[p] = min(hi[p], b)

    for s in problem.sources:
        t = s.type
        for k in range(N_SLOTS[t]):
            p = int(s.pidx[k])
            if p < 0:
                continue
            if t in (SERSIC, EXPONENTIAL, GAUSSIAN, MOFFAT) and k == 2:
                clamp(p, 0.05, 1.0)
            elif t == SERSIC and k == 4:
                clamp(p, 0.36, 8.0)
            elif t == MOFFAT and k == 4:
                clamp(p, 1.05, 50.0)
            elif (t == SERSIC and k == 5) or (t in (EXPONENTIAL, GAUSSIAN) and k == 4) or (t == MOFFAT and k == 5):
                clamp(p, 1e-3, np.inf)
    for im in problem.images:   # a live Moffat PSF: the Moffat box for n and Rd
        if psf_is_live(im):
            if int(im.psf_pidx[0]) >= 0:
                clamp(int(im.psf_pidx[0]), 1.05, 50.0)
            if int(im.psf_pidx[1]) >= 0:
                clamp(int(im.psf_pidx[1]), 1e-3, np.inf)
    return lo, hi


def cholesky_lower(M: np.ndarray) -> Optional[np.ndarray]:
    """Plain L L^T factorisation, column by column; None if a pivot is not
    positive (the matrix is not numerically positive definite)."""
    n = M.shape[0]
    L = np.zeros_like(M)
    for j in range(n):
        d = M[j, j] - np.dot(L[j, :j], L[j, :j])
        if not (d > 0.0) or not np.isfinite(d):
            return None
        L[j, j] = math.sqrt(d)
        if j + 1 < n:
            L[j + 1:, j] = (M[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def damped_step(JtWJ: np.ndarray, JtWr: np.ndarray, lam: float):
    """Solve (J^T W J + lambda D) delta = J^T W r with D = diag(J^T W J)
    floored at DIAG_FLOOR * max diag.  On a failed factorisation lambda is
    multiplied by 10 and the solve retried (the LM step never meets a singular
    matrix).  Returns (delta, lambda actually used, ok)."""
    d = np.diag(JtWJ).copy()
    dmax = d.max() if d.size else 0.0
    d = np.maximum(d, DIAG_FLOOR * dmax if dmax > 0 else 1.0)
    for _ in range(CHOL_RETRIES + 1):
        L = cholesky_lower(JtWJ + lam * np.diag(d))
        if L is not None:
            z = _forward_sub(L, JtWr)
            return _back_sub(L.T, z), lam, True
        lam *= 10.0
    return np.zeros_like(JtWr), lam, False


def _forward_sub(L, b):
    n = b.size
    z = np.zeros(n)
    for i in range(n):
        z[i] = (b[i] - L[i, :i] @ z[:i]) / L[i, i]
    return z


def _back_sub(U, z):
    n = z.size
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (z[i] - U[i, i + 1:] @ x[i + 1:]) / U[i, i]
    return x


def lm_iterate(problem, theta, lam, n_iter: int):
    """n_iter LM iterations, each group on its own: solve the damped normal
    equations, clamp the trial point to the bounds, accept iff the group's
    chi^2 strictly decreases (lambda / 9), else keep theta (lambda * 11).

    ``lam`` is an array with one lambda per group.  Returns theta, lambda and
    a history of (chi2 before, chi2 trial, accepted) per iteration."""
    theta = np.array(theta, dtype=np.float64)
    lam = np.array(lam, dtype=np.float64).copy()
    pg = problem.param_group()
    lo, hi = param_bounds(problem)
    hist = []
    for _ in range(n_iter):
        c0 = chi2(problem, theta)
        JtWJ, JtWr = normal_equations(problem, theta)
        trial = theta.copy()
        for g in range(problem.n_groups):
            idx = np.nonzero(pg == g)[0]
            if idx.size == 0:
                continue
            delta, lam[g], _ = damped_step(JtWJ[np.ix_(idx, idx)], JtWr[idx], lam[g])
            trial[idx] = np.clip(theta[idx] + delta, lo[idx], hi[idx])
        c1 = chi2(problem, trial)
        acc = np.isfinite(c1) & (c1 < c0)
        for g in range(problem.n_groups):
            idx = np.nonzero(pg == g)[0]
            if acc[g]:
                theta[idx] = trial[idx]
                lam[g] = max(lam[g] / LAMBDA_DOWN, LAMBDA_MIN)
            else:
                lam[g] = min(lam[g] * LAMBDA_UP, LAMBDA_MAX)
        hist.append((c0, c1, acc))
    return theta, lam, hist


# ---------------------------------------------------------------------------
# Pixel-centred sampling with an interpolated re-shift (Sec. "PSF
# convolution": a convolved model is sampled with its centre moved to the
# nearest pixel centre, convolved, then shifted back to its true sub-pixel
# position by Lanczos or bilinear interpolation)
# ---------------------------------------------------------------------------

SHIFT_LANCZOS3, SHIFT_BILINEAR = 1, 2
LANCZOS_A = 3


def interp_weights(d: float, method: int):
    """Taps t = -3..3 and weights w(t) of a shift by d pixels (|d| <= 1/2):
    shifted(p) = sum_t w(t) f(p - t).  Lanczos (a = 3):
    w(t) = sinc(t - d) sinc((t - d) / 3) for |t - d| < 3, normalised to unit
    sum (reading: the paper does not say; normalised weights keep the flux);
    bilinear: w(t) = max(0, 1 - |t - d|).  sinc(x) = sin(pi x) / (pi x)."""
    t = np.arange(-LANCZOS_A, LANCZOS_A + 1, dtype=np.float64)
    x = t - d
    if method == SHIFT_BILINEAR:
        return t.astype(int), np.maximum(0.0, 1.0 - np.abs(x))
    w = np.where(np.abs(x) < LANCZOS_A, np.sinc(x) * np.sinc(x / LANCZOS_A), 0.0)
    return t.astype(int), w / w.sum()


def interp_shift(img: np.ndarray, du: float, dv: float, method: int) -> np.ndarray:
    """Move an image by du pixels along its columns and dv along its rows
    (separable interpolation, zero beyond the array): out(i, j) =
    sum_{s, t} wv(s) wu(t) img(i - s, j - t)."""
    tu, wu = interp_weights(du, method)
    tv, wv = interp_weights(dv, method)
    H, W = img.shape
    pad = LANCZOS_A
    P = np.zeros((H + 2 * pad, W + 2 * pad))
    P[pad:pad + H, pad:pad + W] = img
    rows = np.zeros((H + 2 * pad, W))
    for t, w in zip(tu, wu):
        if w != 0.0:
            rows += w * P[:, pad - t: pad - t + W]
    out = np.zeros((H, W))
    for t, w in zip(tv, wv):
        if w != 0.0:
            out += w * rows[pad - t: pad - t + H, :]
    return out


def snapped_source(problem, src, theta):
    """The source's slot values with its centre moved to the centre of the
    pixel that holds it, and the sub-pixel shift (du, dv) back to the true
    centre, in the image's pixel coordinates (each in [-1/2, 1/2))."""
    im = problem.images[src.image]
    p = slot_values(src, theta)
    A = np.asarray(im.A, dtype=np.float64)
    o = np.asarray(im.origin, dtype=np.float64)
    u0, v0 = np.linalg.solve(A, np.array([p[0], p[1]]) - o)
    su, sv = math.floor(u0) + 0.5, math.floor(v0) + 0.5
    q = p.copy()
    q[0], q[1] = o + A @ np.array([su, sv])
    return q, u0 - su, v0 - sv


def model_layers_shifted(problem, theta, method: int) -> List[dict]:
    """The model with every convolved profile source (Sersic, exponential,
    Gaussian, Moffat) sampled at its pixel-centred position on its sampling
    box, moved back by its sub-pixel shift, then convolved with the other
    galaxy light.  Reading: the interpolation is a discrete convolution with
    the interpolation kernel and so commutes with the PSF convolution; the
    shift is taken on each source's sampling box (zero beyond it) before the
    shared convolution (a pin checks that convolving first and shifting after
    gives the same image away from the edges).  Unconvolved sources and skies
    as in model_layers."""
    out = []
    for ii, im in enumerate(problem.images):
        h = psf_half(im)
        G = np.zeros((im.H + 2 * h, im.W + 2 * h))
        U = np.zeros((im.H, im.W))
        for src in problem.sources:
            if src.image != ii:
                continue
            shifted = is_convolved(problem, src) and src.type in (SERSIC, EXPONENTIAL, GAUSSIAN, MOFFAT)
            if shifted:
                q, du, dv = snapped_source(problem, src, theta)
                (r0, r1, c0, c1), R, _ = _render_slots(problem, src, q)
                vals = interp_shift(R, du, dv, method) if R.size else R
            else:
                (r0, r1, c0, c1), vals, _ = render_source(problem, src, theta)
            if vals.size == 0:
                continue
            if is_convolved(problem, src):
                G[r0 + h: r1 + h, c0 + h: c1 + h] += vals
            else:
                U[r0:r1, c0:c1] += vals
        M = convolve_layer(G, image_psf(problem, ii, theta)[0], im.H, im.W) if im.psf is not None else np.zeros_like(U)
        out.append(dict(G=G, U=U, M=M, m=M + U))
    return out


def _render_slots(problem, src, p):
    """render_source for explicit slot values p instead of theta."""
    import copy
    n = N_SLOTS[src.type]
    tmp = copy.copy(src)
    tmp.pidx = np.full(8, -1, dtype=np.int64)
    tmp.pidx[:n] = np.arange(n)
    tmp.pfix = np.zeros(8)
    return render_source(problem, tmp, np.asarray(p[:n], dtype=np.float64))


def chi2_shifted(problem, theta, method: int) -> np.ndarray:
    out = np.zeros(problem.n_groups)
    for im, L in zip(problem.images, model_layers_shifted(problem, theta, method)):
        r = np.asarray(im.data, dtype=np.float64) - L["m"]
        out[im.group] += np.sum(weights(im) * r * r)
    return out


# ---------------------------------------------------------------------------
# Sampled outputs for workloads too large to render whole
# ---------------------------------------------------------------------------

def model_at(problem, theta, image: int, pixels: Sequence[tuple]) -> np.ndarray:
    """Model value m(i, j) at a few pixels of one image, each computed on its
    own: the convolved galaxies from the K x K neighbourhood of the pixel, plus
    the unconvolved sources at the pixel."""
    im = problem.images[image]
    h = psf_half(im)
    P = image_psf(problem, image, theta)[0] if im.psf is not None else None
    out = np.zeros(len(pixels))
    for n, (i, j) in enumerate(pixels):
        G = np.zeros((2 * h + 1, 2 * h + 1))
        u = 0.0
        for src in problem.sources:
            if src.image != image:
                continue
            if is_convolved(problem, src):
                (r0, r1, c0, c1), vals, _ = render_source(problem, src, theta, box=(i - h, i + h + 1, j - h, j + h + 1))
                if vals.size:
                    G[r0 - (i - h): r1 - (i - h), c0 - (j - h): c1 - (j - h)] += vals
            else:
                (r0, r1, c0, c1), vals, _ = render_source(problem, src, theta, box=(i, i + 1, j, j + 1))
                if vals.size:
                    u += vals[0, 0]
        conv = 0.0
        if P is not None:
            # M(i, j) = sum P[ty, tx] G(i - ty + h, j - tx + h); G indexed from (i-h, j-h)
            for ty in range(2 * h + 1):
                for tx in range(2 * h + 1):
                    conv += P[ty, tx] * G[2 * h - ty, 2 * h - tx]
        out[n] = conv + u
    return out


# ---------------------------------------------------------------------------
# Adaptive pixel integration  (Sec. "Pixel Integration": a midpoint first
# pass, then deeper quadrature of the pixels whose light varies at second
# order and above, against a per-pixel budget e = tol F / N)
# ---------------------------------------------------------------------------
#
# Readings (the paper describes the scheme in words only):
#  * the scheme runs per source on its sampling box; F is the source's
#    midpoint flux on the box (its absolute value) and N the box's pixel count;
#  * the second-order variation of a pixel is estimated from the midpoint pass
#    by the discrete Laplacian L, the sum over the two axes of the second
#    difference of the three nearest pixels of that axis inside the box
#    (centred, or one-sided at the box's edge; no term on an axis shorter than
#    three pixels); the midpoint rule's error on a pixel is about
#    (f_xx + f_yy)/24 per unit area, so a pixel goes on to order-3 quadrature
#    when |L|/24 > e;
#  * a Gauss-Legendre level is converged when its rule and the rule one order
#    lower, on the same pieces, agree within the budget (the lower rule's
#    error bounds the higher's): the whole pixel with order 3 against order 2,
#    then the pixel split 5 x 5 with order 5 on each sub-pixel against order 4
#    (sums over the sub-pixels), so that, as the section describes, order 3
#    settles most selected pixels and only the steepest (often the centre
#    pixel) go further; comparing order 3 with the midpoint instead would send
#    nearly every selected pixel on, since the selection already found the
#    midpoint off by more than e;
#  * a pixel still not converged has each sub-pixel q checked against e/25 by
#    comparing its order-5 and order-4 values; those above are split 5 x 5
#    again with order 7 on each piece, the others keep their order-5 value;
#    the scheme stops there;
#  * sky models are linear in position: their midpoint is exact (level 0).

ADAPT_SPLIT = 5


def rect_values(problem, src, theta, rows, cols, ou, ov, s, Q):
    """For pixel centres given by the index arrays rows, cols (same shape):
    the integral of the source over the sub-square of side s (pixel units)
    whose lower-left corner is at (j + ou, i + ov) in pixel coordinates, by the
    order-Q Gauss-Legendre rule: |det A| s^2 sum_ab (w_a w_b / 4) I(node_ab),
    node_ab at (j + ou + s (1 + u_a)/2, i + ov + s (1 + u_b)/2)."""
    im = problem.images[src.image]
    u, w = gl_rule(Q)
    A = np.asarray(im.A, dtype=np.float64)
    o = np.asarray(im.origin, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.float64)[..., None, None]
    cols = np.asarray(cols, dtype=np.float64)[..., None, None]
    ou = np.asarray(ou, dtype=np.float64)[..., None, None]
    ov = np.asarray(ov, dtype=np.float64)[..., None, None]
    uu = cols + ou + s * 0.5 * (1.0 + u[:, None])      # axis -2: column node a
    vv = rows + ov + s * 0.5 * (1.0 + u[None, :])      # axis -1: row node b
    x = o[0] + A[0, 0] * uu + A[0, 1] * vv
    y = o[1] + A[1, 0] * uu + A[1, 1] * vv
    I, _ = profile(src.type, slot_values(src, theta), x, y, im, False)
    W2 = 0.25 * w[:, None] * w[None, :]
    return det_A(im) * s * s * np.einsum("...ab,ab->...", I, W2)


def render_source_adaptive(problem, src, theta, tol: float, margin: float = 0.01, near_abs: float = 0.0):
    """Adaptive pixel integration of one source on its sampling box.

    Returns (box, values[nr, nc], levels[nr, nc], near[nr, nc]): levels 0
    midpoint, 1 order 3, 2 split 5 x 5 with order 5, 3 with sub-pixels split
    again (order 7); near marks pixels where one of the decisions taken was
    within margin (relative) + near_abs x the size of the compared values of
    its threshold, where a rounding difference may decide it the other way
    (a caller computing in another precision may then take the other level;
    both results are within the budget's reach of each other).  margin and
    near_abs only mark pixels: they change no value."""
    box = source_box(problem, src)
    r0, r1, c0, c1 = box
    nr, nc = max(r1 - r0, 0), max(c1 - c0, 0)
    vals = np.zeros((nr, nc))
    levels = np.zeros((nr, nc), dtype=np.int8)
    near = np.zeros((nr, nc), dtype=bool)
    if nr == 0 or nc == 0:
        return box, vals, levels, near
    R, C = np.meshgrid(np.arange(r0, r1, dtype=np.float64), np.arange(c0, c1, dtype=np.float64), indexing="ij")
    v0 = rect_values(problem, src, theta, R, C, 0.0, 0.0, 1.0, 1)
    vals[:] = v0
    if src.type in (SKY_FLAT, SKY_PLANE):
        return box, vals, levels, near
    e = tol * abs(v0.sum()) / (nr * nc)

    def is_near(crit, thr, scale):
        return abs(crit - thr) <= margin * thr + near_abs * scale

    L = np.zeros((nr, nc))
    for a in range(nr):
        if nr >= 3:
            m = min(max(a, 1), nr - 2)          # centre of the three rows used
            L[a, :] += v0[m - 1, :] - 2.0 * v0[m, :] + v0[m + 1, :]
    for b in range(nc):
        if nc >= 3:
            m = min(max(b, 1), nc - 2)
            L[:, b] += v0[:, m - 1] - 2.0 * v0[:, m] + v0[:, m + 1]
    d0 = np.abs(L) / 24.0
    near |= np.abs(d0 - e) <= margin * e + near_abs * np.abs(v0) / 6.0
    for a, b in zip(*np.nonzero(d0 > e)):
        i, j = r0 + a, c0 + b
        v1 = float(rect_values(problem, src, theta, np.array(i), np.array(j), 0.0, 0.0, 1.0, 3))
        w1 = float(rect_values(problem, src, theta, np.array(i), np.array(j), 0.0, 0.0, 1.0, 2))
        near[a, b] |= is_near(abs(v1 - w1), e, abs(v1))
        if abs(v1 - w1) <= e:
            vals[a, b], levels[a, b] = v1, 1
            continue
        sub = 1.0 / ADAPT_SPLIT
        qy, qx = np.meshgrid(np.arange(ADAPT_SPLIT), np.arange(ADAPT_SPLIT), indexing="ij")
        qy, qx = qy.ravel(), qx.ravel()          # q = qy * 5 + qx
        ii, jj = np.full(qx.size, float(i)), np.full(qx.size, float(j))
        g5 = rect_values(problem, src, theta, ii, jj, qx * sub, qy * sub, sub, 5)      # one value per sub-pixel
        g4 = rect_values(problem, src, theta, ii, jj, qx * sub, qy * sub, sub, 4)
        v2 = g5.sum()
        near[a, b] |= is_near(abs(v2 - g4.sum()), e, abs(v2))
        if abs(v2 - g4.sum()) <= e:
            vals[a, b], levels[a, b] = v2, 2
            continue
        total = 0.0
        for q in range(qx.size):
            near[a, b] |= is_near(abs(g5[q] - g4[q]), e / ADAPT_SPLIT ** 2, abs(g5[q]))
            if abs(g5[q] - g4[q]) > e / ADAPT_SPLIT ** 2:
                s2 = sub / ADAPT_SPLIT
                py, px = np.meshgrid(np.arange(ADAPT_SPLIT), np.arange(ADAPT_SPLIT), indexing="ij")
                total += float(rect_values(problem, src, theta, np.full(px.size, float(i)), np.full(px.size, float(j)),
                                           qx[q] * sub + px.ravel() * s2, qy[q] * sub + py.ravel() * s2, s2, 7).sum())
            else:
                total += g5[q]
        vals[a, b], levels[a, b] = total, 3
    return box, vals, levels, near


def model_layers_adaptive(problem, theta, tol: float, margin: float = 0.01, near_abs: float = 0.0) -> List[dict]:
    """model_layers() with every source sampled by adaptive pixel
    integration (per image: G, U, M, m and the per-source boxes, levels and
    near-threshold flags)."""
    out = []
    for ii, im in enumerate(problem.images):
        h = psf_half(im)
        G = np.zeros((im.H + 2 * h, im.W + 2 * h))
        U = np.zeros((im.H, im.W))
        per_src = {}
        for k, src in enumerate(problem.sources):
            if src.image != ii:
                continue
            (r0, r1, c0, c1), vals, lev, near = render_source_adaptive(problem, src, theta, tol, margin, near_abs)
            per_src[k] = ((r0, r1, c0, c1), vals, lev, near)
            if vals.size == 0:
                continue
            if is_convolved(problem, src):
                G[r0 + h: r1 + h, c0 + h: c1 + h] += vals
            else:
                U[r0:r1, c0:c1] += vals
        M = convolve_layer(G, image_psf(problem, ii, theta)[0], im.H, im.W) if im.psf is not None else np.zeros_like(U)
        out.append(dict(G=G, U=U, M=M, m=M + U, sources=per_src))
    return out


def chi2_adaptive(problem, theta, tol: float) -> np.ndarray:
    """chi^2 per group of the adaptively integrated model."""
    out = np.zeros(problem.n_groups)
    for im, L in zip(problem.images, model_layers_adaptive(problem, theta, tol)):
        r = np.asarray(im.data, dtype=np.float64) - L["m"]
        out[im.group] += float((weights(im) * r * r).sum())
    return out
