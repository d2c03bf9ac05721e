"""Seeded synthetic workloads standing in for the paper's images.

The paper fits real DESI / GALEX / unWISE images and GALFIT-made mocks; none
of them is available, so every workload here is drawn from a seed with the
shapes, sizes and parameter distributions of the paper's examples (Table 1 of
the GPU benchmark section, the LM/NUTS mock of the Bayesian section, the
seven-band joint fit).  The five named workloads are:

* ``single_sersic``   128x128, one Sersic + flat sky, 11x11 Gaussian PSF.
* ``field_1k``        1024x1024, 50 Sersic + 200 Moffat point sources, plane sky,
                      25x25 Moffat PSF.
* ``cutouts_256``     256 independent cutouts of side U{64..512}, 1-8 sources each,
                      own 15..31 Moffat PSF per cutout.
* ``crowded_4k``      4096x4096, 2000 Sersic + 5000 Moffat, 51x51 Moffat PSF with a
                      Gaussian wing, 2 % of pixels masked.
* ``joint_12x2k``     4 bands x 3 epochs of 2048x2048, rotated and dithered, shared
                      galaxy shapes and star positions, per-band fluxes.

This module only draws numbers: parameters, windows, PSF images, masks and
unit-normal noise draws.  The data image itself is formed by
``problem.attach_data`` from a noise-free model that the caller renders.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from .problem import (EXPONENTIAL, GAUSSIAN, MOFFAT, PSF_STAR, SERSIC, SKY_FLAT, SKY_PLANE,
                      ImageSpec, Problem, SourceSpec)

SEED_BASE = 2308019570


# --------------------------------------------------------------------------
# small helpers (input synthesis only)
# --------------------------------------------------------------------------

def _pidx(*idx):
    out = np.full(8, -1, dtype=np.int64)
    out[: len(idx)] = idx
    return out


def _pfix(**kw):
    return np.zeros(8, dtype=np.float64)


def moffat_rd(fwhm: float, beta: float) -> float:
    """Moffat core radius R_d for a given FWHM and index beta."""
    return fwhm / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0))


def psf_moffat(K: int, fwhm: float, beta: float = 3.0) -> np.ndarray:
    """Moffat PSF image sampled at pixel centres, unit sum, float32."""
    c = (K - 1) / 2.0
    y, x = np.mgrid[0:K, 0:K].astype(np.float64)
    r2 = (x - c) ** 2 + (y - c) ** 2
    p = (1.0 + r2 / moffat_rd(fwhm, beta) ** 2) ** (-beta)
    return (p / p.sum()).astype(np.float32)


def psf_gaussian(K: int, sigma: float) -> np.ndarray:
    c = (K - 1) / 2.0
    y, x = np.mgrid[0:K, 0:K].astype(np.float64)
    p = np.exp(-((x - c) ** 2 + (y - c) ** 2) / (2.0 * sigma * sigma))
    return (p / p.sum()).astype(np.float32)


def psf_moffat_wing(K: int, fwhm: float, wing_amp: float = 0.01, wing_sigma: float = 10.0):
    """Moffat core plus a broad Gaussian wing (each unit-sum, wing weighted)."""
    core = psf_moffat(K, fwhm).astype(np.float64)
    wing = psf_gaussian(K, wing_sigma).astype(np.float64)
    p = core + wing_amp * wing
    return (p / p.sum()).astype(np.float32)


def sersic_ie_from_flux(F, n, Re, q):
    """Invert the closed-form total Sersic flux 2 pi n Ie Re^2 q e^b Gamma(2n)/b^(2n)."""
    b = special.gammaincinv(2.0 * n, 0.5)
    tot_per_ie = 2.0 * math.pi * n * Re * Re * q * math.exp(b) * special.gamma(2.0 * n) / b ** (2.0 * n)
    return F / tot_per_ie


def _world_to_pixel(A, origin, xy):
    """Continuous (column, row) coordinate of a world point; pixel j spans [j, j+1)."""
    return np.linalg.solve(A, np.asarray(xy, dtype=np.float64) - origin)


def window_for(A, origin, H, W, xy, half):
    """Half-open pixel box of half-size ``half`` around the pixel holding ``xy``,
    clipped to the image; None when it misses the image."""
    u, v = _world_to_pixel(A, origin, xy)
    jc, ic = int(math.floor(u)), int(math.floor(v))
    x0, x1 = max(jc - half, 0), min(jc + half + 1, W)
    y0, y1 = max(ic - half, 0), min(ic + half + 1, H)
    if x0 >= x1 or y0 >= y1:
        return None
    return (x0, x1, y0, y1)


def sersic_half_size(Re, pixscale=1.0):
    return int(min(max(math.ceil(6.0 * Re / pixscale), 16), 256))


STAR_HALF = 16


def _noise(rng, H, W):
    return rng.standard_normal((H, W), dtype=np.float32)


# --------------------------------------------------------------------------
# workload 1: one Sersic + flat sky (precision anchor)
# --------------------------------------------------------------------------

def single_sersic(seed: int = SEED_BASE + 1, H: int = 128, W: int = 128) -> Problem:
    rng = np.random.default_rng(seed)
    A = np.eye(2)
    origin = np.zeros(2)
    psf = psf_gaussian(11, 1.5)
    im = ImageSpec(H=H, W=W, A=A, origin=origin, psf=psf, group=0)
    theta = np.array([64.3, 63.8, 0.7, 0.6, 2.5, 12.0, 10.0, 1.0])
    gal = SourceSpec(SERSIC, 0, window_for(A, origin, H, W, theta[:2], sersic_half_size(12.0)),
                     True, _pidx(0, 1, 2, 3, 4, 5, 6), _pfix())
    sky = SourceSpec(SKY_FLAT, 0, (0, W, 0, H), False, _pidx(7), _pfix())
    s = rng.choice([-1.0, 1.0], size=theta.size)
    init = theta * (1.0 + 0.1 * s)
    return Problem("single_sersic", [im], [gal, sky], theta.size, theta, init, quad_order=3,
                   noise=[_noise(rng, H, W)], var_floor=[0.5],
                   note="128x128, Sersic n=2.5 Re=12 q=0.7 PA=0.6 Ie=10 + flat sky 1, Gaussian PSF 11x11 sigma 1.5")


# --------------------------------------------------------------------------
# crowded fields (workloads 2 and 4, and their reduced versions in tests)
# --------------------------------------------------------------------------

def _draw_sersic(rng, lo_xy, hi_xy, re_cap=None):
    x, y = rng.uniform(lo_xy, hi_xy, size=2)
    n = rng.uniform(0.5, 6.0)
    Re = math.exp(rng.uniform(math.log(2.0), math.log(40.0)))
    if re_cap is not None:
        Re = min(Re, re_cap)
    q = rng.uniform(0.2, 1.0)
    PA = rng.uniform(0.0, math.pi)
    F = 10.0 ** rng.normal(3.0, 1.0)
    Ie = sersic_ie_from_flux(F, n, Re, q)
    return np.array([x, y, q, PA, n, Re, Ie])


def _draw_star(rng, lo_xy, hi_xy):
    x, y = rng.uniform(lo_xy, hi_xy, size=2)
    F = math.exp(rng.uniform(math.log(1e1), math.log(1e4)))
    return np.array([x, y, F])


def _perturb_sersic(rng, p):
    q = float(np.clip(p[2] * rng.normal(1.0, 0.1), 0.2, 1.0))
    n = float(np.clip(p[4] + rng.normal(0.0, 0.3), 0.5, 6.0))
    return np.array([p[0] + rng.normal(0, 0.5), p[1] + rng.normal(0, 0.5), q,
                     p[3] + rng.normal(0, math.radians(5.0)), n,
                     p[5] * rng.normal(1.0, 0.1), p[6] * rng.normal(1.0, 0.1)])


def _perturb_star(rng, p):
    return np.array([p[0] + rng.normal(0, 0.3), p[1] + rng.normal(0, 0.3), p[2] * rng.normal(1.0, 0.1)])


def crowded_field(name, seed, H, W, n_sersic, n_moffat, psf, star_fwhm=3.0, beta=3.0,
                  mask_frac=0.0, sky=(1.0, 1e-4, 1e-4), var_floor=1.0, quad_order=3,
                  A=None, origin=None) -> Problem:
    """One image with n_sersic convolved Sersic galaxies, n_moffat unconvolved Moffat
    point sources (beta, FWHM fixed; x0, y0, F free) and a plane sky."""
    rng = np.random.default_rng(seed)
    A = np.eye(2) if A is None else np.asarray(A, dtype=np.float64)
    origin = np.zeros(2) if origin is None else np.asarray(origin, dtype=np.float64)
    mask = None
    if mask_frac > 0:
        mask = (rng.random((H, W)) < mask_frac).astype(np.uint8)
    im = ImageSpec(H=H, W=W, A=A, origin=origin, psf=psf, mask=mask, group=0)
    lo = np.array([0.0, 0.0])
    hi = np.array([float(W), float(H)])
    theta, init, sources = [], [], []
    Rd = moffat_rd(star_fwhm, beta)
    for _ in range(n_sersic):
        p = _draw_sersic(rng, lo, hi)
        win = window_for(A, origin, H, W, p[:2], sersic_half_size(p[5]))
        base = len(theta)
        theta.extend(p)
        init.extend(_perturb_sersic(rng, p))
        sources.append(SourceSpec(SERSIC, 0, win, True, _pidx(*range(base, base + 7)), _pfix()))
    for _ in range(n_moffat):
        p = _draw_star(rng, lo, hi)
        win = window_for(A, origin, H, W, p[:2], STAR_HALF)
        base = len(theta)
        theta.extend(p)
        init.extend(_perturb_star(rng, p))
        pfix = np.zeros(8)
        pfix[2], pfix[3], pfix[4], pfix[5] = 1.0, 0.0, beta, Rd
        sources.append(SourceSpec(MOFFAT, 0, win, False, _pidx(base, base + 1, -1, -1, -1, -1, base + 2), pfix))
    base = len(theta)
    theta.extend(sky)
    init.extend([sky[0] * rng.normal(1.0, 0.01), sky[1], sky[2]])
    sources.append(SourceSpec(SKY_PLANE, 0, (0, W, 0, H), False, _pidx(base, base + 1, base + 2), _pfix()))
    theta = np.asarray(theta)
    return Problem(name, [im], sources, theta.size, theta, np.asarray(init), quad_order=quad_order,
                   noise=[_noise(rng, H, W)], var_floor=[var_floor])


def field_1k(seed: int = SEED_BASE + 2) -> Problem:
    pr = crowded_field("field_1k", seed, 1024, 1024, 50, 200, psf_moffat(25, 3.0))
    pr.note = "1024x1024, 50 Sersic + 200 Moffat (beta 3, FWHM 3), plane sky, Moffat PSF 25x25"
    return pr


def crowded_4k(seed: int = SEED_BASE + 4) -> Problem:
    pr = crowded_field("crowded_4k", seed, 4096, 4096, 2000, 5000, psf_moffat_wing(51, 3.0),
                       mask_frac=0.02)
    pr.note = "4096x4096, 2000 Sersic + 5000 Moffat, 51x51 Moffat+Gaussian-wing PSF, 2% masked"
    return pr


# --------------------------------------------------------------------------
# workload 3: batched independent cutouts
# --------------------------------------------------------------------------

def cutouts(seed: int = SEED_BASE + 3, n_cut: int = 256, side_lo: int = 64, side_hi: int = 512,
            max_src: int = 8, name: str = "cutouts_256") -> Problem:
    rng = np.random.default_rng(seed)
    images, sources, theta, init, noise, floors = [], [], [], [], [], []
    for c in range(n_cut):
        s = int(rng.integers(side_lo, side_hi + 1))
        K = int(rng.choice(np.arange(15, 32, 2)))
        fwhm = rng.uniform(2.5, 4.0)
        im = ImageSpec(H=s, W=s, A=np.eye(2), origin=np.zeros(2), psf=psf_moffat(K, fwhm), group=c)
        images.append(im)
        lo = np.array([0.2 * s, 0.2 * s])
        hi = np.array([0.8 * s, 0.8 * s])
        n_src = int(rng.integers(1, max_src + 1))
        for _ in range(n_src):
            base = len(theta)
            if rng.random() < 0.5:
                p = _draw_sersic(rng, lo, hi, re_cap=s / 8.0)
                win = window_for(im.A, im.origin, s, s, p[:2], sersic_half_size(p[5]))
                theta.extend(p)
                init.extend(_perturb_sersic(rng, p))
                sources.append(SourceSpec(SERSIC, c, win, True, _pidx(*range(base, base + 7)), _pfix()))
            else:
                p = _draw_star(rng, lo, hi)
                win = window_for(im.A, im.origin, s, s, p[:2], STAR_HALF)
                theta.extend(p)
                init.extend(_perturb_star(rng, p))
                pfix = np.zeros(8)
                pfix[2], pfix[4], pfix[5] = 1.0, 3.0, moffat_rd(fwhm, 3.0)
                sources.append(SourceSpec(MOFFAT, c, win, False,
                                          _pidx(base, base + 1, -1, -1, -1, -1, base + 2), pfix))
        base = len(theta)
        theta.append(1.0)
        init.append(rng.normal(1.0, 0.01))
        sources.append(SourceSpec(SKY_FLAT, c, (0, s, 0, s), False, _pidx(base), _pfix()))
        noise.append(_noise(rng, s, s))
        floors.append(1.0)
    theta = np.asarray(theta)
    return Problem(name, images, sources, theta.size, theta, np.asarray(init), quad_order=3,
                   noise=noise, var_floor=floors,
                   note=f"{n_cut} cutouts, side U{{{side_lo}..{side_hi}}}, 1-{max_src} Sersic/Moffat + flat sky, own Moffat PSF 15..31")


# --------------------------------------------------------------------------
# workload 5: joint multi-band multi-epoch fit with shared parameters
# --------------------------------------------------------------------------

def joint(seed: int = SEED_BASE + 5, n_band: int = 4, n_epoch: int = 3, side: int = 2048,
          n_sersic: int = 300, n_star: int = 1000, K: int = 31, name: str = "joint_12x2k") -> Problem:
    rng = np.random.default_rng(seed)
    centre = np.array([0.0, 0.0])
    images, noise, floors = [], [], []
    for b in range(n_band):
        for e in range(n_epoch):
            phi = rng.uniform(0.0, 2.0 * math.pi)
            A = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
            dither = rng.uniform(0.0, 1.0, size=2)
            origin = centre - A @ np.array([side / 2.0, side / 2.0]) + dither
            fwhm = rng.uniform(2.5, 4.0)
            images.append(ImageSpec(H=side, W=side, A=A, origin=origin, psf=psf_moffat(K, fwhm), group=0))
            noise.append(_noise(rng, side, side))
            floors.append(1.0)
    # sources live inside the disc every rotated image covers
    rmax = 0.45 * side

    def draw_xy():
        while True:
            xy = rng.uniform(-rmax, rmax, size=2)
            if xy @ xy < rmax * rmax:
                return xy

    theta, init, sources = [], [], []
    for _ in range(n_sersic):
        xy = draw_xy()
        p = _draw_sersic(rng, xy, xy)
        p[0], p[1] = xy
        base = len(theta)
        pert = _perturb_sersic(rng, p)
        theta.extend(p[:6])
        init.extend(pert[:6])
        band_idx = []
        for b in range(n_band):
            band_idx.append(len(theta))
            Ie_b = p[6] * 10.0 ** rng.normal(0.0, 0.2)
            theta.append(Ie_b)
            init.append(Ie_b * rng.normal(1.0, 0.1))
        for i, im in enumerate(images):
            win = window_for(im.A, im.origin, im.H, im.W, p[:2], sersic_half_size(p[5]))
            if win is None:
                continue
            b = i // n_epoch
            sources.append(SourceSpec(SERSIC, i, win, True,
                                      _pidx(base, base + 1, base + 2, base + 3, base + 4, base + 5, band_idx[b]),
                                      _pfix()))
    for _ in range(n_star):
        xy = draw_xy()
        p = _draw_star(rng, xy, xy)
        p[0], p[1] = xy
        base = len(theta)
        pert = _perturb_star(rng, p)
        theta.extend(p[:2])
        init.extend(pert[:2])
        band_idx = []
        for b in range(n_band):
            band_idx.append(len(theta))
            Fb = p[2] * 10.0 ** rng.normal(0.0, 0.2)
            theta.append(Fb)
            init.append(Fb * rng.normal(1.0, 0.1))
        for i, im in enumerate(images):
            win = window_for(im.A, im.origin, im.H, im.W, p[:2], STAR_HALF)
            if win is None:
                continue
            b = i // n_epoch
            pfix = np.zeros(8)
            pfix[2], pfix[4], pfix[5] = 1.0, 3.0, moffat_rd(3.0, 3.0)
            sources.append(SourceSpec(MOFFAT, i, win, False,
                                      _pidx(base, base + 1, -1, -1, -1, -1, band_idx[b]), pfix))
    for i, im in enumerate(images):
        base = len(theta)
        theta.extend([1.0, 1e-4, 1e-4])
        init.extend([rng.normal(1.0, 0.01), 1e-4, 1e-4])
        sources.append(SourceSpec(SKY_PLANE, i, (0, im.W, 0, im.H), False, _pidx(base, base + 1, base + 2), _pfix()))
    theta = np.asarray(theta)
    return Problem(name, images, sources, theta.size, theta, np.asarray(init), quad_order=3,
                   noise=noise, var_floor=floors,
                   note=f"{n_band} bands x {n_epoch} epochs of {side}^2, rotated + dithered, {n_sersic} Sersic "
                        f"(shared shape, per-band Ie) + {n_star} stars (shared x,y, per-band F), per-image plane sky, Moffat PSF {K}")


# --------------------------------------------------------------------------
# small mixed problems for parity tests: every profile type, rotation, skew,
# masks, asymmetric PSF, shared parameters, several groups, ragged sizes
# --------------------------------------------------------------------------

def mixed_small(seed: int = SEED_BASE + 11, H: int = 45, W: int = 70, K: int = 7, rotate: bool = True,
                mask_frac: float = 0.05, n_images: int = 1, groups: int = 1, quad_order: int = 3,
                asym_psf: bool = True, psf_star: bool = True, live_psf: bool = False) -> Problem:
    """live_psf: every image's PSF is a live circular Moffat whose (n, Rd) are
    parameters shared by the images of a group and by their fixed-shape Moffat
    stars (no PSF stars then: their map would be the live PSF)."""
    rng = np.random.default_rng(seed)
    rng_star = np.random.default_rng(seed + 7777)   # PSF-star draws: the other draws stay as they were
    psf_star = psf_star and not live_psf
    images, noise, floors = [], [], []
    for i in range(n_images):
        if rotate:
            phi = rng.uniform(0, 2 * math.pi)
            sc = rng.uniform(0.8, 1.2)
            A = sc * np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
            A[0, 1] += 0.05  # a little skew
        else:
            A = np.eye(2)
        origin = -A @ np.array([W / 2.0, H / 2.0]) + rng.uniform(0, 1, size=2)
        psf = None
        if K > 0:
            psf = psf_moffat(K, 2.0).astype(np.float64)
            if asym_psf:
                psf = psf * (1.0 + 0.3 * rng.random(psf.shape))
                psf[0, 1] += 0.02
            psf = psf.astype(np.float32)
        mask = (rng.random((H, W)) < mask_frac).astype(np.uint8) if mask_frac > 0 else None
        images.append(ImageSpec(H=H, W=W, A=A, origin=origin, psf=psf, mask=mask, group=i % groups))
        noise.append(_noise(rng, H, W))
        floors.append(0.5)
    theta, init, sources = [], [], []

    def add(vals, pert):
        base = len(theta)
        theta.extend(vals)
        init.extend(pert)
        return list(range(base, base + len(vals)))

    live_idx = {}   # group -> theta indices of the live PSF's (n, Rd)
    for i, im in enumerate(images):
        conv = im.psf is not None
        def cxy():
            return rng.uniform(-0.3, 0.3, size=2) * np.array([W, H]) * 0.8
        # Sersic
        xy = cxy()
        p = [xy[0], xy[1], rng.uniform(0.4, 0.9), rng.uniform(0, math.pi), rng.uniform(0.7, 4.0),
             rng.uniform(2.0, 6.0), rng.uniform(2.0, 10.0)]
        idx = add(p, [p[0] + 0.3, p[1] - 0.2, p[2] * 1.05, p[3] + 0.05, p[4] * 1.1, p[5] * 0.95, p[6] * 1.1])
        win = window_for(im.A, im.origin, H, W, xy, 20)
        sources.append(SourceSpec(SERSIC, i, win, conv, _pidx(*idx), _pfix()))
        # exponential
        xy = cxy()
        p = [xy[0], xy[1], rng.uniform(0.3, 0.9), rng.uniform(0, math.pi), rng.uniform(2.0, 5.0), rng.uniform(1.0, 5.0)]
        idx = add(p, [p[0] - 0.2, p[1] + 0.3, p[2] * 0.95, p[3] - 0.05, p[4] * 1.05, p[5] * 0.9])
        sources.append(SourceSpec(EXPONENTIAL, i, window_for(im.A, im.origin, H, W, xy, 14), conv, _pidx(*idx), _pfix()))
        # Gaussian
        xy = cxy()
        p = [xy[0], xy[1], rng.uniform(0.5, 1.0), rng.uniform(0, math.pi), rng.uniform(1.0, 3.0), rng.uniform(20.0, 80.0)]
        idx = add(p, [p[0] + 0.1, p[1] + 0.1, p[2] * 0.97, p[3] + 0.02, p[4] * 1.05, p[5] * 1.1])
        sources.append(SourceSpec(GAUSSIAN, i, window_for(im.A, im.origin, H, W, xy, 12), conv, _pidx(*idx), _pfix()))
        # Moffat with all seven slots free (not convolved: a point source / PSF model)
        xy = cxy()
        p = [xy[0], xy[1], rng.uniform(0.7, 1.0), rng.uniform(0, math.pi), rng.uniform(2.0, 4.0), rng.uniform(1.0, 2.5),
             rng.uniform(30.0, 100.0)]
        idx = add(p, [p[0] + 0.2, p[1] - 0.1, p[2] * 0.98, p[3] + 0.03, p[4] * 1.05, p[5] * 1.05, p[6] * 0.9])
        sources.append(SourceSpec(MOFFAT, i, window_for(im.A, im.origin, H, W, xy, 10), False, _pidx(*idx), _pfix()))
        # a Moffat star with fixed shape (with a live PSF: the PSF's n and Rd)
        xy = cxy()
        idx = add([xy[0], xy[1], 50.0], [xy[0] + 0.1, xy[1] + 0.1, 45.0])
        pfix = np.zeros(8)
        pfix[2], pfix[3], pfix[4], pfix[5] = 1.0, 0.0, 3.0, moffat_rd(2.5, 3.0)
        star_pidx = _pidx(idx[0], idx[1], -1, -1, -1, -1, idx[2])
        if live_psf and im.psf is not None:
            if im.group not in live_idx:
                live_idx[im.group] = add([2.8, 1.9], [3.1, 1.75])
            star_pidx[4], star_pidx[5] = live_idx[im.group]
            im.psf_pidx = np.array(live_idx[im.group], dtype=np.int64)
            im.psf_pfix = np.zeros(2)
        sources.append(SourceSpec(MOFFAT, i, window_for(im.A, im.origin, H, W, xy, 8), False, star_pidx, pfix))
        # a point source drawn with the image's PSF image as its pixel map
        if psf_star and im.psf is not None:
            xy = rng_star.uniform(-0.3, 0.3, size=2) * np.array([W, H]) * 0.8
            F = rng_star.uniform(40.0, 90.0)
            idx = add([xy[0], xy[1], F], [xy[0] - 0.15, xy[1] + 0.1, F * 1.08])
            sources.append(SourceSpec(PSF_STAR, i, window_for(im.A, im.origin, H, W, xy, 9), False, _pidx(*idx),
                                      _pfix()))
        # plane sky on even images, flat on odd
        if i % 2 == 0:
            idx = add([0.5, 2e-3, -1e-3], [0.52, 2e-3, -1e-3])
            sources.append(SourceSpec(SKY_PLANE, i, (0, W, 0, H), False, _pidx(*idx), _pfix()))
        else:
            idx = add([0.7], [0.71])
            sources.append(SourceSpec(SKY_FLAT, i, (0, W, 0, H), False, _pidx(*idx), _pfix()))
    # a Sersic shared between image 0 and every other image of its group: shape
    # parameters shared, one Ie per image
    if n_images > 1:
        xy = np.array([1.5, -2.0])
        shape = [xy[0], xy[1], 0.6, 0.4, 1.5, 4.0]
        sidx = add(shape, [shape[0] + 0.2, shape[1] + 0.2, 0.62, 0.42, 1.6, 4.2])
        for i, im in enumerate(images):
            if im.group != images[0].group:
                continue
            ie = add([5.0 + i], [5.5 + i])
            win = window_for(im.A, im.origin, H, W, xy, 18)
            if win is None:
                continue
            sources.append(SourceSpec(SERSIC, i, win, im.psf is not None, _pidx(*sidx, ie[0]), _pfix()))
    theta = np.asarray(theta, dtype=np.float64)
    return Problem(f"mixed_small_s{seed}", images, [s for s in sources if s.win is not None], theta.size, theta,
                   np.asarray(init, dtype=np.float64), quad_order=quad_order, noise=noise, var_floor=floors)


# --------------------------------------------------------------------------
# the paper's GPU benchmark (Sec. "GPU acceleration", Table 1): overlapping
# Sersic models on a 1000 x 1000 image of pixel scale 1
# --------------------------------------------------------------------------

def table1(n_sersic: int = 16, seed: int = SEED_BASE + 6, quad_order: int = 3) -> Problem:
    """n_sersic Sersic models drawn as the paper's Table 1: X, Y ~ U(50, 950),
    q ~ U(0.3, 0.9), PA ~ U(0, 180) deg, n ~ U(0.5, 4), Re ~ 10^U(1.5, 2.5) px,
    Ie ~ 10^N(0, 0.5); initialised at X + N(0, 2), Y + N(0, 2), q N(1, 0.1),
    PA + N(0, 5 deg), n + N(0, 1), Re N(1, 0.1), Ie N(1, 0.1), q and n clipped
    back to their ranges.  Noise of sigma = sqrt(1 + f) / 10 (var = (f + 1) / 100,
    f the pixel's flux).  Readings: no PSF and no sky (the table lists none);
    the data's 5x-oversampled rendering is stood in for by order-7
    Gauss-Legendre on every pixel (data_quad_order); windows by the generator's
    Sersic rule (half-size clamp(6 Re, 16, 256))."""
    rng = np.random.default_rng(seed + n_sersic)
    H = W = 1000
    im = ImageSpec(H=H, W=W, A=np.eye(2), origin=np.zeros(2), psf=None, group=0)
    theta, init, sources = [], [], []
    for _ in range(n_sersic):
        x, y = rng.uniform(50.0, 950.0, size=2)
        q = rng.uniform(0.3, 0.9)
        PA = math.radians(rng.uniform(0.0, 180.0))
        n = rng.uniform(0.5, 4.0)
        Re = 10.0 ** rng.uniform(1.5, 2.5)
        Ie = 10.0 ** rng.normal(0.0, 0.5)
        p = [x, y, q, PA, n, Re, Ie]
        ini = [x + rng.normal(0.0, 2.0), y + rng.normal(0.0, 2.0), float(np.clip(q * rng.normal(1.0, 0.1), 0.3, 0.9)),
               PA + math.radians(rng.normal(0.0, 5.0)), float(np.clip(n + rng.normal(0.0, 1.0), 0.5, 4.0)),
               Re * rng.normal(1.0, 0.1), Ie * rng.normal(1.0, 0.1)]
        base = len(theta)
        theta.extend(p)
        init.extend(ini)
        win = window_for(im.A, im.origin, H, W, np.array([x, y]), sersic_half_size(Re))
        sources.append(SourceSpec(SERSIC, 0, win, False, _pidx(*range(base, base + 7)), _pfix()))
    theta = np.asarray(theta)
    pr = Problem(f"table1_{n_sersic}", [im], sources, theta.size, theta, np.asarray(init), quad_order=quad_order,
                 noise=[_noise(rng, H, W)], var_floor=[1.0], var_scale=0.01, data_quad_order=7,
                 note=f"the paper's Table 1 benchmark: {n_sersic} overlapping Sersic on 1000x1000, "
                      "sigma = sqrt(1 + f) / 10, ~10% perturbed start")
    return pr


WORKLOADS = {
    "single_sersic": single_sersic,
    "field_1k": field_1k,
    "cutouts_256": cutouts,
    "crowded_4k": crowded_4k,
    "joint_12x2k": joint,
}
WORKLOADS.update({f"table1_{n}": (lambda n=n: table1(n)) for n in (1, 16, 64)})
