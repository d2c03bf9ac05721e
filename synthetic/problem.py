"""Plain containers for a forward-modelling problem: images, sources, parameter vector.

This module holds data only.  It performs none of the method's arithmetic: no
profile, quadrature, convolution or likelihood code lives here.  Both the CPU
oracle and the GPU binding read these objects by attribute (duck typing), so
neither has to import the other.

Conventions (the method's problem statement, Sec. "Image Modeling",
"chi^2 Optimization" and the multi-band example of the paper):

* An image has ``H`` rows and ``W`` columns, stored row-major.  Row ``i`` and
  column ``j`` name the pixel whose centre sits at world position
  ``origin + A @ (j + 1/2, i + 1/2)``: ``A`` is the 2x2 pixel-scale matrix
  (rotation and skew allowed), ``origin`` the world position of the image's
  bottom-left corner.
* ``variance`` is the per-pixel sigma^2 map, ``mask`` (optional, uint8) marks
  excluded pixels with 1, ``psf`` (optional) is an odd KxK image, centre at
  ((K-1)/2, (K-1)/2), not necessarily normalised.
* ``group`` names the independent fitting problem an image belongs to: images
  of one group share one chi^2 and one Levenberg-Marquardt state.
* A source has a profile ``type`` (codes below), the ``image`` it is drawn on,
  a half-open pixel window ``win = (x0, x1, y0, y1)`` (columns x0..x1-1, rows
  y0..y1-1), a ``psf_convolve`` flag and, for each of its parameter slots,
  either an index into theta (``pidx[k] >= 0``; several sources may share an
  index) or a fixed value (``pidx[k] == -1``, value in ``pfix[k]``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# Profile type codes shared by every consumer of a problem description.
SERSIC = 0        # slots: x0, y0, q, PA, n, Re, Ie
EXPONENTIAL = 1   # slots: x0, y0, q, PA, Re, Ie
GAUSSIAN = 2      # slots: x0, y0, q, PA, sigma, F
MOFFAT = 3        # slots: x0, y0, q, PA, n, Rd, F
SKY_FLAT = 4      # slots: S
SKY_PLANE = 5     # slots: S, gx, gy
PSF_STAR = 6      # slots: x0, y0, F   (the image's PSF image as a pixel map)

N_SLOTS = {SERSIC: 7, EXPONENTIAL: 6, GAUSSIAN: 6, MOFFAT: 7, SKY_FLAT: 1, SKY_PLANE: 3, PSF_STAR: 3}
SLOT_NAMES = {
    SERSIC: ("x0", "y0", "q", "PA", "n", "Re", "Ie"),
    EXPONENTIAL: ("x0", "y0", "q", "PA", "Re", "Ie"),
    GAUSSIAN: ("x0", "y0", "q", "PA", "sigma", "F"),
    MOFFAT: ("x0", "y0", "q", "PA", "n", "Rd", "F"),
    SKY_FLAT: ("S",),
    SKY_PLANE: ("S", "gx", "gy"),
    PSF_STAR: ("x0", "y0", "F"),
}
MAX_SLOTS = 8


@dataclass
class ImageSpec:
    H: int
    W: int
    A: np.ndarray                      # (2, 2) float64, pixel -> world
    origin: np.ndarray                 # (2,) float64
    psf: Optional[np.ndarray] = None   # (K, K) float32
    mask: Optional[np.ndarray] = None  # (H, W) uint8, 1 = excluded
    group: int = 0
    data: Optional[np.ndarray] = None      # (H, W) float32
    variance: Optional[np.ndarray] = None  # (H, W) float32
    # a live PSF: a circular Moffat (n, Rd) built from theta (psf_pidx[k] >= 0)
    # or fixed values (psf_pidx[k] = -1, value in psf_pfix[k]); psf then only
    # gives its K x K size
    psf_pidx: Optional[np.ndarray] = None  # (2,) int64
    psf_pfix: Optional[np.ndarray] = None  # (2,) float64


@dataclass
class SourceSpec:
    type: int
    image: int
    win: tuple                 # (x0, x1, y0, y1) half-open pixel box
    psf_convolve: bool
    pidx: np.ndarray           # (8,) int64, -1 = fixed
    pfix: np.ndarray           # (8,) float64


@dataclass
class Problem:
    name: str
    images: List[ImageSpec]
    sources: List[SourceSpec]
    n_params: int
    theta_true: np.ndarray
    theta_init: np.ndarray
    quad_order: int = 3
    # per image: standard normal draws for the noise and the additive
    # variance floor of the noise model var = model + floor
    noise: List[np.ndarray] = field(default_factory=list)
    var_floor: List[float] = field(default_factory=list)
    note: str = ""
    # noise model var = (model + floor) * var_scale, and the quadrature order
    # the data are rendered with (0: the fit's own)
    var_scale: float = 1.0
    data_quad_order: int = 0

    @property
    def n_groups(self) -> int:
        return 1 + max(im.group for im in self.images)

    def param_group(self) -> np.ndarray:
        """Group of every theta index (the group of the first source using it)."""
        g = np.full(self.n_params, -1, dtype=np.int64)
        for s in self.sources:
            for k in range(N_SLOTS[s.type]):
                p = int(s.pidx[k])
                if p >= 0 and g[p] < 0:
                    g[p] = self.images[s.image].group
        for im in self.images:   # live PSF parameters (after every source)
            if im.psf_pidx is not None:
                for p in im.psf_pidx:
                    if p >= 0 and g[p] < 0:
                        g[p] = im.group
        return g


def attach_data(problem: Problem, model_images: List[np.ndarray]) -> None:
    """Fill data and variance from noise-free model images and stored noise draws.

    The noise model of the workloads: var = (model + floor) var_scale,
    d = model + sqrt(var) z, stored as float32.  ``model_images`` may come from
    any renderer; the draws ``z`` are fixed by the problem's seed.
    """
    for im, m, z, floor in zip(problem.images, model_images, problem.noise, problem.var_floor):
        m = np.asarray(m, dtype=np.float64)
        var = (np.maximum(m, 0.0) + floor) * problem.var_scale
        im.variance = var.astype(np.float32)
        im.data = (m + np.sqrt(var) * z).astype(np.float32)
