"""Python face of libastrophot_gb300: a context object and a torch.autograd.Function.

PyTorch provides device memory and streams; every computation happens in the
library's kernels behind the C ABI (include/astrophot_gb300.h).  Images are
read by attribute (H, W, A, origin, group, data, variance, mask, psf); sources
by (type, image, win, psf_convolve, pidx, pfix).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L


@dataclass
class DeviceImage:
    """An image whose planes live on the GPU (float32 data / variance / PSF,
    uint8 mask)."""
    H: int
    W: int
    A: np.ndarray
    origin: np.ndarray
    group: int
    data: torch.Tensor
    variance: torch.Tensor
    mask: Optional[torch.Tensor]
    psf: Optional[torch.Tensor]
    psf_pidx: Optional[np.ndarray] = None   # live PSF: theta indices of (n, Rd), -1 = fixed
    psf_pfix: Optional[np.ndarray] = None   # live PSF: values of fixed slots


def to_device_images(images, device="cuda") -> List[DeviceImage]:
    """Copy host images (numpy planes) to the GPU as DeviceImage objects."""
    out = []
    for im in images:
        t = lambda a, dt: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(device)
        out.append(DeviceImage(int(im.H), int(im.W), np.asarray(im.A, float), np.asarray(im.origin, float),
                               int(im.group), t(im.data, torch.float32), t(im.variance, torch.float32),
                               t(im.mask, torch.uint8), t(im.psf, torch.float32),
                               getattr(im, "psf_pidx", None), getattr(im, "psf_pfix", None)))
    return out


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("library arguments must be contiguous CUDA tensors")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


class Context:
    """One problem on one GPU.  precision: "mixed" (float32 render, convolution
    and Jacobian; float64 reductions and solve) or "f64" (all float64)."""

    JCOL_MODES = {"auto": 0, "direct": 1, "fft": 2}

    def __init__(self, precision: str = "mixed", quad_order: int = 3, device: int = 0, tile=None,
                 jcol: str = "auto", conv_variant=None, gram_tc_min: int = 0):
        self.lib = L.load()
        self.f64 = precision == "f64"
        self.device = torch.device("cuda", device)
        opt = L.ApOptions(L.AP_PREC_F64 if self.f64 else L.AP_PREC_MIXED, int(quad_order), int(device),
                          int(tile[0]) if tile else 0, int(tile[1]) if tile else 0, self.JCOL_MODES[jcol],
                          0 if conv_variant is None else int(conv_variant) + 1, int(gram_tc_min))
        h = C.c_void_p()
        L.check(self.lib.ap_create(C.byref(h), C.byref(opt)), "ap_create")
        self.h = h
        self._keep = []
        self.n_params = 0
        self.n_groups = 0
        self.images = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.ap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- problem ---------------------------------------------------------
    def set_problem(self, images: Sequence, sources: Sequence, n_params: int, stream=None):
        imgs = (L.ApImageDesc * len(images))()
        for k, im in enumerate(images):
            d = imgs[k]
            d.H, d.W = int(im.H), int(im.W)
            A = np.asarray(im.A, dtype=np.float64).reshape(4)
            for a in range(4):
                d.A[a] = float(A[a])
            d.origin[0], d.origin[1] = float(im.origin[0]), float(im.origin[1])
            d.data_dev, d.variance_dev = _ptr(im.data), _ptr(im.variance)
            d.mask_dev = _ptr(im.mask)
            d.psf_dev = _ptr(im.psf)
            d.K = 0 if im.psf is None else int(im.psf.shape[0])
            d.group = int(im.group)
            live = getattr(im, "psf_pidx", None)
            if live is not None:
                d.psf_live = 1
                for k in range(2):
                    d.psf_pidx[k] = int(live[k])
                    d.psf_pfix[k] = float(im.psf_pfix[k])
        srcs = (L.ApSourceDesc * max(len(sources), 1))()
        for k, s in enumerate(sources):
            d = srcs[k]
            d.type, d.image = int(s.type), int(s.image)
            for a in range(4):
                d.win[a] = int(s.win[a])
            d.psf_convolve = 1 if s.psf_convolve else 0
            for a in range(8):
                d.pidx[a] = int(s.pidx[a])
                d.pfix[a] = float(s.pfix[a])
        L.check(self.lib.ap_set_problem(self.h, imgs, len(images), srcs, len(sources), int(n_params),
                                        _stream(stream)), "ap_set_problem", self.h)
        self._keep = [images]
        self.images = list(images)
        self.n_src = len(sources)
        self.n_params = int(n_params)
        ng = C.c_int()
        pg = np.zeros(max(n_params, 1), dtype=np.int32)
        L.check(self.lib.ap_get_layout(self.h, C.byref(ng), pg.ctypes.data_as(C.POINTER(C.c_int))), "ap_get_layout",
                self.h)
        self.n_groups = ng.value
        self.param_group = pg[:n_params].copy()
        self._pg_dev = torch.as_tensor(self.param_group.astype(np.int64), device=self.device)

    def _theta(self, theta) -> torch.Tensor:
        t = torch.as_tensor(theta, dtype=torch.float64, device=self.device).contiguous()
        if t.numel() != self.n_params:
            raise ValueError(f"theta has {t.numel()} entries, problem has {self.n_params}")
        return t

    # -- calls -----------------------------------------------------------
    def render(self, theta, stream=None) -> List[torch.Tensor]:
        th = self._theta(theta)
        dt = torch.float64 if self.f64 else torch.float32
        outs = [torch.empty((im.H, im.W), dtype=dt, device=self.device) for im in self.images]
        arr = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        L.check(self.lib.ap_render(self.h, th.data_ptr(), arr, _stream(stream)), "ap_render", self.h)
        return outs

    def adaptive_layout(self):
        """(sample count, first sample of each source or -1) of the adaptive
        pixel integration: a source's samples cover its sampling box
        row-major."""
        n = C.c_int64()
        off = np.zeros(max(self.n_src, 1), dtype=np.int64)
        L.check(self.lib.ap_get_adaptive_layout(self.h, C.byref(n), off.ctypes.data), "ap_get_adaptive_layout", self.h)
        return n.value, off[: self.n_src]

    def eval_adaptive(self, theta, tol: float = 0.01, model: bool = False, levels: bool = False,
                      counts: bool = False, stream=None):
        """chi^2 per group of the model sampled by adaptive pixel integration
        (budget tol); optionally the model images, each sample's final level
        and the per-level counts.  Returns a dict with keys chi2, model,
        levels, counts (None where not asked)."""
        th = self._theta(theta)
        chi2 = torch.empty(self.n_groups, dtype=torch.float64, device=self.device)
        dt = torch.float64 if self.f64 else torch.float32
        outs = [torch.empty((im.H, im.W), dtype=dt, device=self.device) for im in self.images] if model else None
        arr = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs]) if model else None
        lev = None
        if levels:
            n, _ = self.adaptive_layout()
            lev = torch.empty(max(n, 1), dtype=torch.uint8, device=self.device)[:n]
        cnt = np.zeros(5, dtype=np.int64) if counts else None
        L.check(self.lib.ap_eval_adaptive(self.h, th.data_ptr(), float(tol), chi2.data_ptr(), arr,
                                          lev.data_ptr() if lev is not None else None,
                                          cnt.ctypes.data if counts else None, _stream(stream)),
                "ap_eval_adaptive", self.h)
        return {"chi2": chi2, "model": outs, "levels": lev, "counts": cnt}

    SHIFT_METHODS = {"lanczos3": 1, "bilinear": 2}

    def eval_shifted(self, theta, method: str = "lanczos3", model: bool = False, stream=None):
        """chi^2 per group (and optionally the model images) with every
        convolved profile source sampled at its pixel-centred position and
        moved back by Lanczos-3 or bilinear interpolation (ap_eval_shifted)."""
        th = self._theta(theta)
        chi2 = torch.empty(self.n_groups, dtype=torch.float64, device=self.device)
        dt = torch.float64 if self.f64 else torch.float32
        outs = [torch.empty((im.H, im.W), dtype=dt, device=self.device) for im in self.images] if model else None
        arr = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs]) if model else None
        L.check(self.lib.ap_eval_shifted(self.h, th.data_ptr(), self.SHIFT_METHODS[method], chi2.data_ptr(), arr,
                                         _stream(stream)), "ap_eval_shifted", self.h)
        return chi2, outs

    def eval(self, theta, grad: bool = True, stream=None, out=None):
        th = self._theta(theta)
        if out is None:
            chi2 = torch.empty(self.n_groups, dtype=torch.float64, device=self.device)
            g = torch.empty(self.n_params, dtype=torch.float64, device=self.device) if grad else None
        else:
            chi2, g = out
        L.check(self.lib.ap_eval(self.h, th.data_ptr(), chi2.data_ptr(), g.data_ptr() if g is not None else None,
                                 _stream(stream)), "ap_eval", self.h)
        return chi2, g

    def normal_eq(self, theta, stream=None):
        """J^T W r (device tensor) and J^T W J as CSR (row_ptr, col_idx host arrays, values device tensor)."""
        th = self._theta(theta)
        jtwr = torch.empty(self.n_params, dtype=torch.float64, device=self.device)
        L.check(self.lib.ap_normal_eq(self.h, th.data_ptr(), jtwr.data_ptr(), _stream(stream)), "ap_normal_eq", self.h)
        nnz = C.c_int64()
        L.check(self.lib.ap_get_jtwj_nnz(self.h, C.byref(nnz)), "ap_get_jtwj_nnz", self.h)
        row_ptr = np.zeros(self.n_params + 1, dtype=np.int64)
        col_idx = np.zeros(max(nnz.value, 1), dtype=np.int32)
        L.check(self.lib.ap_get_jtwj_structure(self.h, row_ptr.ctypes.data, col_idx.ctypes.data),
                "ap_get_jtwj_structure", self.h)
        vals = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=self.device)
        L.check(self.lib.ap_copy_jtwj(self.h, vals.data_ptr(), _stream(stream)), "ap_copy_jtwj", self.h)
        return jtwr, (row_ptr, col_idx[: nnz.value], vals[: nnz.value])

    def jtwj_nnz(self) -> int:
        """Stored entries of J^T W J (both triangles)."""
        nnz = C.c_int64()
        L.check(self.lib.ap_get_jtwj_nnz(self.h, C.byref(nnz)), "ap_get_jtwj_nnz", self.h)
        return int(nnz.value)

    def jtwj_dense(self, csr) -> np.ndarray:
        row_ptr, col_idx, vals = csr
        v = vals.cpu().numpy()
        M = np.zeros((self.n_params, self.n_params))
        for r in range(self.n_params):
            a, b = row_ptr[r], row_ptr[r + 1]
            M[r, col_idx[a:b]] = v[a:b]
        return M

    def lm_solve(self, lam, stream=None):
        lam_t = torch.as_tensor(lam, dtype=torch.float64, device=self.device).reshape(self.n_groups).clone()
        delta = torch.empty(self.n_params, dtype=torch.float64, device=self.device)
        L.check(self.lib.ap_lm_solve(self.h, lam_t.data_ptr(), delta.data_ptr(), _stream(stream)), "ap_lm_solve",
                self.h)
        return delta, lam_t

    def lm_iterate(self, theta, lam, n_iter: int, log: bool = False, stream=None):
        th = self._theta(theta).clone()
        lam_t = torch.as_tensor(lam, dtype=torch.float64, device=self.device).reshape(self.n_groups).clone()
        chi2 = torch.empty(self.n_groups, dtype=torch.float64, device=self.device)
        log_buf = np.zeros((max(n_iter, 1), self.n_groups, 4)) if log else None
        L.check(self.lib.ap_lm_iterate(self.h, th.data_ptr(), lam_t.data_ptr(), chi2.data_ptr(), int(n_iter),
                                       log_buf.ctypes.data if log else None, _stream(stream)),
                "ap_lm_iterate", self.h)
        return th, lam_t, chi2, (log_buf[:n_iter] if log else None)

    def lm_continue(self, n_iter: int, log: bool = False, stream=None):
        """n_iter more LM iterations of the fit the last lm_iterate() /
        lm_continue() left in the context (image data unchanged since);
        returns (theta, lambda, chi2, log) after them."""
        th = torch.empty(self.n_params, dtype=torch.float64, device=self.device)
        lam_t = torch.empty(self.n_groups, dtype=torch.float64, device=self.device)
        chi2 = torch.empty(self.n_groups, dtype=torch.float64, device=self.device)
        log_buf = np.zeros((max(n_iter, 1), self.n_groups, 4)) if log else None
        L.check(self.lib.ap_lm_continue(self.h, th.data_ptr(), lam_t.data_ptr(), chi2.data_ptr(), int(n_iter),
                                        log_buf.ctypes.data if log else None, _stream(stream)),
                "ap_lm_continue", self.h)
        return th, lam_t, chi2, (log_buf[:n_iter] if log else None)

    def jcol_mode(self):
        """("direct" or "fft", ms of one direct launch, ms of one FFT launch)
        as planned by set_problem (-1 where not timed)."""
        return self.jcol_plan()[:3]

    def jcol_plan(self):
        """jcol_mode() plus the FFT mode's block counts (64^2, 128^2)."""
        m, a, b, n64, n128 = C.c_int(), C.c_double(), C.c_double(), C.c_int(), C.c_int()
        L.check(self.lib.ap_get_jcol_mode(self.h, C.byref(m), C.byref(a), C.byref(b), C.byref(n64), C.byref(n128)),
                "ap_get_jcol_mode", self.h)
        return ("fft" if m.value == 2 else "direct"), a.value, b.value, n64.value, n128.value

    def conv_variant(self):
        """(variant the context runs, [(tile_w, tile_h, threads) per variant],
        [autotuner ms per variant, -1 where not timed])."""
        v, n = C.c_int(), C.c_int()
        L.check(self.lib.ap_get_conv_variant(self.h, C.byref(v), C.byref(n), None, None), "ap_get_conv_variant", self.h)
        shp = (C.c_int * (3 * n.value))()
        ms = (C.c_double * n.value)()
        L.check(self.lib.ap_get_conv_variant(self.h, C.byref(v), C.byref(n), shp, ms), "ap_get_conv_variant", self.h)
        return v.value, [tuple(shp[3 * k:3 * k + 3]) for k in range(n.value)], list(ms)

    def state(self):
        """(chi^2 per group of the last LM iteration, LM iterations run, CG
        iterations of each group's last solve)."""
        chi2 = np.zeros(max(self.n_groups, 1))
        its = C.c_int64()
        cg = np.zeros(max(self.n_groups, 1), dtype=np.int32)
        L.check(self.lib.ap_get_state(self.h, chi2.ctypes.data, C.byref(its), cg.ctypes.data), "ap_get_state", self.h)
        return chi2[: self.n_groups], its.value, cg[: self.n_groups]

    def status(self, stream=None) -> int:
        s = C.c_int()
        L.check(self.lib.ap_get_status(self.h, C.byref(s), _stream(stream)), "ap_get_status", self.h)
        return s.value

    def set_timing(self, on: bool):
        L.check(self.lib.ap_set_timing(self.h, 1 if on else 0), "ap_set_timing", self.h)

    def get_timing(self, counts: bool = False):
        """Average ms per launch by kernel name (and launch counts if asked)
        since the previous call."""
        names = C.create_string_buffer(4096)
        ms = (C.c_double * 64)()
        cnt = (C.c_int * 64)()
        n = C.c_int()
        L.check(self.lib.ap_get_timing(self.h, names, 4096, ms, cnt, 64, C.byref(n)), "ap_get_timing", self.h)
        keys = names.value.decode().split(";") if n.value else []
        avg = {k: ms[i] for i, k in enumerate(keys)}
        if counts:
            return avg, {k: cnt[i] for i, k in enumerate(keys)}
        return avg


class Chi2(torch.autograd.Function):
    """chi^2 per group as a differentiable function of theta; backward is the
    library's adjoint gradient (computed in the same forward call)."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, apctx: Context):
        chi2, grad = apctx.eval(theta.detach(), grad=True)
        ctx.save_for_backward(grad, apctx._pg_dev)
        return chi2

    @staticmethod
    def backward(ctx, gout):
        grad, pg = ctx.saved_tensors
        w = torch.where(pg >= 0, gout[pg.clamp(min=0)], torch.zeros_like(grad))
        return grad * w, None


def chi2(theta: torch.Tensor, apctx: Context) -> torch.Tensor:
    return Chi2.apply(theta, apctx)
