"""The C-ABI library builds for sm_103a, loads, and exports every entry point
the header declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "astrophot_gb300.h")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s*(ap_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("ap_create", "ap_set_problem", "ap_render", "ap_eval", "ap_normal_eq", "ap_lm_solve",
              "ap_lm_iterate", "ap_get_status", "ap_destroy"):
        assert n in names


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2308_01957_gb300 import build
    path = build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    for n in declared():
        assert hasattr(lib, n), n


def test_binding_signatures_cover_the_header(lib):
    from paper_2308_01957_gb300 import _lib
    assert sorted(_lib.EXPORTED) == declared()
    L = _lib.load()
    assert L.ap_strerror(0) == b"ok"
    assert L.ap_strerror(3).startswith(b"damped")


def test_create_without_gpu_fails_cleanly(lib):
    """ap_create on a machine without a usable device returns an error code
    (no abort), and invalid options are rejected before touching the GPU."""
    from paper_2308_01957_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p()
    bad = _lib.ApOptions(7, 3, 0, 0, 0)
    assert L.ap_create(ctypes.byref(h), ctypes.byref(bad)) == _lib.AP_ERR_ARG
    bad_q = _lib.ApOptions(0, 4, 0, 0, 0)
    assert L.ap_create(ctypes.byref(h), ctypes.byref(bad_q)) == _lib.AP_ERR_ARG
    bad_j = _lib.ApOptions(0, 3, 0, 0, 0, 3)
    assert L.ap_create(ctypes.byref(h), ctypes.byref(bad_j)) == _lib.AP_ERR_ARG
    bad_v = _lib.ApOptions(0, 3, 0, 0, 0, 0, 99)
    assert L.ap_create(ctypes.byref(h), ctypes.byref(bad_v)) == _lib.AP_ERR_ARG
    # the variant table needs no context state
    n = ctypes.c_int()
    assert L.ap_get_conv_variant(None, None, ctypes.byref(n), None, None) == _lib.AP_ERR_ARG


def test_struct_layouts_match_header():
    from paper_2308_01957_gb300 import _lib
    # precision, quad_order, device, tile_w, tile_h, jcol_mode, conv_variant, gram_tc_min
    assert ctypes.sizeof(_lib.ApOptions) == 8 * 4
    # int H, W; double A[4]; double origin[2]; 4 pointers; int K; int group; int psf_live;
    # int psf_pidx[2]; (pad); double psf_pfix[2]
    assert ctypes.sizeof(_lib.ApImageDesc) == 8 + 32 + 16 + 32 + 8 + 4 + 8 + 4 + 16
    # int type, image, win[4], psf_convolve, pidx[8]; (pad) double pfix[8]
    assert ctypes.sizeof(_lib.ApSourceDesc) == 4 * 15 + 4 + 64


def _header_params():
    """Parameter count of every declared entry point (from the header text)."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"^\s*(?:int|void|const char\s*\*)\s*(ap_\w+)\s*\(([^)]*)\)\s*;", text, re.M):
        args = [a for a in m.group(2).split(",") if a.strip() and a.strip() != "void"]
        out[m.group(1)] = len(args)
    return out


def test_binding_argument_counts_match_the_header(lib):
    """Every ctypes signature marshals as many arguments as the C declaration
    takes (a missing or extra argument would shift every one after it)."""
    from paper_2308_01957_gb300 import _lib
    L = _lib.load()
    params = _header_params()
    assert set(params) == set(_lib.EXPORTED)
    for name, n in params.items():
        fn = getattr(L, name)
        assert fn.argtypes is not None and len(fn.argtypes) == n, (name, n, fn.argtypes)


def test_null_context_is_rejected_by_every_call(lib):
    """Each call that takes a context returns AP_ERR_ARG for a NULL one,
    before any device work (so this runs without a GPU)."""
    from paper_2308_01957_gb300 import _lib
    L = _lib.load()
    for name in _lib.EXPORTED:
        fn = getattr(L, name)
        if fn.restype is not ctypes.c_int or not fn.argtypes or fn.argtypes[0] is not ctypes.c_void_p:
            continue
        if name in ("ap_create", "ap_lm_solve_noalloc"):
            continue
        args = [0.0 if t is ctypes.c_double else (0 if t in (ctypes.c_int, ctypes.c_int64) else None)
                for t in fn.argtypes]
        assert fn(*args) == _lib.AP_ERR_ARG, name
