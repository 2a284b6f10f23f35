"""CPU-side checks of the C ABI: the library loads, exports every function include/st.h
declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2009_08875_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "st.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(st_[a-z_A-Z0-9]+)\s*\(", txt)))


def lib_or_skip():
    try:
        return _lib.load()
    except ImportError as e:
        pytest.skip(str(e))


def test_header_declares_the_hot_path_entry_points():
    names = declared_functions()
    for n in ("st_setup", "st_apply_S", "st_apply_KX", "st_pcg_solve", "st_rhs", "st_synthesize", "st_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = lib_or_skip()
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_signatures_cover_the_header():
    assert set(declared_functions()) == set(_lib._SIGS)


def test_default_config_is_the_papers():
    lib = lib_or_skip()
    cfg = _lib.StConfig()
    lib.st_default_config(ctypes.byref(cfg))
    assert (cfg.alpha, cfg.n_vcycles, cfg.n_pre, cfg.n_post) == (0.3, 2, 3, 3)
    # the heat equation: D = Id, c = 0
    assert tuple(cfg.diffusion) == (1.0, 0.0, 1.0) and cfg.reaction == 0.0


@pytest.mark.parametrize("d11,d12,d22,c", [(0.0, 0.0, 1.0, 0.0), (1.0, 1.0, 1.0, 0.0), (1.0, 2.0, 1.0, 0.0),
                                           (-1.0, 0.0, -1.0, 0.0), (1.0, 0.0, 1.0, -0.5),
                                           (1.0, 0.0, float("nan"), 0.0)])
def test_setup_rejects_non_spd_D_or_negative_c_without_gpu(d11, d12, d22, c):
    lib = lib_or_skip()
    cfg = _lib.StConfig()
    lib.st_default_config(ctypes.byref(cfg))
    cfg.diffusion[0], cfg.diffusion[1], cfg.diffusion[2], cfg.reaction = d11, d12, d22, c
    h = ctypes.c_void_p()
    assert lib.st_setup(ctypes.byref(h), 0, 3, 3, ctypes.byref(cfg), None) == _lib.ST_ERR_ARG
    assert h.value is None
    assert "positive definite" in lib.st_last_error().decode()


@pytest.mark.parametrize("domain,K,J", [(3, 3, 3), (1, 1, 3), (0, 0, 3), (0, 13, 3), (0, 3, 0), (0, 3, 15),
                                        (2, 9, 3), (2, 0, 3)])
def test_setup_rejects_bad_sizes_without_gpu(domain, K, J):
    lib = lib_or_skip()
    h = ctypes.c_void_p()
    st = lib.st_setup(ctypes.byref(h), domain, K, J, None, None)
    assert st == _lib.ST_ERR_ARG
    assert h.value is None
    assert lib.st_last_error().decode().startswith("st_setup")


@pytest.mark.parametrize("field,value", [("diffusion", (2.0, 0.0, 2.0)), ("precision", 3)])
def test_cube_rejects_unsupported_settings_without_gpu(field, value):
    lib = lib_or_skip()
    cfg = _lib.StConfig()
    lib.st_default_config(ctypes.byref(cfg))
    if field == "diffusion":
        cfg.diffusion[0], cfg.diffusion[1], cfg.diffusion[2] = value
    else:
        cfg.precision = value
    h = ctypes.c_void_p()
    assert lib.st_setup(ctypes.byref(h), 2, 3, 3, ctypes.byref(cfg), None) == _lib.ST_ERR_ARG
    assert h.value is None


def test_null_handle_is_an_argument_error():
    lib = lib_or_skip()
    assert lib.st_apply_S(None, None, None) == _lib.ST_ERR_ARG
    assert lib.st_destroy(None) == _lib.ST_OK
