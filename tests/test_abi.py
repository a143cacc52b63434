"""The C ABI library loads and exports what include/lbm.h declares (no GPU needed)."""

import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lbm():
    from paper_1805_08643_gb300 import _build

    _build.build()
    from paper_1805_08643_gb300 import lbm as mod

    return mod


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for name in ("lbm_create", "lbm_init_droplet", "lbm_init_flat", "lbm_step", "lbm_moments",
                 "lbm_destroy", "lbm_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(lbm):
    lib = ctypes.CDLL(lbm.LIB_PATH)
    for name in _declared_symbols():
        assert hasattr(lib, name), name
    assert set(_declared_symbols()) == set(lbm.SIGNATURES)


def _create(lbm, grid=(8, 8, 8), op=1, prec=0, eos_kind=0, G=-1.0, sigma=0.0, rates=None):
    eos = lbm.LbmEos(eos_kind, 1.0, 4.0, 1.0, 0.07, 1.0, 1.0)
    r = lbm.LbmRates(*(rates or (1.1, 1.0, 1.1, 1.1, 1.1, 1.1)))
    g = (ctypes.c_int * 3)(*grid)
    h = ctypes.c_void_p()
    st = lbm.lib.lbm_create(ctypes.byref(g), ctypes.byref(eos), G, ctypes.byref(r), op, prec, sigma,
                            None, ctypes.byref(h))
    return st, h


def test_create_validates_arguments_without_touching_the_gpu(lbm):
    assert _create(lbm, grid=(2, 8, 8))[0] == lbm.ERR_ARG
    assert _create(lbm, op=5)[0] == lbm.ERR_ARG
    assert _create(lbm, prec=3)[0] == lbm.ERR_ARG
    assert _create(lbm, eos_kind=7)[0] == lbm.ERR_ARG
    assert _create(lbm, rates=(2.5, 1, 1, 1, 1, 1))[0] == lbm.ERR_ARG
    assert _create(lbm, G=0.0)[0] == lbm.ERR_ARG  # sqrt pseudopotential needs G != 0
    assert _create(lbm, eos_kind=2, sigma=0.1)[0] == lbm.ERR_ARG
    st, h = _create(lbm)
    assert st == lbm.OK and h.value
    # state errors are caught on the host before any launch
    assert lbm.lib.lbm_step(h, 1) == lbm.ERR_STATE
    assert b"before an init" in lbm.lib.lbm_last_error(h)
    assert lbm.lib.lbm_step(h, 0) == lbm.ERR_ARG
    assert lbm.lib.lbm_step_count(h) == 0
    pb, sb, xb = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    assert lbm.lib.lbm_buffer_bytes(h, ctypes.byref(pb), ctypes.byref(sb), ctypes.byref(xb)) == lbm.OK
    assert pb.value == 19 * 512 * 8 and sb.value == 2 * 512 * 8  # two psi time levels
    lbm.lib.lbm_destroy(h)
    st, h = _create(lbm, prec=2)
    lbm.lib.lbm_buffer_bytes(h, ctypes.byref(pb), ctypes.byref(sb), ctypes.byref(xb))
    assert pb.value == 19 * 512 * 2 and sb.value == 2 * 512 * 4
    lbm.lib.lbm_destroy(h)
    assert lbm.lib.lbm_status_string(4) == b"LBM_ERR_NONFINITE"


def test_set_tuning_validates_modes_without_touching_the_gpu(lbm):
    st, h = _create(lbm)  # FP64
    assert st == lbm.OK
    for mode in (1, 2, 3, 4):  # every single pass needs FP32 arithmetic
        assert lbm.lib.lbm_set_tuning(h, mode, 1, 0) == lbm.ERR_ARG
    assert lbm.lib.lbm_set_tuning(h, 5, 1, 0) == lbm.ERR_ARG
    assert lbm.lib.lbm_set_tuning(h, 0, 3, 0) == lbm.ERR_ARG
    assert lbm.lib.lbm_set_tuning(h, 0, 1, -1) == lbm.ERR_ARG
    lbm.lib.lbm_destroy(h)
    st, h = _create(lbm, grid=(9, 8, 8), prec=1)  # FP32, odd Nx: no two-node kernels
    assert st == lbm.OK
    assert lbm.lib.lbm_set_tuning(h, 3, 1, 0) == lbm.ERR_ARG
    assert lbm.lib.lbm_set_tuning(h, 4, 1, 0) == lbm.ERR_ARG
    assert b"even Nx" in lbm.lib.lbm_last_error(h)
    assert lbm.lib.lbm_set_tuning(h, 1, 2, 16) == lbm.OK  # the one-node single pass takes any Nx
    sp, t, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lbm.lib.lbm_get_tuning(h, ctypes.byref(sp), ctypes.byref(t), ctypes.byref(z)) == lbm.OK
    assert (sp.value, t.value, z.value) == (1, 2, 16)
    lbm.lib.lbm_destroy(h)


def test_d3q15_contexts_size_their_buffers_and_reject_d3q19_only_paths(lbm):
    st, h = _create(lbm, op=2)  # LBM_OP_NONORTHOGONAL_D3Q15, FP64
    assert st == lbm.OK
    pb, sb, xb = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    assert lbm.lib.lbm_buffer_bytes(h, ctypes.byref(pb), ctypes.byref(sb), ctypes.byref(xb)) == lbm.OK
    assert pb.value == 15 * 512 * 8 and sb.value == 2 * 512 * 8
    # null buffers are rejected before anything else (the D3Q15 rejection itself is a GPU test
    # with real buffers: no invented device address is ever passed to an entry point that launches)
    assert lbm.lib.lbm_step_static(h, None, None) == lbm.ERR_ARG
    lbm.lib.lbm_destroy(h)
    st, h = _create(lbm, op=2, prec=1)
    assert st == lbm.OK
    for mode in (1, 2, 3, 4):
        assert lbm.lib.lbm_set_tuning(h, mode, 1, 0) == lbm.ERR_ARG
    assert b"D3Q19" in lbm.lib.lbm_last_error(h)
    assert lbm.lib.lbm_set_tuning(h, 0, 1, 0) == lbm.OK
    lbm.lib.lbm_destroy(h)
    st, h = _create(lbm, op=2, prec=2)
    lbm.lib.lbm_buffer_bytes(h, ctypes.byref(pb), ctypes.byref(sb), ctypes.byref(xb))
    assert pb.value == 4 * 512 * 8  # 15 halves per node are less than the 4 doubles lbm_moments stages
    lbm.lib.lbm_destroy(h)
    assert _create(lbm, op=3)[0] == lbm.ERR_ARG


def test_create_rejects_boxes_beyond_the_index_limits(lbm):
    # 32-bit node index and 32-bit element offsets (19 N < 2^32), the grid-z launch limit
    assert _create(lbm, grid=(1024, 1024, 256))[0] == lbm.ERR_ARG  # 19 * 2^28 >= 2^32
    assert _create(lbm, grid=(2048, 2048, 512))[0] == lbm.ERR_ARG  # N = 2^31
    assert _create(lbm, grid=(3, 3, 65536))[0] == lbm.ERR_ARG
    st, h = _create(lbm, grid=(1024, 1024, 200))  # 19 N just under 2^32: accepted (no allocation yet)
    assert st == lbm.OK
    lbm.lib.lbm_destroy(h)
    st, h = _create(lbm, grid=(3, 3, 65535))
    assert st == lbm.OK
    lbm.lib.lbm_destroy(h)
