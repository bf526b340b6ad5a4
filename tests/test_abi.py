"""C-ABI checks that need no GPU: the library builds, loads, exports every entry
point declared in include/gbr.h, sizes workspaces and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

import __graft_entry__
from paper_2303_10785_b300 import gbr
from paper_2303_10785_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return gbr.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gbr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbr_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(gbr.exported_symbols())


def test_workspace_bytes(lib):
    p = gbr.make_params(I.case_params(3, (32, 24, 16), reynolds=100.0))
    nb = lib.gbr_workspace_bytes(ctypes.byref(p))
    assert nb > 0 and nb % 256 == 0
    # more cells, more bytes; viscous and moving need more than inviscid static
    p2 = gbr.make_params(I.case_params(3, (64, 24, 16), reynolds=100.0))
    assert lib.gbr_workspace_bytes(ctypes.byref(p2)) > nb
    p3 = gbr.make_params(I.case_params(3, (32, 24, 16)))
    assert lib.gbr_workspace_bytes(ctypes.byref(p3)) < nb
    p4 = gbr.make_params(I.case_params(3, (32, 24, 16), reynolds=100.0, moving=1))
    assert lib.gbr_workspace_bytes(ctypes.byref(p4)) > nb
    # the mixed path stores primitives, gradients and fluxes in FP32
    p5 = gbr.make_params(I.case_params(3, (32, 24, 16), reynolds=100.0, precision="mixed"))
    assert p5.precision == gbr.GBR_PREC_MIXED
    assert 0 < lib.gbr_workspace_bytes(ctypes.byref(p5)) < nb


@pytest.mark.parametrize("bad", [dict(ndim=4), dict(n=(4, 8, 8)), dict(gamma=1.0), dict(ghost=True),
                                 dict(precision=7)])
def test_invalid_params_rejected(lib, bad):
    kw = dict(reynolds=0.0)
    nd = bad.get("ndim", 3)
    n = bad.get("n", (8, 8, 8))
    case = I.case_params(3, n, **kw)
    case["ndim"] = nd
    if "gamma" in bad:
        case["gamma"] = bad["gamma"]
    if "ghost" in bad:
        case["periodic"] = (0, 1, 1)
        case["ghost_nodes"] = 4
    p = gbr.make_params(case)
    if "precision" in bad:
        p.precision = bad["precision"]
    assert lib.gbr_workspace_bytes(ctypes.byref(p)) == 0
    out = ctypes.c_void_p()
    dummy = (ctypes.c_double * 8)()
    rc = lib.gbr_create(ctypes.byref(p), dummy, None, ctypes.c_void_p(256), ctypes.c_size_t(1 << 40), None,
                        ctypes.byref(out))
    assert rc == gbr.GBR_EINVAL
    assert lib.gbr_last_global_error()


def test_grid_beyond_32bit_offsets_rejected(lib):
    # the interface kernels address their arrays with 32-bit offsets: a grid whose (fields + 1) x
    # padded cells reach 2^32 is rejected on the host (it would need ~1 TB of workspace anyway)
    ok = gbr.make_params(I.case_params(3, (512, 512, 512)))
    assert lib.gbr_workspace_bytes(ctypes.byref(ok)) > 0
    big = gbr.make_params(I.case_params(3, (1024, 1024, 1024)))
    assert lib.gbr_workspace_bytes(ctypes.byref(big)) == 0
    assert b"32-bit" in lib.gbr_last_global_error()


def test_small_workspace_is_enomem_before_any_device_work(lib):
    p = gbr.make_params(I.case_params(3, (16, 16, 16)))
    need = lib.gbr_workspace_bytes(ctypes.byref(p))
    out = ctypes.c_void_p()
    dummy = (ctypes.c_double * 8)()
    rc = lib.gbr_create(ctypes.byref(p), dummy, None, ctypes.c_void_p(256), ctypes.c_size_t(need - 256), None,
                        ctypes.byref(out))
    assert rc == gbr.GBR_ENOMEM
    rc = lib.gbr_create(ctypes.byref(p), dummy, None, ctypes.c_void_p(260), ctypes.c_size_t(need), None,
                        ctypes.byref(out))
    assert rc == gbr.GBR_EINVAL  # misaligned workspace


def test_null_context_calls_fail_cleanly(lib):
    assert lib.gbr_compute_metrics(None) == gbr.GBR_EINVAL
    assert lib.gbr_rk_step(None, ctypes.c_double(0.4)) == gbr.GBR_EINVAL
    assert lib.gbr_sync(None, ctypes.c_double(1.0)) == gbr.GBR_EINVAL
    assert lib.gbr_check_bounded_wait(None, 64) == gbr.GBR_EINVAL
    assert lib.gbr_batch_check_barrier(None, 64) == gbr.GBR_EINVAL
    assert lib.gbr_set_state_async(None, None, None) == gbr.GBR_EINVAL
    assert lib.gbr_get_state_async(None, None, None) == gbr.GBR_EINVAL
    lib.gbr_destroy(None)


@pytest.mark.parametrize("bad", ["long_axis", "many_ghosts", "negative_ghosts"])
def test_axis_and_ghost_bounds_rejected_before_size_arithmetic(lib, bad):
    # an axis of 2^30 cells (with the others 1 wide the cell count alone would pass) or an absurd
    # number of ghost node layers would overflow the padded extents; both are refused up front,
    # by gbr_workspace_bytes, gbr_create and the allocation-free gbr_rhs_static alike
    if bad == "long_axis":
        case = I.case_params(2, (1 << 30, 6))
    else:
        case = I.case_params(2, (16, 16), periodic=(0, 1), ghost_nodes=5000 if bad == "many_ghosts" else -3)
    p = gbr.make_params(case)
    assert lib.gbr_workspace_bytes(ctypes.byref(p)) == 0
    why = b"axis too long" if bad == "long_axis" else b"ghost_nodes out of range"
    assert why in lib.gbr_last_global_error()
    dummy = (ctypes.c_double * 8)()
    msg = ctypes.create_string_buffer(128)
    rc = lib.gbr_rhs_static(ctypes.byref(p), dummy, None, ctypes.c_void_p(256), ctypes.c_void_p(256), None, msg,
                            ctypes.c_size_t(128))
    assert rc == gbr.GBR_EINVAL
    assert why in msg.value
