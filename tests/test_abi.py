"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/rapdb.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rapdb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rapdb_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rapdb_create", "rapdb_solve", "rapdb_kkt_residual", "rapdb_destroy",
                 "rapdb_create_batched", "rapdb_solve_batched", "rapdb_coupling_pass"):
        assert must in names


def test_library_builds_and_exports_every_symbol():
    from paper_2605_29291_gb300 import build as B
    lib_path = B.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_info_and_extras_struct_layouts():
    """rapdb_info: six int32 counters, five doubles, the int64 launch count,
    the switch iteration and its padding; rapdb_extras: the equality block,
    the hyperplane pointer and its constant."""
    from paper_2605_29291_gb300 import rapdb as R
    assert ctypes.sizeof(R.CInfo) == 6 * 4 + 5 * 8 + 8 + 2 * 4
    assert R.CInfo.switch_iter.offset == 6 * 4 + 5 * 8 + 8
    assert ctypes.sizeof(R.CExtras) == 8 + 3 * 8 + 8
    assert R.CExtras.x_hyp_beta.offset == 32


def test_binding_loads_and_mirrors_defaults():
    from paper_2605_29291_gb300 import rapdb as R
    import json
    gp = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_params.json")))
    yx, xy = R.Params.default(R.YX), R.Params.default(R.XY)
    assert (yx.eta, yx.c_alpha, yx.delta) == (gp["eta"]["value"], gp["yx"]["c_alpha"], gp["yx"]["delta"])
    assert (xy.c_alpha, xy.c_beta, xy.delta) == (gp["xy"]["c_alpha"], gp["xy"]["c_beta"], gp["xy"]["delta"])
    assert yx.xi == gp["xi"]["value"] and yx.q == gp["q"]["value"]
    assert yx.gap_first == gp["gap_first"]["yx"] and xy.gap_first == gp["gap_first"]["xy"]
    # struct layout: the ctypes mirror must match the C struct size (the last
    # 8 bytes: restart_warm_tau and pack_sym)
    assert ctypes.sizeof(R.CParams) == 4 * 4 + 7 * 8 + 2 * 4 + 2 * 8 + 2 * 4 + 2 * 4 + 8 + 4 * 4 + 2 * 8 + 2 * 4 + 8 + 8 + 8


def test_create_rejects_bad_sizes_without_touching_the_gpu():
    from paper_2605_29291_gb300 import rapdb as R
    ctx = ctypes.c_void_p()
    p = R.Params.default().to_c()
    st = R.lib.rapdb_create(ctypes.byref(ctx), 0, 3, 0, None, None, None, None, None, None,
                            ctypes.byref(p), None)
    assert st == R.ERR_INVALID and not ctx.value
    assert b"size" in R.lib.rapdb_last_error(None)
    st = R.lib.rapdb_create(ctypes.byref(ctx), 10, 3, 0, None, None, None, None, None, None,
                            ctypes.byref(p), None)
    assert st == R.ERR_INVALID and b"NULL" in R.lib.rapdb_last_error(None)


def test_wait_selftest_rejects_bad_arguments_without_touching_the_gpu():
    from paper_2605_29291_gb300 import rapdb as R
    for complete, limit in ((0, 0), (1, -5), (0, 2000001), (2, 1000)):
        assert R.lib.rapdb_wait_selftest(complete, limit, None, None, None) == R.ERR_INVALID


def test_params_struct_matches_the_library_layout():
    """rapdb_default_params writes exactly sizeof(CParams) bytes and its last
    fields land where the ctypes mirror reads them."""
    from paper_2605_29291_gb300 import rapdb as R
    size = ctypes.sizeof(R.CParams)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    R.lib.rapdb_default_params(ctypes.cast(buf, ctypes.POINTER(R.CParams)), 0)
    assert all(b == 0xAB for b in bytes(buf)[size:])
    p = R.CParams.from_buffer_copy(bytes(buf)[:size])
    assert p.dual_set == R.DUAL_NONNEG and p.dual_radius == 1.0 and p.pass_variant == 0
    assert p.restart_warm_tau == 0 and p.pack_sym == 0


def test_pack_sym_argument_checks_without_touching_the_gpu():
    """pack_sym needs refine = 1 and a single-instance context; both are
    refused before any device call (the data pointers are never read)."""
    from paper_2605_29291_gb300 import rapdb as R
    dummy = (ctypes.c_float * 16)()
    ptr = ctypes.cast(dummy, ctypes.c_void_p)
    ctx = ctypes.c_void_p()
    p = R.Params.default(pack_sym=1, refine=0).to_c()
    st = R.lib.rapdb_create(ctypes.byref(ctx), 4, 1, 0, ptr, None, ptr, ptr, ptr, ptr, ctypes.byref(p), None)
    assert st == R.ERR_INVALID and b"refine" in R.lib.rapdb_last_error(None)
    p = R.Params.default(pack_sym=2).to_c()
    st = R.lib.rapdb_create(ctypes.byref(ctx), 4, 1, 0, ptr, None, ptr, ptr, ptr, ptr, ctypes.byref(p), None)
    assert st == R.ERR_INVALID and b"pack_sym" in R.lib.rapdb_last_error(None)
    p = R.Params.default(pack_sym=1).to_c()
    n = (ctypes.c_int64 * 1)(4)
    m = (ctypes.c_int64 * 1)(1)
    arr = (ctypes.c_void_p * 1)(ptr.value)
    st = R.lib.rapdb_create_batched(ctypes.byref(ctx), 1, n, m, arr, arr, arr, arr, arr, ctypes.byref(p), None)
    assert st == R.ERR_INVALID and b"single-instance" in R.lib.rapdb_last_error(None)
