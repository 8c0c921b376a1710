"""The C-ABI library loads and exports every entry point include/ffcz.h declares
(no GPU needed: nothing here launches device work)."""
import ctypes
import os
import re

import paper_2601_01596_b300 as ffcz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "ffcz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ffcz_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared() == sorted(ffcz.SYMBOLS)


def test_library_exports_every_symbol():
    L = ffcz.lib()
    for name in declared():
        assert hasattr(L, name), name


def test_host_only_calls():
    o = ffcz.default_opts()
    assert o.max_iters == 10000 and o.min_iters == 0 and o.precision == 32
    assert o.shrink == 2.0 ** -16 and o.K == 50 and o.ckpt_every == 10
    L = ffcz.lib()
    for s in range(9):
        assert L.ffcz_strerror(s)
    assert L.ffcz_launch_count() >= 0
    # struct layouts match the header (checked on the host compiler's ABI)
    assert ctypes.sizeof(ffcz.Opts) == 64 and ctypes.sizeof(ffcz.Stats) == 80   # 14 int32 + 1 double


def test_invalid_arguments_fail_before_any_device_work():
    L = ffcz.lib()
    h = ctypes.c_void_p()
    sh = (ctypes.c_int64 * 3)(32, 32, 32)
    assert L.ffcz_plan(None, 3, sh, 1, None, None) == ffcz.ERR_INVALID
    assert L.ffcz_plan(ctypes.byref(h), 4, sh, 1, None, None) == ffcz.ERR_INVALID
    assert L.ffcz_plan(ctypes.byref(h), 3, sh, 0, None, None) == ffcz.ERR_INVALID
    bad = (ctypes.c_int64 * 3)(32, 24, 32)
    assert L.ffcz_plan(ctypes.byref(h), 3, bad, 1, None, None) == ffcz.ERR_UNSUPPORTED
    assert b"power" in L.ffcz_last_error()
    assert L.ffcz_correct(None, None, None, None, None) == ffcz.ERR_INVALID
    assert L.ffcz_ckpt_floats(None) == 0
    assert L.ffcz_correct_ckpt(None, None, None, None, None, None) == ffcz.ERR_INVALID
    assert L.ffcz_correct_backward_ckpt(None, None, None, None, None, None, None) == ffcz.ERR_INVALID
    L.ffcz_destroy(None)


def test_projection_variant_options_are_checked_on_the_host():
    L = ffcz.lib()
    h = ctypes.c_void_p()
    sh3 = (ctypes.c_int64 * 3)(32, 32, 32)
    sh1 = (ctypes.c_int64 * 1)(4096)
    assert ffcz.default_opts().method == 0
    assert ffcz.default_opts(method="dykstra").method == 1
    assert ffcz.default_opts(method="dr").method == 2 and ffcz.default_opts(method="admm").method == 3
    o = ffcz.default_opts(method=4)
    assert L.ffcz_plan(ctypes.byref(h), 3, sh3, 1, ctypes.byref(o), None) == ffcz.ERR_INVALID
    for kw in ({"method": 1, "edits": 1}, {"method": 2, "pointwise": 1}, {"method": 3, "precision": 64}):
        o = ffcz.default_opts(**kw)
        assert L.ffcz_plan(ctypes.byref(h), 3, sh3, 1, ctypes.byref(o), None) == ffcz.ERR_UNSUPPORTED, kw
    o = ffcz.default_opts(method=1, edits=1)   # 1D items: the same rules
    assert L.ffcz_plan(ctypes.byref(h), 1, sh1, 1, ctypes.byref(o), None) == ffcz.ERR_UNSUPPORTED
