"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/*.h declares, rejects bad arguments before touching a
device, and its host-side pieces agree with the oracle's definitions."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2104_12922_gb300 import build as b
    b.build()
    import paper_2104_12922_gb300 as p
    return p


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(synth_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_boundary():
    names = _declared_functions()
    for required in ("synth_create", "synth_destroy", "synth_render", "synth_render_plain",
                     "synth_sync", "synth_is_test", "synth_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(pkg):
    lib = ctypes.CDLL(pkg.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(pkg):
    for s in range(7):
        assert pkg.synth_status_string(s)
    assert pkg.synth_status_string(99) == "unknown status"


def test_create_rejects_bad_config_without_device(pkg):
    L = pkg.lib()
    cfg = pkg.synth_default_config()
    h = ctypes.c_void_p()
    assert L.synth_create(None, ctypes.byref(h)) == pkg.SYNTH_ERR_ARG
    for field, bad in [("seconds", 0.0), ("sample_rate", -1.0), ("max_batch", 0)]:
        c = pkg.synth_default_config()
        setattr(c, field, bad)
        assert L.synth_create(ctypes.byref(c), ctypes.byref(h)) == pkg.SYNTH_ERR_ARG
    c = pkg.synth_default_config()
    c.control_rate = 441.3  # fractional R from a control rate that is not an integer in Hz
    assert L.synth_create(ctypes.byref(c), ctypes.byref(h)) == pkg.SYNTH_ERR_UNSUPPORTED
    c = pkg.synth_default_config()
    c.control_rate = 44100.0 / 3  # R = 3 < 4
    assert L.synth_create(ctypes.byref(c), ctypes.byref(h)) == pkg.SYNTH_ERR_UNSUPPORTED
    c = pkg.synth_default_config()
    c.sample_rate, c.carry = 16000.0, pkg.SYNTH_CARRY_FP32  # FP32 carries need integer R % 4 == 0
    assert L.synth_create(ctypes.byref(c), ctypes.byref(h)) == pkg.SYNTH_ERR_UNSUPPORTED
    c = pkg.synth_default_config()
    c.control_rate = 44100.0 / 65536  # R = 2^16: above the 16-bit in-interval index
    assert L.synth_create(ctypes.byref(c), ctypes.byref(h)) == pkg.SYNTH_ERR_UNSUPPORTED
    c = pkg.synth_default_config()
    c.carry = 7
    assert L.synth_create(ctypes.byref(c), ctypes.byref(h)) == pkg.SYNTH_ERR_ARG


def test_calls_on_null_handle_return_status(pkg):
    L = pkg.lib()
    assert L.synth_render(None, 0, 0, 1, None, None, None, None) == pkg.SYNTH_ERR_STATE
    assert L.synth_sync(None, None) == pkg.SYNTH_ERR_STATE
    assert L.synth_selftest_wait_timeout(None, None) == pkg.SYNTH_ERR_STATE
    assert L.synth_destroy(None) == pkg.SYNTH_ERR_ARG


def test_split_rule(pkg):
    """Sec. 2.2: 9 blocks of 1024 train, then 1024 test, repeating."""
    for g in [0, 1023, 9 * 1024 - 1, 10 * 1024 - 1, 19 * 1024 + 5]:
        assert pkg.synth_is_test(g) == (g >= 9 * 1024 and g < 10 * 1024 or 19 * 1024 <= g < 20 * 1024)
    flags = np.array([pkg.synth_is_test(g) for g in range(0, 20 * 1024, 256)])
    assert flags.mean() == pytest.approx(0.1)


def test_split_voice_enumerates_each_split_in_order(pkg):
    """synth_split_voice(split, i) is the i-th voice of the split, checked
    by brute-force enumeration of g with synth_is_test over three periods
    and at indices past 2^40 (closed form against a local enumeration)."""
    train = [g for g in range(3 * 10240) if not pkg.synth_is_test(g)]
    test = [g for g in range(3 * 10240) if pkg.synth_is_test(g)]
    assert [pkg.synth_split_voice(pkg.SPLIT_TRAIN, i) for i in range(len(train))] == train
    assert [pkg.synth_split_voice(pkg.SPLIT_TEST, i) for i in range(len(test))] == test
    assert [pkg.synth_split_voice(pkg.SPLIT_ALL, i) for i in (0, 5, 10**12)] == [0, 5, 10**12]
    base = (1 << 40) // 10240 * 10240  # a period boundary
    big_train = [g for g in range(base, base + 10240) if not pkg.synth_is_test(g)]
    i0 = base // 10240 * 9216
    assert [pkg.synth_split_voice(pkg.SPLIT_TRAIN, i0 + i) for i in range(9216)] == big_train
    i1 = base // 10240 * 1024
    assert pkg.synth_split_voice(pkg.SPLIT_TEST, i1) == base + 9216


def test_stream_features_argument_errors_without_device(pkg):
    lib = pkg.lib()
    # a NULL model is rejected before any argument is looked at
    assert lib.synth_stream_features(None, 0, 1, 0, 4, 0, None, None, None) == pkg.SYNTH_ERR_STATE


def test_default_nebula_matches_oracle(pkg, oracle_mod):
    """The library's n0 table and the oracle's are written independently."""
    lib_nb = pkg.nebula_dict(pkg.synth_default_nebula())
    ora_nb = oracle_mod.default_nebula()
    for k in ("lo", "hi", "curve", "symmetric"):
        assert np.array_equal(lib_nb[k], ora_nb[k]), k


def test_checked_build_exports_the_same_calls(pkg):
    """The bounds-checked library (build(checks=True): the same sources with
    -DSYNTH_CHECKS) builds, exports every declared call, says it is the
    checked build, and validates its arguments like the release build."""
    from paper_2104_12922_gb300 import build as b
    path = b.build(checks=True)
    C = ctypes.CDLL(path)
    for name in _declared_functions():
        assert hasattr(C, name), name
    C.synth_checked_build.restype = ctypes.c_int32
    C.synth_selftest_bounds.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert C.synth_checked_build() == 1
    assert pkg.lib().synth_checked_build() == 0
    assert C.synth_selftest_bounds(None, None) == pkg.SYNTH_ERR_STATE
    assert pkg.lib().synth_selftest_bounds(None, None) == pkg.SYNTH_ERR_STATE
