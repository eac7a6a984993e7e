"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point include/simjoin.h declares, and rejects invalid arguments before
touching the device.  CPU only: no compute call is made."""
import ctypes
import math
import shutil
import subprocess

import numpy as np
import pytest

from paper_2209_11287_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not build.up_to_date():
        pytest.skip("nvcc not available")
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    declared = binding.header_symbols()
    assert "sj_build_index" in declared and "sj_self_join" in declared and "sj_join_batch" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(lib, s)


def test_no_stray_exports(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True, check=True).stdout
    ours = {line.split()[-1] for line in out.splitlines() if " T " in line and line.split()[-1].startswith("sj")}
    assert ours <= set(binding.header_symbols())


def test_error_strings_and_defaults(lib):
    assert binding.sj_error_string(0) == "ok"
    assert "argument" in binding.sj_error_string(binding.SJ_ERR_ARG)
    assert binding.sj_error_string(12345) == "unknown status"
    o = binding.sj_default_options()
    assert o.kernel == binding.SJ_KERNEL_AUTO and o.symmetric == 1 and o.emit_distances == 0
    assert "sm_103a" in binding.sj_version()


@pytest.mark.parametrize("n,d,eps", [(0, 2, 0.1), (-3, 2, 0.1), (10, 0, 0.1), (10, 129, 0.1), (10, 2, 0.0),
                                     (10, 2, -1.0), (10, 2, math.nan), (10, 2, math.inf), (2 ** 31, 2, 0.1)])
def test_invalid_arguments_rejected(lib, n, d, eps):
    x = np.zeros((4, 2))
    h = ctypes.c_void_p()
    st = lib.sj_build_index(x.ctypes.data, n, d, eps, None, None, ctypes.byref(h))
    assert st == binding.SJ_ERR_ARG
    assert h.value is None
    assert binding.sj_last_error_message()


def test_null_arguments_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.sj_build_index(None, 4, 2, 0.1, None, None, ctypes.byref(h)) == binding.SJ_ERR_ARG
    assert lib.sj_build_index(np.zeros(8).ctypes.data, 4, 2, 0.1, None, None, None) == binding.SJ_ERR_ARG
    r = binding.sj_result()
    assert lib.sj_self_join(None, ctypes.byref(r)) == binding.SJ_ERR_ARG
    assert lib.sj_result_copy(None, None, None) == binding.SJ_ERR_ARG
    lib.sj_result_free(None)
    lib.sj_destroy(None)


def test_invalid_options_rejected(lib):
    x = np.zeros((4, 2))
    o = binding.sj_default_options()
    o.kernel = 99
    h = ctypes.c_void_p()
    assert lib.sj_build_index(x.ctypes.data, 4, 2, 0.1, ctypes.byref(o), None, ctypes.byref(h)) == binding.SJ_ERR_ARG


def test_tune_cache_lookup(lib, tmp_path):
    """The tuning cache is host logic: nearest round(log2 n) within 1 for
    single joins, exact padded dimension for batched groups, later lines
    win, a missing file is empty, a malformed line is an error."""
    p = tmp_path / "tune.txt"
    assert binding.sj_tune_lookup(str(p), 0, 4, 1 << 20) is None  # no file
    p.write_text(
        "# comment line\n"
        "single d=4 nlog2=20 kernel=3 qpi=8 m=3 ms=1.5\n"
        "single d=4 nlog2=21 kernel=5 qpi=0 m=0 ms=2.0   # trailing comment\n"
        "\n"
        "batch dp=16 kernel=5 qpi=62 ms=3.0\n"
        "batch dp=16 kernel=4 qpi=0 ms=2.5\n"
    )
    assert binding.sj_tune_lookup(str(p), 0, 4, 1 << 20) == {"kernel": 3, "qpi": 8, "m": 3}
    assert binding.sj_tune_lookup(str(p), 0, 4, 1 << 21) == {"kernel": 5, "qpi": 0, "m": 0}
    assert binding.sj_tune_lookup(str(p), 0, 4, 1 << 19) == {"kernel": 3, "qpi": 8, "m": 3}  # gap 1
    assert binding.sj_tune_lookup(str(p), 0, 4, 1 << 23) is None                             # gap 2
    assert binding.sj_tune_lookup(str(p), 0, 8, 1 << 20) is None                             # other d
    assert binding.sj_tune_lookup(str(p), 1, 16) == {"kernel": 4, "qpi": 0, "m": 0}          # later wins
    assert binding.sj_tune_lookup(str(p), 1, 32) is None
    with open(p, "a") as f:  # a later single entry for the same key overrides
        f.write("single d=4 nlog2=20 kernel=4 qpi=16 m=2 ms=1.0\n")
    assert binding.sj_tune_lookup(str(p), 0, 4, 1 << 20) == {"kernel": 4, "qpi": 16, "m": 2}
    for bad in ("single d=4 kernel=3\n", "batch dp=16 kernel=9\n", "single d=0 nlog2=3 kernel=3\n",
                "tile d=4\n", "batch dp=16 kernel=3 qpi=x\n"):
        q = tmp_path / "bad.txt"
        q.write_text(bad)
        with pytest.raises(binding.SimJoinError) as ei:
            binding.sj_tune_lookup(str(q), 0, 4, 16)
        assert ei.value.status == binding.SJ_ERR_ARG
    assert "malformed line 1" in binding.sj_last_error_message()


def test_options_layout(lib):
    """The binding's options mirror the header: defaults come back from C."""
    o = binding.sj_default_options()
    assert o.kernel == binding.SJ_KERNEL_AUTO and o.symmetric == 1 and o.graph == 0 and o.tune_cache is None
    o = binding.sj_default_options(graph=1, tune_cache="/tmp/x", queries_per_item=8)
    assert o.graph == 1 and o.tune_cache == b"/tmp/x" and o.queries_per_item == 8


def test_new_entry_points_reject_bad_arguments_before_the_device(lib):
    """The autotuner, the round-based join to host memory and the tuning
    cache reject invalid arguments without touching a GPU."""
    x = np.zeros((4, 2))
    best = binding.sj_options()
    ms = ctypes.c_double()
    # sj_autotune: NULL points, n < 1, d out of range, eps invalid, NULL result
    assert lib.sj_autotune(None, 4, 2, 0.1, None, None, 1, None, ctypes.byref(best), ctypes.byref(ms)) == binding.SJ_ERR_ARG
    assert lib.sj_autotune(x.ctypes.data, 0, 2, 0.1, None, None, 1, None, ctypes.byref(best), None) == binding.SJ_ERR_ARG
    assert lib.sj_autotune(x.ctypes.data, 4, 0, 0.1, None, None, 1, None, ctypes.byref(best), None) == binding.SJ_ERR_ARG
    assert lib.sj_autotune(x.ctypes.data, 4, 2, math.nan, None, None, 1, None, ctypes.byref(best), None) == binding.SJ_ERR_ARG
    assert lib.sj_autotune(x.ctypes.data, 4, 2, 0.1, None, None, 1, None, None, None) == binding.SJ_ERR_ARG
    # sj_autotune_batch: no instances, a dimension out of range
    ptrs = (ctypes.c_void_p * 1)(x.ctypes.data)
    ns = (ctypes.c_int64 * 1)(4)
    es = (ctypes.c_double * 1)(0.1)
    ng = ctypes.c_int32()
    for count, d in ((0, 2), (1, 0), (1, 129)):
        ds = (ctypes.c_int32 * 1)(d)
        assert lib.sj_autotune_batch(ptrs, ns, ds, es, count, None, None, 1, None, 0, ctypes.byref(ng), None, None,
                                     None, None) == binding.SJ_ERR_ARG
    # sj_self_join_to_host: NULL handle, NULL count, a buffer below 1024 pairs
    cnt = ctypes.c_int64()
    out = np.zeros((8, 2), dtype=np.int32)
    assert lib.sj_self_join_to_host(None, out.ctypes.data, 8, 4096, ctypes.byref(cnt), None) == binding.SJ_ERR_ARG
    assert lib.sj_self_join_to_host(None, out.ctypes.data, 8, 4096, None, None) == binding.SJ_ERR_ARG
    assert lib.sj_self_join_to_host(None, out.ctypes.data, 8, 100, ctypes.byref(cnt), None) == binding.SJ_ERR_ARG
    # sj_tune_lookup: NULL path
    assert lib.sj_tune_lookup(None, 0, 2, 4, None, None, None) == binding.SJ_ERR_ARG
    # indexed_dims below SJ_NO_INDEX is an invalid option
    o = binding.sj_default_options(indexed_dims=-2)
    h = ctypes.c_void_p()
    assert lib.sj_build_index(x.ctypes.data, 4, 2, 0.1, ctypes.byref(o), None, ctypes.byref(h)) == binding.SJ_ERR_ARG
