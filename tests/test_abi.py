"""The C-ABI library builds, loads and exports every symbol include/rid.h
declares; host-side argument checks reject bad calls before any CUDA work
(these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1205_3830_gb300 import _native, build
    build.build()
    return _native.load()


def declared_symbols():
    with open(os.path.join(ROOT, "include", "rid.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"RID_API\s+[\w\s\*]*?\b(rid_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("rid_plan_create", "rid_plan_destroy", "rid_sketch", "rid_select", "rid_solve",
                     "rid_error", "rid_sync_status", "rid_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1205_3830_gb300 import _native
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(rid_\w+)$", out, flags=re.M))
    for name in declared_symbols():
        assert name in exported, name
        assert hasattr(lib, name)
    # nothing beyond the declared ABI leaks out of the library
    assert exported == set(declared_symbols())
    assert set(_native.SIGNATURES) == set(declared_symbols())


def test_status_strings(lib):
    from paper_1205_3830_gb300 import _native
    for code in range(7):
        s = _native.status_string(code)
        assert s.startswith("RID_")
    assert "unknown" in _native.status_string(99)


@pytest.mark.parametrize("args", [
    (0, 10, 1, 2), (10, 0, 1, 2), (10, 10, 0, 2), (10, 10, 3, 2),   # m, n, k, l out of range
    (10, 4, 5, 6), (4, 10, 5, 6),                                    # k > n, k > m
])
def test_plan_create_rejects_bad_sizes(lib, args):
    from paper_1205_3830_gb300 import _native
    h = ctypes.c_void_p()
    m, n, k, l = args
    st = lib.rid_plan_create(ctypes.byref(h), m, n, k, l, 0, 0, 1, None)
    assert st == _native.RID_EINVAL and not h.value


def test_plan_create_rejects_unsupported_combinations(lib):
    from paper_1205_3830_gb300 import _native
    h = ctypes.c_void_p()
    assert lib.rid_plan_create(ctypes.byref(h), 100, 100, 5, 600, 0, 0, 1, None) == _native.RID_EUNSUPPORTED
    assert lib.rid_plan_create(ctypes.byref(h), 100, 100, 5, 8, 0, _native.RID_MIXED_BF16, 1, None) == \
        _native.RID_EUNSUPPORTED
    assert lib.rid_plan_create(ctypes.byref(h), 100, 100, 5, 8, 1, _native.RID_FP64_NATIVE, 1, None) == \
        _native.RID_EUNSUPPORTED
    assert lib.rid_plan_create(ctypes.byref(h), 100, 100, 5, 8, 7, 0, 1, None) == _native.RID_EINVAL
    assert lib.rid_plan_create(None, 100, 100, 5, 8, 0, 0, 1, None) == _native.RID_EINVAL


def test_calls_reject_null_plan(lib):
    from paper_1205_3830_gb300 import _native
    E = _native.RID_EINVAL
    out = (ctypes.c_double * 2)()
    assert lib.rid_sketch(None, None, 1, None, 1) == E
    assert lib.rid_select(None, None, 1, None) == E
    assert lib.rid_solve(None, None, 1, None, 1) == E
    assert lib.rid_error(None, None, 1, None, None, 1, 8, 1, out) == E
    assert lib.rid_sync_status(None) == E
    assert lib.rid_plan_set_omega(None, None, 1) == E
    assert lib.rid_plan_set_select_grid(None, 0) == E
    ptr, ld = ctypes.c_void_p(), ctypes.c_int64()
    assert lib.rid_plan_probe_products(None, ctypes.byref(ptr), ctypes.byref(ld)) == E
    assert lib.rid_plan_destroy(None) == _native.RID_OK


def test_plain_c99_consumer_compiles_links_and_runs(lib):
    """include/rid.h is a C header: a C99 program compiles against it with
    -pedantic -Werror, links librid.so and gets the documented statuses from
    the calls that need no GPU (tests/c/abi_consumer.c)."""
    import shutil
    from paper_1205_3830_gb300 import _native
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(_native.LIB_PATH)
    exe = os.path.join(libdir, "abi_consumer")
    subprocess.run([gcc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_consumer.c"), "-L", libdir, "-lrid",
                    "-Wl,-rpath," + libdir, "-o", exe], check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "ok"


def test_batch_tc_calls_reject_bad_arguments_before_cuda_work(lib):
    """The tensor-core batch checks its items and tile choices on the host
    (fake, aligned device pointers: nothing is dereferenced before the checks)."""
    from paper_1205_3830_gb300 import _native
    E = _native.RID_EINVAL
    h = ctypes.c_void_p()
    out = (ctypes.c_double * 4)()
    assert lib.rid_batch_tc_info(None, out) == E
    assert lib.rid_batch_tc_run(None, None) == E
    assert lib.rid_batch_tc_times(None, out) == E
    items = (_native.BatchItem * 1)()
    it = items[0]
    it.m, it.n, it.k, it.l = 100, 80, 4, 12
    it.A, it.lda, it.Y, it.ldy, it.perm, it.T, it.ldt, it.seed = 256, 100, 512, 12, 768, 1024, 4, 1
    err, status = ctypes.c_void_p(2048), ctypes.c_void_p(4096)
    call = lambda tn, ks, cnt=1, npr=8: lib.rid_batch_tc_create_tuned(
        ctypes.byref(h), ctypes.byref(items), cnt, npr, 1, err, status,
        ctypes.cast(tn, ctypes.c_void_p) if tn is not None else None,
        ctypes.cast(ks, ctypes.c_void_p) if ks is not None else None, 0, None)
    for bad in (8, 129, 100):
        assert call((ctypes.c_int32 * 1)(bad), None) == E and not h.value
    assert call(None, (ctypes.c_int32 * 1)(-1)) == E
    assert call(None, None, cnt=0) == E
    assert call(None, None, npr=0) == E and call(None, None, npr=17) == E
    it.k = 70                                                   # k > 64: beyond the batch's limit
    it.l = 72
    it.ldy = 72
    it.ldt = 70
    assert lib.rid_batch_tc_create_tuned(ctypes.byref(h), ctypes.byref(items), 1, 8, 1, err, status, None, None, 0,
                                         None) == _native.RID_EUNSUPPORTED
