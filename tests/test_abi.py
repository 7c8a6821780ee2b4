"""The C-ABI library: builds, loads, exports every declared symbol, and
validates arguments on the host (no GPU needed; no compute call is made)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nqs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nqs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_07625_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    import paper_2408_07625_gb300 as nqs
    return nqs.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nqs_ham_load", "nqs_find_coupled_pairs", "nqs_local_energy",
                     "nqs_local_energy_backward", "nqs_stage", "nqs_variational_energy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version(lib):
    assert lib.nqs_version() == 100


def test_host_side_argument_errors(lib):
    h = ctypes.c_void_p()
    x = np.zeros(1, np.uint64); z = np.zeros(1, np.uint64); c = np.ones(1)
    assert lib.nqs_ham_load(0, 1, x.ctypes.data, z.ctypes.data, c.ctypes.data, ctypes.byref(h)) == -1
    assert lib.nqs_ham_load(300, 1, x.ctypes.data, z.ctypes.data, c.ctypes.data, ctypes.byref(h)) == -2
    # a mask bit beyond n_qubits
    xb = np.array([1 << 5], np.uint64)
    assert lib.nqs_ham_load(4, 1, xb.ctypes.data, z.ctypes.data, c.ctypes.data, ctypes.byref(h)) == -1
    assert b"bits" in lib.nqs_last_error()
    # (a string with an odd number of Y is accepted: it makes H complex; loading needs a device)
    assert lib.nqs_ham_load(4, 1, None, None, None, ctypes.byref(h)) == -1
    assert lib.nqs_ham_load(4, 1, x.ctypes.data, z.ctypes.data, c.ctypes.data, None) == -1
    nan = np.array([np.nan])
    assert lib.nqs_ham_load(4, 1, x.ctypes.data, z.ctypes.data, nan.ctypes.data, ctypes.byref(h)) == -1
    assert lib.nqs_stage_bytes(None, 10) < 0
    assert lib.nqs_variational_energy(0, None, None, None, None, None) == -1
    assert lib.nqs_ham_free(None) == 0
    # the sharded search's host-side checks (no device work is reached)
    lib.nqs_route_scratch_bytes.restype = ctypes.c_int64
    assert lib.nqs_route_scratch_bytes(0) < 0 and lib.nqs_route_scratch_bytes(1025) < 0
    assert lib.nqs_route_scratch_bytes(8) > 0
    b = np.array([0, 5, 3], np.int64)  # not ascending
    cnt = np.zeros(2, np.int64)
    i64 = ctypes.c_int64
    p64 = ctypes.POINTER(ctypes.c_int64)
    bp, cp = b.ctypes.data_as(p64), cnt.ctypes.data_as(p64)
    args = (None, None, None, i64(0), None, None, None, i64(0), cp)
    assert lib.nqs_route_records(0, bp, *args, None, i64(0), None) == -1
    assert lib.nqs_route_records(2, None, *args, None, i64(0), None) == -1
    assert lib.nqs_route_records(2, bp, *args, None, i64(0), None) == -1  # no scratch
    raw = np.zeros(4096, np.uint8)
    scr = raw[(-raw.ctypes.data) % 256:][:1024]  # 256-byte aligned (host memory: never reached)
    assert lib.nqs_route_records(2, bp, *args, scr.ctypes.data, i64(1024), None) == -1
    assert b"ascending" in lib.nqs_last_error()
    assert lib.nqs_find_pairs_part(None, None, i64(0), None, 0, 1, None, None, None, i64(0), None, None) == -1
    # the device-count sampler: its limit, and argument errors before any device work
    lib.nqs_gumbel_async_max_parents.restype = ctypes.c_int64
    limit = lib.nqs_gumbel_async_max_parents()
    assert limit == 262144
    one = np.ones(1, np.int64)
    ga = (None, None, None, None, None, i64(4), None, i64(0), None, None, None, one.ctypes.data, None)
    assert lib.nqs_gumbel_topk_level_async(8, 0, i64(limit + 1), one.ctypes.data, *ga) == -2
    assert lib.nqs_gumbel_topk_level_async(8, 0, i64(10), None, *ga) == -1
    assert lib.nqs_gumbel_topk_level_async(8, 9, i64(10), one.ctypes.data, *ga) == -1


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2408_07625_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "import synth" not in src and "from synth" not in src, f
