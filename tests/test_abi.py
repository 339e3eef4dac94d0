"""The C-ABI library on a machine without a GPU: it loads, exports every entry point
include/msi.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def msi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_00786_gb300 as m
    return m


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "msi.h")).read()
    return sorted(set(re.findall(r"MSI_API\s+[\w\s\*]+?\b(msi_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for want in ("msi_build", "msi_knn", "msi_free", "msi_status_str", "msi_last_error", "msi_index_info_get"):
        assert want in names


def test_library_exports_every_declared_symbol(msi):
    lib = ctypes.CDLL(msi.library_path())
    for name in declared_entry_points():
        assert hasattr(lib, name), f"{name} is declared in include/msi.h but not exported"


def test_status_strings_and_version(msi):
    assert msi.msi_abi_version() == 3
    names = [msi.msi_status_str(s) for s in range(6)]
    assert names == ["MSI_OK", "MSI_EINVAL", "MSI_ENOMEM", "MSI_ECUDA", "MSI_ETIMEOUT", "MSI_EINTERNAL"]
    assert msi.msi_status_str(99) == "MSI_UNKNOWN"


def _raw_build(msi, series, n, length, segs, card, cap=0, flags=0):
    lib = msi._lib
    opts = msi._BuildOpts(cap, flags, None, 0, 0)
    out = ctypes.c_void_p(123)
    p = ctypes.c_void_p(series.ctypes.data) if series is not None else None
    st = lib.msi_build(p, n, length, segs, card, ctypes.byref(opts), ctypes.byref(out))
    return st, out.value


@pytest.mark.parametrize("n,length,segs,card,cap,flags,needle", [
    (0, 256, 16, 256, 0, 0, "n = 0"),
    (-5, 256, 16, 256, 0, 0, "n = -5"),
    (10, 0, 16, 256, 0, 0, "len = 0"),
    (10, 5000, 16, 256, 0, 0, "len = 5000"),
    (10, 250, 16, 256, 0, 0, "multiple"),
    (10, 256, 0, 256, 0, 0, "segments = 0"),
    (10, 256, 17, 256, 0, 0, "segments = 17"),
    (10, 256, 16, 100, 0, 0, "power of two"),
    (10, 256, 16, 512, 0, 0, "power of two"),
    (10, 256, 16, 1, 0, 0, "power of two"),
    (10, 256, 16, 256, -1, 0, "leaf_capacity"),
    (10, 256, 16, 256, 0, 0x10, "flags"),
])
def test_build_rejects_bad_arguments_without_a_device(msi, n, length, segs, card, cap, flags, needle):
    x = np.zeros((4, 256), np.float32)
    st, out = _raw_build(msi, x, n, length, segs, card, cap, flags)
    assert st == msi.MSI_EINVAL
    assert out is None  # *out is cleared on failure
    assert needle in msi.msi_last_error()


def test_build_null_series(msi):
    st, _ = _raw_build(msi, None, 10, 256, 16, 256)
    assert st == msi.MSI_EINVAL and "NULL" in msi.msi_last_error()


def test_knn_and_helpers_reject_null_index(msi):
    lib = msi._lib
    ids = np.zeros(4, np.int64)
    q = np.zeros(256, np.float32)
    assert lib.msi_knn(None, ctypes.c_void_p(q.ctypes.data), 1, 1, ctypes.c_void_p(ids.ctypes.data), None, None) == msi.MSI_EINVAL
    assert "NULL" in msi.msi_last_error()
    qp, ip = ctypes.c_void_p(q.ctypes.data), ctypes.c_void_p(ids.ctypes.data)
    assert lib.msi_knn_dtw(None, qp, 1, 1, 25, ip, None, None, None) == msi.MSI_EINVAL
    assert "NULL" in msi.msi_last_error()
    assert lib.msi_knn_dtw(None, qp, 1, 1, -1, ip, None, None, None) == msi.MSI_EINVAL
    assert "negative" in msi.msi_last_error()
    info = msi._IndexInfo()
    assert lib.msi_index_info_get(None, ctypes.byref(info)) == msi.MSI_EINVAL
    assert lib.msi_set_timing(None, 1) == msi.MSI_EINVAL
    st = msi._QueryStats()
    assert lib.msi_query_stats_get(None, ctypes.byref(st), 0) == msi.MSI_EINVAL
    tr = msi._TuneResult()
    assert lib.msi_autotune(None, qp, 4, 1, 0, ctypes.byref(tr), None) == msi.MSI_EINVAL
    assert "NULL" in msi.msi_last_error()
    lib.msi_free(None)  # no-op


def test_python_binding_raises_msierror(msi):
    with pytest.raises(msi.MsiError) as e:
        msi.msi_build(np.zeros((3, 250), np.float32), segments=16)
    assert e.value.status == msi.MSI_EINVAL


def test_product_package_does_not_load_the_oracle():
    pkg = os.path.join(ROOT, "paper_2009_00786_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, re.M), f
                assert "liboracle" not in text and "oracle.c" not in text, f


def test_index_load_rejects_bad_files_before_the_device(msi, tmp_path):
    import struct
    lib = msi._lib
    out = ctypes.c_void_p(7)
    missing = str(tmp_path / "missing.idx").encode()
    assert lib.msi_index_load(missing, None, None, ctypes.byref(out)) == msi.MSI_EINVAL and out.value is None
    garbage = tmp_path / "garbage.idx"
    garbage.write_bytes(b"not an index at all" * 10)
    assert lib.msi_index_load(str(garbage).encode(), None, None, ctypes.byref(out)) == msi.MSI_EINVAL
    assert "not an index file" in msi.msi_last_error()
    # a consistent header (n = 1000, len 256, 16 segments, cardinality 256, 4 leaves)
    # whose arrays are missing: rejected by its size
    hdr = struct.pack("<8sIIqiiiiiiIiqqQ4Q", b"MSIINDEX", 3, 112, 1000, 256, 16, 256, 8, 16, 2000, 0, 1, 4,
                      (1000 + 31) // 32, 0, 0, 0, 0, 0)
    assert len(hdr) == 112
    short = tmp_path / "short.idx"
    short.write_bytes(hdr + b"\0" * 100)
    assert lib.msi_index_load(str(short).encode(), None, None, ctypes.byref(out)) == msi.MSI_EINVAL
    assert "truncated" in msi.msi_last_error()
    # the same header claiming a borrowed collection needs one
    hdr_b = struct.pack("<8sIIqiiiiiiIiqqQ4Q", b"MSIINDEX", 3, 112, 1000, 256, 16, 256, 8, 16, 2000, 1, 0, 4,
                        (1000 + 31) // 32, 0, 0, 0, 0, 0)
    borrowed = tmp_path / "borrowed.idx"
    borrowed.write_bytes(hdr_b)
    assert lib.msi_index_load(str(borrowed).encode(), None, None, ctypes.byref(out)) == msi.MSI_EINVAL
    assert "borrows" in msi.msi_last_error()
    # files of earlier formats (no fine PAA section; the fine PAA in leaf order) are
    # refused by their version
    for v in (1, 2):
        old = tmp_path / f"v{v}.idx"
        old.write_bytes(hdr[:8] + struct.pack("<I", v) + hdr[12:] + b"\0" * 100)
        assert lib.msi_index_load(str(old).encode(), None, None, ctypes.byref(out)) == msi.MSI_EINVAL
        assert "version" in msi.msi_last_error()
    assert lib.msi_index_save(None, str(tmp_path / "x.idx").encode()) == msi.MSI_EINVAL
