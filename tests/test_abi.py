"""The C-ABI library loads and exports every entry point include/rsvd.h declares;
argument validation happens on the host before anything is launched (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsvd.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(rsvd_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1502_05366_gb300 import build as b
    b.build()
    import paper_1502_05366_gb300 as rs
    return rs.lib()


def test_every_declared_symbol_exported(lib):
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    import paper_1502_05366_gb300 as rs
    assert sorted(rs.exported_symbols()) == _declared()


def test_status_strings_and_defaults(lib):
    import paper_1502_05366_gb300 as rs
    assert lib.rsvd_status_string(0) == b"RSVD_OK"
    assert lib.rsvd_status_string(8) == b"RSVD_ERR_TIMEOUT"
    o = rs.make_opts()
    assert (o.s, o.max_sweeps, o.precision) == (1, 30, 0)
    assert lib.rsvd_version() >= 100


def test_workspace_queries_reject_bad_sizes(lib):
    import paper_1502_05366_gb300 as rs
    assert lib.rsvd_svd_workspace_size(100, 50, 0, 5, 1, rs.F32, None) == 0     # k = 0
    assert lib.rsvd_svd_workspace_size(100, 50, 40, 20, 1, rs.F32, None) == 0   # l > n
    assert lib.rsvd_svd_workspace_size(100, 50, 10, 5, 1, 7, None) == 0         # dtype
    assert lib.rsvd_id_workspace_size(100, 50, 50, 0, 1, rs.F64, None) == 0     # k = n
    assert lib.rsvd_svd_workspace_size(100, 50, 10, 5, 1, rs.F64, None) > 0
    assert lib.rsvd_svd_id_cur_workspace_size(50000, 20000, 200, 20, 2, rs.F32, None) > 0


def test_calls_reject_invalid_arguments_without_launching(lib):
    import paper_1502_05366_gb300 as rs
    vp = ctypes.c_void_p
    fake = vp(0x1000)
    # k = 0
    st = lib.rsvd_svd(100, 50, 0, 5, 1, 1, rs.F32, fake, 50, fake, 1, fake, fake, 1, fake,
                      1 << 20, None, None, None)
    assert st == 1
    # null A
    st = lib.rsvd_svd(100, 50, 5, 5, 1, 1, rs.F32, vp(0), 50, fake, 5, fake, fake, 5, fake,
                      1 << 20, None, None, None)
    assert st == 1
    # lda < n
    st = lib.rsvd_qb(100, 50, 5, 5, 1, 1, rs.F64, fake, 49, fake, 10, fake, 10, fake, 1 << 20,
                     None, None, None)
    assert st == 1
    # bf16 storage is not part of this build's paths
    st = lib.rsvd_qb(100, 50, 5, 5, 1, 1, rs.BF16, fake, 50, fake, 10, fake, 10, fake, 1 << 20,
                     None, None, None)
    assert st == 4
    # workspace too small
    st = lib.rsvd_qb(100, 50, 5, 5, 1, 1, rs.F64, fake, 50, fake, 10, fake, 10, fake, 16, None,
                     None, None)
    assert st == 2
    # bad options
    o = rs.make_opts()
    o.reserved[3] = 1
    st = lib.rsvd_qb(100, 50, 5, 5, 1, 1, rs.F64, fake, 50, fake, 10, fake, 10, fake, 1 << 20,
                     None, None, ctypes.byref(o))
    assert st == 1
