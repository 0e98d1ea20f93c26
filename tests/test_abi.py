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


def test_workspace_queries_wide_shapes(lib):
    """Short, wide A (m < n) is accepted while l = k + p <= m; the CUR also
    needs k < m (it selects k of the m rows)."""
    import paper_1502_05366_gb300 as rs
    for dt in (rs.F32, rs.F64):
        assert lib.rsvd_svd_workspace_size(700, 1900, 30, 10, 1, dt, None) > 0
        assert lib.rsvd_svd_id_cur_workspace_size(517, 2049, 37, 11, 2, dt, None) > 0
        assert lib.rsvd_svd_workspace_size(60, 500, 50, 10, 1, dt, None) > 0      # l = m
        assert lib.rsvd_svd_workspace_size(60, 500, 50, 11, 1, dt, None) == 0     # l > m
        assert lib.rsvd_cur_workspace_size(60, 500, 60, 0, 1, dt, None) == 0      # k = m
    assert lib.rsvd_svd_id_cur_workspace_size(520, 2048, 37, 11, 2, rs.BF16, None) > 0


def test_id_and_cur_rank_limit(lib):
    """Every call that forms an ID or a CUR takes k <= 880 (its triangular
    solve); beyond, the workspace queries return 0 and the calls return
    RSVD_ERR_UNSUPPORTED before launching anything.  The SVD alone has no
    such bound."""
    import paper_1502_05366_gb300 as rs
    m, n, p, q = 2000, 1500, 0, 1
    queries = (lib.rsvd_id_workspace_size, lib.rsvd_cur_workspace_size,
               lib.rsvd_svd_id_cur_workspace_size, lib.rsvd_id_tol_workspace_size,
               lib.rsvd_cur_tol_workspace_size, lib.rsvd_id_left_workspace_size)
    for dt in (rs.F32, rs.F64):
        for f in queries:
            assert f(m, n, 880, p, q, dt, None) > 0
            assert f(m, n, 881, p, q, dt, None) == 0
        assert lib.rsvd_svd_workspace_size(m, n, 881, p, q, dt, None) > 0
    assert lib.rsvd_cpqr_workspace_size(900, n, 880) > 0
    assert lib.rsvd_cpqr_workspace_size(900, n, 881) == 0
    vp = ctypes.c_void_p
    fake = vp(0x1000)
    k = 881
    st = lib.rsvd_id(m, n, k, p, q, 1, rs.F32, fake, n, fake, fake, n - k, fake, 1 << 20, None,
                     None, None)
    assert st == 4
    rank = ctypes.c_int(0)
    st = lib.rsvd_id_tol(m, n, k, p, q, 1e-3, 1, rs.F32, fake, n, fake, fake, n - 1,
                         ctypes.byref(rank), fake, 1 << 20, None, None, None)
    assert st == 4
    st = lib.rsvd_cpqr_id(900, n, k, fake, n, fake, fake, n - k, None, fake, 1 << 20, None, None)
    assert st == 4
    # the binding reports a zero workspace query beyond the bound as unsupported
    assert rs.ID_MAX_K == 880
    with pytest.raises(rs.RsvdError) as e:
        rs._no_workspace("rsvd_id_workspace_size", 881)
    assert e.value.code == 4
    with pytest.raises(rs.RsvdError) as e:
        rs._no_workspace("rsvd_id_workspace_size", 880)
    assert e.value.code == 1


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
    # bf16 A whose rows are not 16-byte aligned (lda % 8 != 0): not TMA-addressable
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


def test_bf16_and_mixed_workspace_queries(lib):
    import paper_1502_05366_gb300 as rs
    assert lib.rsvd_svd_workspace_size(3000, 2000, 40, 10, 2, rs.BF16, None) > 0
    simt = rs.make_opts(precision=rs.PREC_SIMT)
    assert lib.rsvd_svd_workspace_size(3000, 2000, 40, 10, 2, rs.BF16, ctypes.byref(simt)) == 0
    mixed = rs.make_opts(precision=rs.PREC_MIXED)
    assert lib.rsvd_svd_workspace_size(3000, 2000, 40, 10, 2, rs.F32, ctypes.byref(mixed)) > 0
    bad = rs.make_opts()
    bad.precision = 4
    assert lib.rsvd_svd_workspace_size(3000, 2000, 40, 10, 2, rs.F32, ctypes.byref(bad)) == 0
    # the FP8 sketch: tensor-core path only (FP32 or BF16 A), with its Omega^T
    fp8 = rs.make_opts(precision=rs.PREC_FP8)
    plain = lib.rsvd_svd_workspace_size(3000, 2000, 40, 10, 2, rs.F32, None)
    assert lib.rsvd_svd_workspace_size(3000, 2000, 40, 10, 2, rs.F32, ctypes.byref(fp8)) > plain
    assert lib.rsvd_svd_workspace_size(3000, 2000, 40, 10, 2, rs.F64, ctypes.byref(fp8)) == 0
    assert lib.rsvd_sample_workspace_size(3000, 2000, 50, rs.F64, ctypes.byref(fp8)) == 0
    # widths above 256 (column chunks) up to 1024 on the tensor-core path
    assert lib.rsvd_svd_workspace_size(100000, 50000, 500, 50, 2, rs.BF16, None) > 0
    assert lib.rsvd_svd_workspace_size(100000, 50000, 1000, 50, 2, rs.BF16, None) == 0


def _items(rs, sizes):
    items = (rs.BatchItem * len(sizes))()
    a = u = v = s = 0
    for i, (m, n, k) in enumerate(sizes):
        items[i].m, items[i].n, items[i].k = m, n, k
        items[i].a_off, items[i].u_off, items[i].v_off, items[i].s_off = a, u, v, s
        a, u, v, s = a + m * n, u + m * k, v + n * k, s + k
    return items


def test_batched_workspace_and_validation(lib):
    import paper_1502_05366_gb300 as rs
    good = _items(rs, [(300, 150, 8), (1000, 700, 16), (96, 80, 64)])
    w = lib.rsvd_svd_batched_workspace_size(3, good, 8, 1)
    assert w > 0
    # more problems or a wider sketch need more workspace
    assert lib.rsvd_svd_batched_workspace_size(2, good, 8, 1) < w
    assert lib.rsvd_svd_batched_workspace_size(3, good, 16, 1) > w
    assert lib.rsvd_svd_batched_workspace_size(3, _items(rs, [(300, 150, 121)] * 3), 8, 1) == 0
    assert lib.rsvd_svd_batched_workspace_size(1, _items(rs, [(100, 50, 45)]), 8, 1) == 0
    assert lib.rsvd_svd_batched_workspace_size(1, _items(rs, [(100, 50, 0)]), 8, 1) == 0
    assert lib.rsvd_svd_batched_workspace_size(0, good, 8, 1) == 0
    assert lib.rsvd_svd_batched_workspace_size(3, good, 8, -1) == 0


def test_batched_call_rejects_without_launching(lib):
    import paper_1502_05366_gb300 as rs
    vp = ctypes.c_void_p
    fake = vp(0x100000)
    good = _items(rs, [(300, 150, 8), (1000, 700, 16)])
    w = lib.rsvd_svd_batched_workspace_size(2, good, 8, 1)
    # null A
    assert lib.rsvd_svd_batched(2, good, 8, 1, 5, vp(0), fake, fake, fake, fake, w, None,
                                None) == 1
    # work not 256-byte aligned
    assert lib.rsvd_svd_batched(2, good, 8, 1, 5, fake, fake, fake, fake, vp(0x100010), w,
                                None, None) == 1
    # workspace too small
    assert lib.rsvd_svd_batched(2, good, 8, 1, 5, fake, fake, fake, fake, fake, w - 4096,
                                None, None) == 2
    # a bad item
    bad = _items(rs, [(300, 150, 8), (100, 50, 45)])
    assert lib.rsvd_svd_batched(2, bad, 8, 1, 5, fake, fake, fake, fake, fake, w, None,
                                None) == 1


def test_batched_workload_sizes():
    from synth import BATCH_CONFIGS, batch_sizes
    c = BATCH_CONFIGS["c4_f32_batched512"]
    ms, ns, ks = batch_sizes("c4_f32_batched512")
    assert len(ms) == len(ns) == len(ks) == 512
    assert batch_sizes("c4_f32_batched512") == (ms, ns, ks)      # seeded
    for m, n, k in zip(ms, ns, ks):
        assert c["m_range"][0] <= m <= c["m_range"][1]
        assert k in c["ks"]
        assert k + c["p"] <= n <= m


def test_adaptive_qb_workspace_and_validation(lib):
    import paper_1502_05366_gb300 as rs
    ws = lib.rsvd_qb_adaptive_workspace_size
    assert ws(3000, 2000, 32, 8, 1, rs.F32, None) > 0
    assert ws(3000, 2000, 32, 8, 1, rs.F64, None) > 0
    assert ws(3000, 2000, 32, 8, 1, rs.BF16, None) == 0          # A is updated in place
    assert ws(300, 200, 64, 4, 1, rs.F32, None) == 0             # b M > min(m, n)
    assert ws(300, 200, 0, 4, 1, rs.F32, None) == 0              # b = 0
    assert ws(300, 200, 16, 0, 1, rs.F32, None) == 0             # M = 0
    assert ws(3000, 2000, 1040, 1, 1, rs.F32, None) == 0         # b > 1024
    # more blocks need more re-projection scratch
    assert ws(3000, 2000, 32, 16, 1, rs.F32, None) > ws(3000, 2000, 32, 2, 1, rs.F32, None)
    rank = ctypes.c_int(-1)
    fake = ctypes.c_void_p(256)        # never dereferenced: every call below fails its checks
    call = lib.rsvd_qb_adaptive

    def st(**kw):
        a = dict(m=300, n=200, b=16, M=4, q=1, eps=1e-3, rel=1, dt=rs.F32, A=fake, lda=200,
                 Q=fake, ldq=64, Bt=fake, ldbt=64, resid=fake, rank=ctypes.byref(rank),
                 work=None, wb=0)
        a.update(kw)
        return call(a["m"], a["n"], a["b"], a["M"], a["q"], a["eps"], a["rel"], 1, a["dt"],
                    a["A"], a["lda"], a["Q"], a["ldq"], a["Bt"], a["ldbt"], a["resid"],
                    a["rank"], a["work"], a["wb"], None, None, None)

    assert st(eps=-1.0) == 1
    assert st(eps=float("nan")) == 1
    assert st(eps=float("inf")) == 1
    assert st(A=None) == 1
    assert st(resid=None) == 1
    assert st(rank=None) == 1
    assert st(lda=199) == 1
    assert st(ldq=63) == 1
    assert st(ldbt=63) == 1
    assert st(b=64) == 1
    assert st(dt=rs.BF16) == 4
    assert st(q=65) == 1
    assert st() == 2                   # no workspace
    assert rank.value == -1            # nothing ran


def test_noalloc_scratch_limits(lib):
    """The 16 MiB static scratch of rsvd_small_svd_noalloc holds the small-SVD
    workspace up to l = 512 (FP64) and l = 720 (FP32), and no further: the
    documented limits follow the workspace layout."""
    import paper_1502_05366_gb300 as rs
    cap = 16 << 20
    assert lib.rsvd_small_svd_workspace_size(512, rs.F64, None) <= cap
    assert lib.rsvd_small_svd_workspace_size(513, rs.F64, None) > cap
    assert lib.rsvd_small_svd_workspace_size(720, rs.F32, None) <= cap
    assert lib.rsvd_small_svd_workspace_size(721, rs.F32, None) > cap


def test_barrier_wait_test_aid_arguments(lib):
    assert lib.rsvd_test_set_barrier_wait(-1, 0) == 1        # RSVD_ERR_INVALID_ARG
    assert lib.rsvd_test_set_barrier_wait(1000, 1) == 0
    assert lib.rsvd_test_set_barrier_wait(0, 1) == 0          # defaults restored
