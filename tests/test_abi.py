"""The C ABI library builds, loads and exports what include/rmq.h declares;
host-only entry points behave (no GPU needed, no device work is issued)."""
import ctypes
import math
import os
import re

import pytest

from paper_1706_06940_gb300 import _build, rmq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rmq.h")
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return rmq.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(rmq_[a-z_]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rmq_batch", "rmq_batch_ex", "rmq_build", "rmq_query", "rmq_free", "rmq_stream_status",
                 "rmq_strerror", "rmq_handle_bytes", "rmq_table_bytes", "rmq_tune"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(rmq.exported_symbols()) == names


def test_table_bytes_reproduces_table2(lib):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table2_memory.txt"))
            if l.strip() and not l.startswith("#")]
    for k, p8, p9 in rows:
        for n, printed in ((10**8, p8), (10**9, p9)):
            pct = 100.0 * rmq.rmq_table_bytes(n, int(k)) / (4 * n)
            assert abs(pct - float(printed)) <= 0.005 + 1e-9, (k, n, pct, printed)


def test_table_bytes_rejects_bad_arguments(lib):
    assert rmq.rmq_table_bytes(0, 512) == -1
    assert rmq.rmq_table_bytes(100, 48) == -1
    assert rmq.rmq_table_bytes(100, 16) == -1
    assert rmq.rmq_table_bytes(100, 1 << 17) == -1
    assert rmq.rmq_table_bytes(1, 32) == 8


@pytest.mark.parametrize("n,k", [(10**8, 1024), (10**9, 512), (10**9, 4096), (1000, 32), (5, 64)])
def test_plain_workspace_between_level_zero_and_the_full_table(lib, n, k):
    """The plain form keeps levels 0..lc of the block table (at least level 0,
    at most the full table of Table 2) plus, for k >= 128, one key per 128 cells."""
    ws = rmq.rmq_batch_workspace_bytes(n, 1000, rmq.Variant.PLAIN, k=k)
    nb = -(-n // k)
    m1 = 8 * (-(-n // 128)) if k >= 128 else 0
    assert 8 * nb + m1 <= ws <= rmq.rmq_table_bytes(n, k) + m1


@pytest.mark.parametrize("n,k", [(10**8, 1024), (10**8, 512), (10**9, 2048), (5000, 32), (1, 64),
                                 (510 * 32, 32), (511 * 32, 32), (1000, 128), (1024, 128), (2**20, 128),
                                 (2**31 - 1, 65536), (3 * 10**6, 256)])
def test_bench_table_geometry_matches_the_library(lib, n, k):
    """bench.py counts the plain form's bytes with its own copy of the coarse
    geometry; it must give the library's workspace exactly."""
    import bench
    want = rmq.rmq_batch_workspace_bytes(n, 1000, rmq.Variant.PLAIN, k=k)
    assert bench.plain_workspace(n, k) == want


def test_contracted_workspace_holds_the_bitmap_and_a_q(lib):
    n = 10**9
    prev = 0
    for q in (10, 10**4, 10**6, 10**7, 10**8, 10**9):
        ws = rmq.rmq_batch_workspace_bytes(n, q, rmq.Variant.CONTRACTED, k_con=256)
        a_q = 8 * (min(2 * q, n) - 1)
        assert ws >= 8 * (n // 32) + a_q, q
        assert ws >= prev
        prev = ws


def test_workspace_bytes_rejects_bad_arguments(lib):
    assert rmq.rmq_batch_workspace_bytes(0, 10) == -1
    assert rmq.rmq_batch_workspace_bytes(100, -1) == -1
    assert rmq.rmq_batch_workspace_bytes(100, 10, k=48) == -1
    assert rmq.rmq_batch_workspace_bytes(100, 10, variant=7) == -1
    assert rmq.rmq_batch_workspace_bytes(100, 0) == 0


@pytest.mark.parametrize("n,q", [(1, 1), (1000, 10), (10**6, 1000), (10**8, 10**7), (2**31 - 1, 2**31 - 1)])
def test_tune_returns_valid_options(lib, n, q):
    t = rmq.rmq_tune(n, q)
    for k in (t["k"], t["k_con"]):
        assert 32 <= k <= 65536 and k & (k - 1) == 0
    assert t["variant"] in (rmq.Variant.PLAIN, rmq.Variant.CONTRACTED)


def test_strerror_covers_every_status(lib):
    for s in rmq.Status:
        assert rmq.strerror(s) and rmq.strerror(s) != "unknown status"
    assert lib.rmq_strerror(99) == b"unknown status"


def test_host_checks_reject_bad_arguments_before_any_device_work(lib):
    o = rmq.rmq_opts(0, 0, 0, 0)
    bad_k = rmq.rmq_opts(0, 48, 0, 0)
    bad_v = rmq.rmq_opts(7, 0, 0, 0)
    bad_f = rmq.rmq_opts(0, 0, 0, 1)
    p = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    E = rmq.Status.ERR_INVALID_ARG
    assert lib.rmq_batch(None, 10, p, p, 5, p, None) == E              # null A
    assert lib.rmq_batch(p, 0, p, p, 5, p, None) == E                  # n <= 0
    assert lib.rmq_batch(p, 2**31, p, p, 5, p, None) == E              # n too large
    assert lib.rmq_batch(p, 10, None, p, 5, p, None) == E              # null l with q > 0
    assert lib.rmq_batch(p, 10, p, p, -1, p, None) == E                # q < 0
    assert lib.rmq_batch(p, 10, p, p, 2**31, p, None) == E             # q too large (2^31 - 1 is the limit)
    assert lib.rmq_batch_ex(p, 10, p, p, 5, p, ctypes.byref(bad_k), None) == E
    assert lib.rmq_batch_ex(p, 10, p, p, 5, p, ctypes.byref(bad_v), None) == E
    assert lib.rmq_batch_ex(p, 10, p, p, 5, p, ctypes.byref(bad_f), None) == E
    assert lib.rmq_batch_ex(p, 10, None, None, 0, None, ctypes.byref(o), None) == 0   # q == 0: no-op
    h = ctypes.c_void_p()
    assert lib.rmq_build(None, 10, None, None, ctypes.byref(h)) == E
    assert lib.rmq_build(p, 10, None, None, None) == E
    assert lib.rmq_query(None, p, p, 1, p, None) == E
    assert lib.rmq_block_minima(p, 10, 33, p, None) == E
    assert lib.rmq_sparse_table_build(None, 10, None) == E
    assert lib.rmq_handle_bytes(None) == 0
    lib.rmq_free(None)


def test_tune_table_load_save_roundtrip(lib, tmp_path):
    rmq.rmq_tune_clear()
    base = rmq.rmq_tune(10**8, 10**7)
    assert base["threads_per_query"] == 0 and base["k1"] == 0
    p = tmp_path / "tune.txt"
    # the older five-field line: a choice that serves every width class of its shape
    p.write_text("# log2n log2q variant k k_con\n27 23 2 2048 256\n")
    rmq.rmq_tune_load(p)
    t = rmq.rmq_tune(10**8, 10**7)                   # log2 1e8 ~ 26.6 -> 27, log2 1e7 ~ 23.3 -> 23
    assert t == {"variant": rmq.Variant.CONTRACTED, "k": 2048, "k_con": 256, "threads_per_query": 0, "k1": 0}
    rmq.rmq_tune_clear()
    # two width classes of one shape; rmq_tune gives the lowest class
    p.write_text("# log2n log2q wclass variant k k_con threads_per_query k1\n"
                 "27 23 25 1 1024 256 8 -1\n27 23 7 2 1024 32 16 0\n")
    rmq.rmq_tune_load(p)
    assert rmq.rmq_tune(10**8, 10**7) == {"variant": rmq.Variant.CONTRACTED, "k": 1024, "k_con": 32,
                                          "threads_per_query": 16, "k1": 0}
    assert rmq.rmq_tune(10**6, 10**3) == rmq.rmq_tune(10**6, 10**3)
    out = tmp_path / "saved.txt"
    rmq.rmq_tune_save(out)
    text = out.read_text()
    assert "27 23 25 1 1024 256 8 -1" in text and "27 23 7 2 1024 32 16 0" in text
    rmq.rmq_tune_clear()
    assert rmq.rmq_tune(10**8, 10**7) == base
    rmq.rmq_tune_load(out)                            # what was saved loads back
    assert rmq.rmq_tune(10**8, 10**7)["k_con"] == 32
    rmq.rmq_tune_clear()
    for bad_line in ("27 23 2 2047 256\n",           # k not a power of two
                     "27 23 7 1 1024 256 12 0\n",     # threads_per_query not 8, 16 or 32
                     "27 23 7 1 256 256 0 512\n",     # k1 > k
                     "27 23\n"):
        bad = tmp_path / "bad.txt"
        bad.write_text(bad_line)
        with pytest.raises(rmq.RmqError):
            rmq.rmq_tune_load(bad)
    with pytest.raises(rmq.RmqError):
        rmq.rmq_tune_load(tmp_path / "missing.txt")


def test_new_option_fields_are_checked_before_device_work(lib):
    p = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    E = rmq.Status.ERR_INVALID_ARG
    for o in (rmq.rmq_opts(0, 0, 0, 0, 12, 0),      # threads_per_query not 8, 16 or 32
              rmq.rmq_opts(0, 0, 0, 0, 0, 48),      # k1 not a power of two
              rmq.rmq_opts(0, 0, 0, 0, 0, 16),      # k1 below 32
              rmq.rmq_opts(1, 256, 0, 0, 0, 512),   # k1 > k
              rmq.rmq_opts(0, 0, 0, 0, 0, -2)):
        assert lib.rmq_batch_ex(p, 10, p, p, 5, p, ctypes.byref(o), None) == E
    assert rmq.rmq_batch_workspace_bytes(10**6, 100, variant=1, k=256, k1=512) == -1
    # k1 sizes the small-block minima of the plain form
    base = rmq.rmq_batch_workspace_bytes(10**6, 100, variant=1, k=1024, k1=-1)
    assert rmq.rmq_batch_workspace_bytes(10**6, 100, variant=1, k=1024, k1=32) == base + 8 * (10**6 // 32)
    assert rmq.rmq_batch_workspace_bytes(10**6, 100, variant=1, k=1024) == base + 8 * (-(-10**6 // 128))
    assert rmq.rmq_batch_workspace_bytes(10**6, 100, variant=1, k=64) == \
        rmq.rmq_batch_workspace_bytes(10**6, 100, variant=1, k=64, k1=-1)


HLEVEL_CASES = [(10**8, (4096, 65536)), (10**8, (128, 1024, 16384)), (10**9, (64, 512, 4096, 65536)),
                (1000, (32,)), (12345, (32, 64)), (10**6, (32, 1 << 30)), (2**31 - 1, (65536, 1 << 20))]


@pytest.mark.parametrize("n,ks", HLEVEL_CASES)
def test_hlevel_bytes_is_the_space_of_sec33(lib, n, ks):
    """Eight bytes per entry of the oracle's space count (minima of levels
    below h, and the sparse table over blocks of k_h); one level is the
    one-level table of Table 2."""
    import oracle
    assert rmq.rmq_hlevel_bytes(n, ks) == 8 * oracle.hlevel_space(n, ks)
    if len(ks) == 1:
        assert rmq.rmq_hlevel_bytes(n, ks) == rmq.rmq_table_bytes(n, ks[0])


def test_hlevel_rejects_bad_block_sizes_before_device_work(lib):
    p = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    E = rmq.Status.ERR_INVALID_ARG
    for ks in ((), (16,), (48, 96), (64, 64), (128, 64), (32, 3 << 29),
               (1 << 17, 1 << 18), tuple(32 << i for i in range(9))):
        assert rmq.rmq_hlevel_bytes(1000, ks) == -1, ks
        arr, h = rmq._ks_array(ks)
        assert lib.rmq_batch_hlevel(p, 1000, p, p, 5, p, ctypes.cast(arr, ctypes.c_void_p), h, None) == E, ks
    arr, h = rmq._ks_array((64, 256))
    assert lib.rmq_batch_hlevel(p, 1000, p, p, 5, p, None, 2, None) == E
    assert lib.rmq_batch_hlevel(None, 1000, p, p, 5, p, ctypes.cast(arr, ctypes.c_void_p), h, None) == E
    assert rmq.rmq_hlevel_bytes(0, (64,)) == -1


@pytest.mark.parametrize("n", [10**6, 10**8, 10**9, 2**31 - 1])
def test_hlevel_paper_ks_follow_sec33(lib, n):
    """h = 2: the two sizes Sec. 3.3 gives first, sqrt(n) / log^(1/3) n and
    sqrt(n) log^(2/3) n, each rounded to the nearest power of two; every h:
    powers of two, each at least twice the one before, and the structure
    smaller than the one-level table of k = k_1."""
    lg, sq = math.log2(n), math.sqrt(n)
    want = (1 << round(math.log2(sq / lg ** (1 / 3))), 1 << round(math.log2(sq * lg ** (2 / 3))))
    assert rmq.rmq_hlevel_paper_ks(n, 2) == want
    for h in range(2, 6):
        ks = rmq.rmq_hlevel_paper_ks(n, h)
        assert len(ks) == h and all(k & (k - 1) == 0 for k in ks)
        assert all(b >= 2 * a for a, b in zip(ks, ks[1:]))
        assert 32 <= ks[0] <= 65536
        assert rmq.rmq_hlevel_bytes(n, ks) < rmq.rmq_table_bytes(n, ks[0])
    with pytest.raises(rmq.RmqError):
        rmq.rmq_hlevel_paper_ks(n, 1)
