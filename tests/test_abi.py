"""The C ABI library builds, loads and exports what include/rmq.h declares;
host-only entry points behave (no GPU needed, no device work is issued)."""
import ctypes
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
                                 (510 * 32, 32), (511 * 32, 32)])
def test_bench_table_geometry_matches_the_library(lib, n, k):
    """bench.py counts the plain form's bytes with its own copy of the coarse
    geometry; it must give the library's workspace exactly."""
    import bench
    nb = -(-n // k)
    m1 = -(-n // 128) if k >= 128 else 0
    want = rmq.rmq_batch_workspace_bytes(n, 1000, rmq.Variant.PLAIN, k=k)
    assert 8 * (nb * (bench.coarse_lc(nb) + 1) + m1) == want


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
    p = tmp_path / "tune.txt"
    p.write_text("# log2n log2q variant k k_con\n27 23 2 2048 256\n")
    rmq.rmq_tune_load(p)
    t = rmq.rmq_tune(10**8, 10**7)                   # log2 1e8 ~ 26.6 -> 27, log2 1e7 ~ 23.3 -> 23
    assert t == {"variant": rmq.Variant.CONTRACTED, "k": 2048, "k_con": 256}
    assert rmq.rmq_tune(10**6, 10**3) == rmq.rmq_tune(10**6, 10**3)
    out = tmp_path / "saved.txt"
    rmq.rmq_tune_save(out)
    assert "27 23 2 2048 256" in out.read_text()
    rmq.rmq_tune_clear()
    assert rmq.rmq_tune(10**8, 10**7) == base
    bad = tmp_path / "bad.txt"
    bad.write_text("27 23 2 2047 256\n")
    with pytest.raises(rmq.RmqError):
        rmq.rmq_tune_load(bad)
    with pytest.raises(rmq.RmqError):
        rmq.rmq_tune_load(tmp_path / "missing.txt")
