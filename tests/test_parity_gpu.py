"""GPU parity: every step of the CUDA path, called through the C ABI, against
the CPU oracle on the same seeded inputs.  Answers are integers (positions),
so every comparison is exact."""
import numpy as np
import pytest

import oracle
from paper_1706_06940_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1706_06940_gb300 import rmq
    return rmq


DEV = "cuda:0"
I32_MIN, I32_MAX = -2**31, 2**31 - 1


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def run_batch(R, A, l, r, variant, k=0, k_con=0, offset=0):
    """Answer on the GPU; `offset` shifts A, l, r and out by that many int32
    cells inside larger buffers to exercise unaligned pointers."""
    n, q = len(A), len(l)
    bufA = torch.zeros(n + offset, dtype=torch.int32, device=DEV)
    bufA[offset:] = dev(A)
    bl = torch.zeros(q + offset, dtype=torch.int32, device=DEV)
    br = torch.zeros(q + offset, dtype=torch.int32, device=DEV)
    bo = torch.full((q + offset,), -7, dtype=torch.int32, device=DEV)
    bl[offset:], br[offset:] = dev(l), dev(r)
    R.rmq_batch_ex(bufA[offset:], bl[offset:], br[offset:], bo[offset:], variant=variant, k=k, k_con=k_con)
    st = R.rmq_stream_status()
    return bo[offset:].cpu().numpy(), st


def check(R, A, l, r, want=None, variants=None, ks=(0,), kcons=(0,), offsets=(0,)):
    if want is None:
        want = oracle.rmq_naive(A, l, r)
    for v in variants or (R.Variant.PLAIN, R.Variant.CONTRACTED):
        for k in ks:
            for kc in kcons:
                for off in offsets:
                    got, st = run_batch(R, A, l, r, v, k, kc, off)
                    bad = np.nonzero(got != want)[0]
                    assert len(bad) == 0, (v.name, k, kc, off, len(bad), bad[:5], got[bad[:5]], want[bad[:5]])
                    expect = R.Status.ERR_QUERY_RANGE if (want < 0).any() else R.Status.OK
                    assert st == expect, (v.name, k, st)


def keys_pos(T):
    return (T.cpu().numpy().view(np.uint64) & np.uint64(0xFFFFFFFF)).astype(np.int64)


def keys_val(T):
    hi = (T.cpu().numpy().view(np.uint64) >> np.uint64(32)).astype(np.uint32)
    return (hi ^ np.uint32(0x80000000)).view(np.int32)


# ------------------------------------------------------------------ step a1

@pytest.mark.parametrize("n,k,hi", [(1, 32, 5), (31, 32, 5), (1000, 32, 3), (1000, 64, 3),
                                    (4096 * 5 + 3, 128, 2**31), (100_000, 512, 100),
                                    (100_001, 4096, 7), (300_000, 65536, 2**31), (12345, 256, 1)])
@pytest.mark.parametrize("offset", [0, 1])
def test_a1_block_minima(R, n, k, hi, offset):
    A = W.uniform_array(n, n + k, -2**31 if hi == 2**31 else 0, hi)
    nb = -(-n // k)
    buf = torch.zeros(n + offset, dtype=torch.int32, device=DEV)
    buf[offset:] = dev(A)
    T0 = torch.zeros(nb, dtype=torch.int64, device=DEV)
    R.rmq_block_minima(buf[offset:], k, T0)
    torch.cuda.synchronize()
    want = oracle.block_minima(A, k)
    assert np.array_equal(keys_pos(T0), want)
    assert np.array_equal(keys_val(T0), A[want])


# ------------------------------------------------------------------ step a2

@pytest.mark.parametrize("n,k,hi", [(32, 32, 5), (64, 32, 5), (33 * 32 + 1, 32, 3), (5000 * 32 + 7, 32, 1000),
                                    (9000 * 64, 64, 2), (4097 * 32 + 5, 32, 2**31)])
def test_a2_block_sparse_table(R, n, k, hi):
    A = W.uniform_array(n, 2 * n + k, 0, hi)
    nb = -(-n // k)
    lv = oracle.sparse_levels(nb)
    T = torch.zeros(nb * lv, dtype=torch.int64, device=DEV)
    R.rmq_block_minima(dev(A), k, T[:nb])
    R.rmq_sparse_table_build(T, nb)
    torch.cuda.synchronize()
    got = keys_pos(T).reshape(lv, nb)
    want = oracle.block_sparse_table(A, k)
    valid = want >= 0
    assert np.array_equal(got[valid], want[valid])


# ------------------------------------------------------------------ step a3 / a7

KS = (32, 64, 128, 512, 4096, 65536)


@pytest.mark.parametrize("n,q,hi", [(1000, 3000, 2**31), (70_001, 20_000, 2**31), (70_001, 20_000, 3),
                                    (200_000, 5_000, 1000)])
def test_a3_a7_uniform_queries_all_k(R, n, q, hi):
    A = W.uniform_array(n, n, 0, hi)
    l, r = W.uniform_queries(n, q, n + 1)
    check(R, A, l, r, ks=KS, kcons=(32, 512, 4096))


@pytest.mark.parametrize("hi", [2**31, 1000, 2])
def test_a3_a7_short_and_tie_heavy(R, hi):
    n = 300_000
    A = W.uniform_array(n, 31, 0, hi)
    l, r = W.log_width_queries(n, 50_000, 32, 1, 10_000)
    check(R, A, l, r, ks=(32, 512, 4096), kcons=(32, 512))


@pytest.mark.parametrize("hi", [2**31, 50])
def test_part_pool_full_and_not_full(R, hi):
    """2,000 short queries run in one CTA of the query kernel, and most of them
    leave edge parts: the first parts go to the CTA's pool (256 at most) and
    are drained after phase A, the rest are drained at once by their warps."""
    n = 1_000_000
    A = W.uniform_array(n, 51, 0, hi)
    l, r = W.log_width_queries(n, 2_000, 52, 100, 3_000)
    check(R, A, l, r, ks=(512, 1024), kcons=(256,))


def test_unaligned_pointers(R):
    n = 50_003
    A = W.uniform_array(n, 41, 0, 50)
    l, r = W.log_width_queries(n, 10_001, 42, 1, 3000)
    check(R, A, l, r, ks=(64, 1024), kcons=(64,), offsets=(0, 1, 2, 3))


def test_ties_straddling_block_boundaries(R):
    n, k = 64 * 1024, 1024
    A = np.full(n, 10, dtype=np.int32)
    for j in range(1, 64):
        A[j * k - 2: j * k + 2] = 1                         # equal minima around every boundary
    A[5 * k + 17] = 0
    A[40 * k - 1] = 0
    l, r = W.uniform_queries(n, 20_000, 43)
    ll = np.repeat(np.arange(1, 64) * k - 3, 1).astype(np.int32)
    l = np.concatenate([l, ll, ll + 1, ll + 2, ll + 3])
    r = np.concatenate([r, ll + 5, ll + 4, ll + 2000, ll + 4000]).clip(max=n - 1).astype(np.int32)
    check(R, A, l, r, ks=(32, 1024, 2048), kcons=(32, 512))


def test_degenerate_arrays_and_queries(R):
    n = 10_000
    for A in (np.full(n, 5, dtype=np.int32), np.arange(n, dtype=np.int32),
              np.arange(n, 0, -1, dtype=np.int32), np.full(n, I32_MIN, dtype=np.int32),
              np.full(n, I32_MAX, dtype=np.int32),
              W.uniform_array(n, 44, I32_MIN, 2**31)):
        l, r = W.uniform_queries(n, 3000, 45)
        l[:100] = r[:100]                                   # l == r
        l[100:200], r[100:200] = 0, n - 1                   # whole array
        l[200:300] = 0                                      # touching both ends
        r[300:400] = n - 1
        check(R, A, l, r, ks=(32, 4096))


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 64, 95, 96, 97, 1000])
def test_small_n_and_few_blocks(R, n):
    A = W.uniform_array(n, n + 50, 0, 4)
    l, r = oracle_all_ranges(n)
    check(R, A, l, r, ks=(32,), kcons=(32,))


# Block counts (k = 32) around the largest coarse summaries that keep one
# block per coarse block (510 coarse blocks for the plain form's 4096-entry
# summary, 766 for the contracted form's 6656-entry one), around the level
# boundaries 512, 1024 and 2048, and around the next doubling (1020/1021,
# 1532/1533); the contracted form sees comparable counts over A_Q.
@pytest.mark.parametrize("nb", [510, 511, 512, 766, 767, 1021, 1024, 1025, 1532, 1533, 2047])
def test_coarse_summary_capacity_boundaries(R, nb):
    n = nb * 32 - 5
    A = W.uniform_array(n, nb + 60, 0, 1000)
    l, r = W.uniform_queries(n, 20_000, nb + 61)
    ls, rs = W.log_width_queries(n, 3000, nb + 62, 1, 3000)
    l, r = np.concatenate([l, ls, [0, n - 1, 0]]), np.concatenate([r, rs, [n - 1, n - 1, 0]])
    check(R, A, l.astype(np.int32), r.astype(np.int32), ks=(32, 64), kcons=(32,))


def oracle_all_ranges(n):
    i, j = np.triu_indices(n)
    return i.astype(np.int32), j.astype(np.int32)


def test_identical_and_single_queries(R):
    n = 100_000
    A = W.uniform_array(n, 46, 0, 100)
    for l, r in ((np.full(5000, 123, dtype=np.int32), np.full(5000, 99_000, dtype=np.int32)),
                 (np.array([7], dtype=np.int32), np.array([88_888], dtype=np.int32)),
                 (np.array([n - 1], dtype=np.int32), np.array([n - 1], dtype=np.int32))):
        check(R, A, l, r, ks=(32, 512), kcons=(32, 512))


def test_empty_batch_is_a_noop(R):
    A = dev(W.uniform_array(100, 47))
    e = torch.zeros(0, dtype=torch.int32, device=DEV)
    for v in (R.Variant.PLAIN, R.Variant.CONTRACTED):
        R.rmq_batch_ex(A, e, e, e, variant=v)
    assert R.rmq_stream_status() == R.Status.OK


def test_invalid_queries_answer_minus_one_and_raise_the_error_word(R):
    n = 1000
    A = W.uniform_array(n, 48, 0, 10)
    l, r = W.uniform_queries(n, 500, 49)
    l[10], r[10] = -1, 5
    l[20], r[20] = 5, n
    l[30], r[30] = 600, 599
    want = oracle.rmq_naive(A, l, r)
    assert (want[[10, 20, 30]] == -1).all()
    check(R, A, l, r, want=want, ks=(32, 256), kcons=(32,))
    assert R.rmq_stream_status() == R.Status.OK             # the word was cleared by the last report


# ------------------------------------------------------------------ steps a4 / a5 / a6

@pytest.mark.parametrize("n,q", [(1, 3), (255, 1000), (256, 1000), (100_000, 1), (1_000_000, 70_000),
                                 (2**27 + 3, 5000)])
def test_a4_sort_endpoints(R, n, q):
    l, r = W.uniform_queries(n, q, n + q)
    l[: q // 10] = r[: q // 10]
    pos = torch.zeros(2 * q, dtype=torch.int32, device=DEV)
    tag = torch.zeros(2 * q, dtype=torch.int32, device=DEV)
    R.rmq_sort_endpoints(dev(l), dev(r), n, pos, tag)
    torch.cuda.synchronize()
    wp, wt = oracle.sort_endpoints(l, r)
    assert np.array_equal(pos.cpu().numpy().view(np.uint32), wp)
    assert np.array_equal(tag.cpu().numpy().view(np.uint32), wt)


@pytest.mark.parametrize("n,q", [(1, 3), (10, 1000), (100_000, 9_999), (1_000_000, 70_000)])
def test_a5_rank_endpoints(R, n, q):
    l, r = W.uniform_queries(n, q, 7 * q)
    wp, wt = oracle.sort_endpoints(l, r)
    P_want, ra_want, rb_want = oracle.rank_endpoints(wp, wt, q)
    P = torch.zeros(2 * q, dtype=torch.int32, device=DEV)
    m = torch.zeros(1, dtype=torch.int64, device=DEV)
    ra = torch.zeros(q, dtype=torch.int32, device=DEV)
    rb = torch.zeros(q, dtype=torch.int32, device=DEV)
    R.rmq_rank_endpoints(dev(wp.view(np.int32)), dev(wt.view(np.int32)), q, P, m, ra, rb)
    torch.cuda.synchronize()
    mm = int(m.item())
    assert mm == len(P_want)
    assert np.array_equal(P.cpu().numpy()[:mm].view(np.uint32), P_want)
    assert np.array_equal(ra.cpu().numpy(), ra_want)
    assert np.array_equal(rb.cpu().numpy(), rb_want)


def bitmap_ranks_host(BP, pos):
    """Rank of each position from the bit words (first half of BP) and the
    counts (second half): count + popcount of the word's bits below the
    position."""
    half = len(BP) // 2
    w = BP[:half].view(np.uint32)
    c = BP[half:].view(np.uint32).astype(np.int64)
    idx = pos >> 5
    below = w[idx] & ((np.uint32(1) << (pos & 31).astype(np.uint32)) - np.uint32(1))
    pc = np.array([bin(int(x)).count("1") for x in below], dtype=np.int64)
    return c[idx] + pc


@pytest.mark.parametrize("n,q", [(1, 3), (33, 1000), (1024, 5000), (100_000, 1), (100_000, 9_999),
                                 (1_000_003, 70_000), (2**27 + 3, 5000)])
def test_a4_a5_endpoint_bitmap(R, n, q):
    """The batch path's step 1: the set bits are the oracle's P, the rank of
    every endpoint is the oracle's rank, and m is the number of distinct
    positions."""
    l, r = W.uniform_queries(n, q, 11 * q + n)
    l[: q // 10] = r[: q // 10]
    nbp = -(-n // 32) + 1
    BP = torch.full((2 * nbp,), -1, dtype=torch.int32, device=DEV)
    m = torch.zeros(1, dtype=torch.int64, device=DEV)
    R.rmq_endpoint_bitmap(dev(l), dev(r), n, BP, m)
    torch.cuda.synchronize()
    assert R.rmq_stream_status() == R.Status.OK
    bp = BP.cpu().numpy()
    wp, wt = oracle.sort_endpoints(l, r)
    P_want, ra_want, rb_want = oracle.rank_endpoints(wp, wt, q)
    bits = np.unpackbits(np.ascontiguousarray(bp[:nbp]).view(np.uint8), bitorder="little")
    assert np.array_equal(np.nonzero(bits)[0].astype(np.uint32), P_want)
    assert int(m.item()) == len(P_want) and bp[-1] == len(P_want) and bp[nbp - 1] == 0
    assert np.array_equal(bitmap_ranks_host(bp, l.astype(np.int64)), ra_want)
    assert np.array_equal(bitmap_ranks_host(bp, r.astype(np.int64)), rb_want)


def test_a4_endpoint_bitmap_clustered_endpoints(R):
    """Endpoints crowded into a few thousand positions (many marks per bit
    word, most contracted segments empty of interior cells) plus a few spread
    out: P, ranks and answers match the oracle."""
    n, q = 1_000_000, 100_000
    rng = np.random.default_rng(77)
    a = rng.integers(0, 3000, size=(q, 2))
    l, r = a.min(axis=1).astype(np.int32), a.max(axis=1).astype(np.int32)
    l[:50] = rng.integers(0, n, size=50)         # a few elsewhere
    r[:50] = np.maximum(l[:50], rng.integers(0, n, size=50)).astype(np.int32)
    nbp = -(-n // 32) + 1
    BP = torch.full((2 * nbp,), -1, dtype=torch.int32, device=DEV)
    m = torch.zeros(1, dtype=torch.int64, device=DEV)
    R.rmq_endpoint_bitmap(dev(l), dev(r), n, BP, m)
    torch.cuda.synchronize()
    bp = BP.cpu().numpy()
    wp, wt = oracle.sort_endpoints(l, r)
    P_want, ra_want, rb_want = oracle.rank_endpoints(wp, wt, q)
    bits = np.unpackbits(np.ascontiguousarray(bp[:nbp]).view(np.uint8), bitorder="little")
    assert np.array_equal(np.nonzero(bits)[0].astype(np.uint32), P_want)
    assert int(m.item()) == len(P_want)
    assert np.array_equal(bitmap_ranks_host(bp, l.astype(np.int64)), ra_want)
    assert np.array_equal(bitmap_ranks_host(bp, r.astype(np.int64)), rb_want)
    A = W.uniform_array(n, 78)
    check(R, A, l, r, want=oracle.rmq_sparse_table(A, l, r), variants=(R.Variant.CONTRACTED,), kcons=(0, 32))


@pytest.mark.parametrize("case", ["ragged_unaligned_invalid", "full_span", "many_buckets"])
def test_a4_endpoint_bitmap_large_batch_edges(R, case):
    """Larger batches at the edges of the marking: a batch that is no
    multiple of 4096 queries, l and r not 16-byte aligned, invalid queries
    (they mark position 0), every query the whole array (all endpoints on
    two positions), and an array of 2^27 + 3 cells.  P, the ranks and m
    equal the oracle's, and so do the contracted answers."""
    if case == "ragged_unaligned_invalid":
        n, q = 65536 * 5 + 3, 65536 + 4097 + 3
        l, r = W.uniform_queries(n, q, 501)
        l[:4], r[:4] = [9, -1, 0, 5], [3, 4, n, n - 1]
    elif case == "full_span":
        n, q = 1_000_000, 100_000
        l, r = np.zeros(q, np.int32), np.full(q, n - 1, np.int32)
    else:
        n, q = 2**27 + 3, 70_000
        l, r = W.uniform_queries(n, q, 502)
    nbp = -(-n // 32) + 1
    BP = torch.full((2 * nbp,), -1, dtype=torch.int32, device=DEV)
    m = torch.zeros(1, dtype=torch.int64, device=DEV)
    bl = torch.zeros(q + 1, dtype=torch.int32, device=DEV)
    br = torch.zeros(q + 1, dtype=torch.int32, device=DEV)
    bl[1:], br[1:] = dev(l), dev(r)                     # offset by one cell: not 16-byte aligned
    R.rmq_endpoint_bitmap(bl[1:], br[1:], n, BP, m)
    torch.cuda.synchronize()
    valid = (l >= 0) & (r >= l) & (r < n)
    assert R.rmq_stream_status() == (R.Status.OK if valid.all() else R.Status.ERR_QUERY_RANGE)
    wl, wr = np.where(valid, l, 0).astype(np.int32), np.where(valid, r, 0).astype(np.int32)
    bp = BP.cpu().numpy()
    wp, wt = oracle.sort_endpoints(wl, wr)
    P_want, ra_want, rb_want = oracle.rank_endpoints(wp, wt, q)
    bits = np.unpackbits(np.ascontiguousarray(bp[:nbp]).view(np.uint8), bitorder="little")
    assert np.array_equal(np.nonzero(bits)[0].astype(np.uint32), P_want)
    assert int(m.item()) == len(P_want) and bp[-1] == len(P_want) and bp[nbp - 1] == 0
    assert np.array_equal(bitmap_ranks_host(bp, wl.astype(np.int64)), ra_want)
    assert np.array_equal(bitmap_ranks_host(bp, wr.astype(np.int64)), rb_want)
    if n <= 1_000_000:
        A = W.uniform_array(n, 503, 0, 50)
        check(R, A, l, r, variants=(R.Variant.CONTRACTED,), kcons=(0, 64), offsets=(0, 1))


def test_a4_endpoint_bitmap_invalid_queries_mark_zero(R):
    n, q = 10_000, 300
    l, r = W.uniform_queries(n, q, 99)
    l[5], r[5] = 7, 3            # l > r
    r[9] = n                     # r out of range
    nbp = -(-n // 32) + 1
    BP = torch.zeros(2 * nbp, dtype=torch.int32, device=DEV)
    m = torch.zeros(1, dtype=torch.int64, device=DEV)
    R.rmq_endpoint_bitmap(dev(l), dev(r), n, BP, m)
    torch.cuda.synchronize()
    assert R.rmq_stream_status() == R.Status.ERR_QUERY_RANGE
    wl, wr = l.copy(), r.copy()
    wl[[5, 9]] = 0
    wr[[5, 9]] = 0
    P_want = np.unique(np.concatenate([wl, wr])).astype(np.uint32)
    bits = np.unpackbits(np.ascontiguousarray(BP.cpu().numpy()[:nbp]).view(np.uint8), bitorder="little")
    assert np.array_equal(np.nonzero(bits)[0].astype(np.uint32), P_want)
    assert int(m.item()) == len(P_want)


@pytest.mark.parametrize("n,q,hi", [(5, 2, 3), (1000, 1, 5), (5000, 3, 5), (100_000, 50_000, 1000),
                                    (3000, 10_000, 5), (70_000, 1, 2**31),
                                    (1_000_003, 2_000, 2**31), (1_000_003, 300_000, 3),
                                    (2_000_000, 20, 2**31)])
@pytest.mark.parametrize("offset", [0, 1])
def test_a6_contract(R, n, q, hi, offset):
    A = W.uniform_array(n, n + q, 0, hi)
    l, r = W.uniform_queries(n, q, n + q + 1)
    P = np.unique(np.concatenate([l, r])).astype(np.uint32)
    m = len(P)
    want = oracle.contract(A, P)
    buf = torch.zeros(n + offset, dtype=torch.int32, device=DEV)
    buf[offset:] = dev(A)
    AQ = torch.zeros(max(m - 1, 1), dtype=torch.int64, device=DEV)
    mdev = torch.tensor([m], dtype=torch.int64, device=DEV)
    R.rmq_contract(buf[offset:], dev(P.view(np.int32)), mdev, m, AQ)
    torch.cuda.synchronize()
    assert np.array_equal(keys_pos(AQ)[: m - 1], want)


# ------------------------------------------------------------------ handles, host API

def test_resident_handle(R):
    n = 500_000
    A = W.uniform_array(n, 51, 0, 1000)
    dA = dev(A)
    for k in (32, 1024, 65536):
        h = R.rmq_build(dA, k=k)
        assert h.k == k and 0 < h.bytes <= R.rmq_table_bytes(n, k) + 8 * 4096
        for seed in (52, 53):
            l, r = W.uniform_queries(n, 20_000, seed)
            out = torch.zeros(len(l), dtype=torch.int32, device=DEV)
            R.rmq_query(h, dev(l), dev(r), out)
            assert np.array_equal(out.cpu().numpy(), oracle.rmq_naive(A, l, r))
        h.free()


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_host_buffers(R, variant):
    n = 200_001
    A = W.uniform_array(n, 54, 0, 5000)
    l, r = W.uniform_queries(n, 30_001, 55)
    out = np.zeros(len(l), dtype=np.int32)
    R.rmq_batch_host(A, l, r, out, variant=variant)
    assert np.array_equal(out, oracle.rmq_naive(A, l, r))


def test_metamorphic_k_and_form_do_not_change_answers(R):
    n = 400_000
    A = W.paper_permutation(n, 56)
    l, r = W.uniform_queries(n, 40_000, 57)
    ref = None
    for v in (R.Variant.PLAIN, R.Variant.CONTRACTED, R.Variant.AUTO):
        for k in (32, 128, 1024, 8192):
            got, st = run_batch(R, A, l, r, v, k, min(k, 4096))
            assert st == R.Status.OK
            if ref is None:
                ref = got
            assert np.array_equal(got, ref), (v, k)
    assert np.array_equal(ref, oracle.rmq_sparse_table(A, l, r))


@pytest.mark.parametrize("offset", [0, 1])
def test_a6_contract_dense_and_sparse_tiles(R, offset):
    """Tiles of 1024 cells whose marks exceed the warp's 512 slots (every cell
    an endpoint; exactly 512 and 513 marks) next to sparse tiles, with ties:
    A_Q matches the oracle's contraction entry by entry."""
    n = 300_000
    A = W.uniform_array(n, 903, 0, 7)
    parts = [np.arange(100_000, 103_072),                     # three whole tiles, every cell marked
             np.arange(200_704, 200_704 + 512),               # one tile with exactly 512 marks
             np.arange(204_800, 204_800 + 513),               # one tile with 513 marks
             np.arange(0, n, 700)]                            # sparse marks elsewhere
    P = np.unique(np.concatenate(parts)).astype(np.uint32)
    m = len(P)
    want = oracle.contract(A, P)
    buf = torch.zeros(n + offset, dtype=torch.int32, device=DEV)
    buf[offset:] = dev(A)
    AQ = torch.zeros(m - 1, dtype=torch.int64, device=DEV)
    mdev = torch.tensor([m], dtype=torch.int64, device=DEV)
    R.rmq_contract(buf[offset:], dev(P.view(np.int32)), mdev, m, AQ)
    torch.cuda.synchronize()
    assert np.array_equal(keys_pos(AQ), want)
    # the same marks as query endpoints through the whole contracted batch
    l, r = P[:-1].astype(np.int32), P[1:].astype(np.int32)
    check(R, A, l, r, want=oracle.rmq_sparse_table(A, l, r), variants=(R.Variant.CONTRACTED,), kcons=(32, 256))


@pytest.mark.parametrize("nb,k", [(3001, 128), (6007, 256), (12001, 128), (25013, 512), (50021, 128),
                                  (100003, 128), (2041, 1024), (130_000, 256)])
def test_coarse_shifts_three_to_eight(R, nb, k):
    """Plain batches whose coarse blocks hold 2^3 .. 2^8 blocks (up to 508
    coarse blocks), with a short last block, ties, uniform and short queries,
    aligned and unaligned arrays: answers match the oracle."""
    n = (nb - 1) * k + 1 + (nb * 7) % (k - 1)
    A = W.uniform_array(n, nb + k, 0, 50)
    l, r = W.uniform_queries(n, 20_000, nb + 1)
    l[:5000], r[:5000] = W.log_width_queries(n, 5000, nb + 2, 1, 4 * k)
    l[5000], r[5000] = 0, n - 1
    l[5001], r[5001] = n - 1, n - 1
    check(R, A, l, r, want=oracle.rmq_sparse_table(A, l, r), variants=(R.Variant.PLAIN,), ks=(k,), offsets=(0, 1))


@pytest.mark.parametrize("k,k1", [(64, 32), (128, 32), (128, 64), (256, 32), (256, 128), (1024, 32), (1024, 64),
                                  (1024, 256), (1024, 512), (4096, 256), (4096, 4096), (64, 64), (1024, -1)])
@pytest.mark.parametrize("hi", [1000, 2**31])
def test_small_blocks_k1(R, k, k1, hi):
    """The two-level layout with small blocks of k1 cells (Sec. 3.3), from
    k1 = 32 to k1 = k and without small blocks: tie-heavy short ranges,
    uniform ranges, a short last block and unaligned arrays; answers match the
    oracle, and the instrumented kernel reads small-block minima exactly when
    k1 is in use."""
    n = 777_777 + k // 3
    A = W.uniform_array(n, k + k1 + hi % 7, 0, hi)
    l, r = W.log_width_queries(n, 40_000, k + 1, 1, 4 * k)
    l[:8000], r[:8000] = W.uniform_queries(n, 8000, k + 2)
    l[8000], r[8000] = 0, n - 1
    for off in (0, 1):
        got, st = run_batch_k1(R, A, l, r, k, k1, off)
        assert st == R.Status.OK
        assert np.array_equal(got, oracle.rmq_sparse_table(A, l, r)), (k, k1, off)
    dA, dl, dr = dev(A), dev(l), dev(r)
    out = torch.empty(len(l), dtype=torch.int32, device=DEV)
    cnt = R.rmq_batch_counted(dA, dl, dr, out, variant=1, k=k, k1=k1)
    assert (cnt["m1_reads"] > 0) == (k1 > 0), cnt


def run_batch_k1(R, A, l, r, k, k1, offset):
    n, q = len(A), len(l)
    bufA = torch.zeros(n + offset, dtype=torch.int32, device=DEV)
    bufA[offset:] = dev(A)
    bl = torch.zeros(q + offset, dtype=torch.int32, device=DEV)
    br = torch.zeros(q + offset, dtype=torch.int32, device=DEV)
    bo = torch.full((q + offset,), -7, dtype=torch.int32, device=DEV)
    bl[offset:], br[offset:] = dev(l), dev(r)
    R.rmq_batch_ex(bufA[offset:], bl[offset:], br[offset:], bo[offset:], variant=1, k=k, k1=k1)
    return bo[offset:].cpu().numpy(), R.rmq_stream_status()
