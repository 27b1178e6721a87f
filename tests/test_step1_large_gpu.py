"""GPU parity of step 1 of BbST_CON (Sec. 3.1) at batch sizes beyond the
edge cases of the step tests: the endpoint bitmap and its rank counts for
2.6e5 to 6e5 queries over arrays of 1e6 to 2^29 positions, endpoints crowded
into one 2^18-position range (many queries sharing ends), full-span and
invalid queries, and the contracted answers on such batches, all against
the oracle's sort, ranks and sparse table."""
import numpy as np
import pytest

import oracle
from paper_1706_06940_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
QMIN = 1 << 18


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1706_06940_gb300 import rmq
    return rmq


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def popcount32(x):
    """Bits set in each uint32 (SWAR, vectorised)."""
    x = x.astype(np.uint64)
    x = x - ((x >> 1) & 0x55555555)
    x = (x & 0x33333333) + ((x >> 2) & 0x33333333)
    x = (x + (x >> 4)) & 0x0F0F0F0F
    return ((x * 0x01010101) & 0xFFFFFFFF) >> 24


def bitmap_ranks(bp, pos):
    half = len(bp) // 2
    w = bp[:half].view(np.uint32)
    c = bp[half:].view(np.uint32).astype(np.int64)
    idx = pos >> 5
    below = w[idx] & ((np.uint32(1) << (pos & 31).astype(np.uint32)) - np.uint32(1))
    return c[idx] + popcount32(below).astype(np.int64)


def check_bitmap(R, n, l, r):
    q = len(l)
    nbp = -(-n // 32) + 1
    BP = torch.full((2 * nbp,), -1, dtype=torch.int32, device=DEV)
    m = torch.zeros(1, dtype=torch.int64, device=DEV)
    R.rmq_endpoint_bitmap(dev(l), dev(r), n, BP, m)
    torch.cuda.synchronize()
    st = R.rmq_stream_status()
    bp = BP.cpu().numpy()
    # an invalid query takes part in step 1 as the pair (0, 0)
    ok = (l >= 0) & (r >= l) & (r < n)
    lq = np.where(ok, l, 0).astype(np.int64)
    rq = np.where(ok, r, 0).astype(np.int64)
    wp, wt = oracle.sort_endpoints(lq, rq)
    P_want, ra_want, rb_want = oracle.rank_endpoints(wp, wt, q)
    words = bp[:nbp].view(np.uint32)
    nz = np.nonzero(words)[0]
    bits = np.unpackbits(np.ascontiguousarray(words[nz]).view(np.uint8), bitorder="little").reshape(-1, 32)
    wi, bi = np.nonzero(bits)
    assert np.array_equal((nz[wi].astype(np.int64) * 32 + bi).astype(np.uint32), P_want)
    assert int(m.item()) == len(P_want) and bp[-1] == len(P_want) and bp[nbp - 1] == 0
    assert np.array_equal(bitmap_ranks(bp, lq), ra_want)
    assert np.array_equal(bitmap_ranks(bp, rq), rb_want)
    return st


# n from 1e6 + 3 to 2^29 - 5 (a multiple of 2^18 among them); q ragged
@pytest.mark.parametrize("n,q", [(1_000_003, QMIN), (5 * 2**18, QMIN + 4099),
                                 (3 * 2**18 + 7, 300_001), (2**27 + 3, 400_000), (2**29 - 5, 270_000)])
def test_bitmap_matches_oracle(R, n, q):
    l, r = W.uniform_queries(n, q, 5 * q + n)
    l[: q // 8] = r[: q // 8]          # single-cell queries: a shared endpoint
    st = check_bitmap(R, n, l, r)
    assert st == R.Status.OK


def test_bitmap_invalid_queries(R):
    """Invalid queries take part as (0, 0) and raise the error word."""
    n, q = 2_000_000, 300_000
    l, r = W.uniform_queries(n, q, 901)
    l[7], r[7] = 5, 4          # l > r
    l[99], r[99] = -1, 10      # l < 0
    r[4321] = n                # r >= n
    st = check_bitmap(R, n, l, r)
    assert st == R.Status.ERR_QUERY_RANGE


def test_bitmap_crowded_endpoints(R):
    """All but 1000 endpoints on 300 positions (many marks of one word)."""
    n, q = 4_000_000, 600_000
    rng = np.random.default_rng(31)
    a = rng.integers(2**18 + 1000, 2**18 + 1300, size=(q, 2))
    l, r = a.min(axis=1).astype(np.int32), a.max(axis=1).astype(np.int32)
    l[:1000] = rng.integers(0, n, size=1000)
    r[:1000] = np.maximum(l[:1000], rng.integers(0, n, size=1000)).astype(np.int32)
    assert check_bitmap(R, n, l, r) == R.Status.OK


def answers(R, A, l, r, offset=0, k_con=0):
    n, q = len(A), len(l)
    bA = torch.zeros(n + offset, dtype=torch.int32, device=DEV)
    bA[offset:] = dev(A)
    bl = torch.zeros(q + offset, dtype=torch.int32, device=DEV)
    br = torch.zeros(q + offset, dtype=torch.int32, device=DEV)
    bo = torch.full((q + offset,), -7, dtype=torch.int32, device=DEV)
    bl[offset:], br[offset:] = dev(l), dev(r)
    R.rmq_batch_ex(bA[offset:], bl[offset:], br[offset:], bo[offset:], variant=R.Variant.CONTRACTED, k_con=k_con)
    st = R.rmq_stream_status()
    return bo[offset:].cpu().numpy(), st


def check_answers(R, A, l, r, offsets=(0,), k_con=0):
    want = oracle.rmq_sparse_table(A, l, r)
    for off in offsets:
        got, st = answers(R, A, l, r, off, k_con)
        bad = np.nonzero(got != want)[0]
        assert len(bad) == 0, (off, len(bad), bad[:5], got[bad[:5]], want[bad[:5]])
        assert st == (R.Status.ERR_QUERY_RANGE if (want < 0).any() else R.Status.OK), st


def test_contracted_uniform_batch(R):
    """Uniform array and queries; aligned and unaligned l, r."""
    n, q = 3_000_017, 300_007
    A = W.uniform_array(n, 41)
    l, r = W.uniform_queries(n, q, 42)
    check_answers(R, A, l, r, offsets=(0, 1))


def test_contracted_short_ties(R):
    """Few distinct values and short ranges (many shared and neighbouring
    endpoints, edge scans on A_Q)."""
    n, q = 2_500_000, 400_000
    A = W.uniform_array(n, 43, 0, 50)
    l, r = W.log_width_queries(n, q, 44, 1, 3000)
    check_answers(R, A, l, r, k_con=64)


def test_contracted_crowded_and_full_span(R):
    """A quarter of the queries span the whole array, half sit in a window
    of 200 positions, the rest are uniform; plus invalid queries."""
    n, q = 1_500_000, 280_000
    A = W.uniform_array(n, 45)
    l, r = W.uniform_queries(n, q, 46)
    rng = np.random.default_rng(47)
    l[: q // 4], r[: q // 4] = 0, n - 1
    a = rng.integers(700_000, 700_200, size=(q // 2, 2))
    l[q // 4: q // 4 + q // 2] = a.min(axis=1)
    r[q // 4: q // 4 + q // 2] = a.max(axis=1)
    l[5], r[5] = 9, 3
    r[77] = n + 5
    check_answers(R, A, l, r)
