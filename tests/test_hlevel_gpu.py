"""GPU parity of the multi-level block sparse table (Sec. 3.3) through the C
ABI: the same answers as the oracle's multi-level query and the naive scan,
for one to four levels, uniform, short and aligned queries, ties, extreme
values, an unaligned array, invalid queries and the paper's block sizes on
the n = 1e8 workloads."""
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


def run(R, A, l, r, ks, dA=None):
    if dA is None:
        dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dl = torch.from_numpy(np.ascontiguousarray(l)).cuda()
    dr = torch.from_numpy(np.ascontiguousarray(r)).cuda()
    out = torch.full((len(l),), -7, dtype=torch.int32, device="cuda")
    R.rmq_batch_hlevel(dA, dl, dr, out, ks)
    st = R.rmq_stream_status()
    return out.cpu().numpy(), st


def mixed_queries(n, ks, seed):
    """Uniform ranges, short ranges around k_1 .. k_h, single cells, and
    ranges whose ends fall on block boundaries of every level."""
    l, r = W.uniform_queries(n, 3000, seed)
    ls, rs = W.log_width_queries(n, 3000, seed + 1, 1, max(2, min(n, 4 * ks[-1])))
    g = W.rng(seed + 2)
    c = g.integers(0, n, 500).astype(np.int32)
    la, ra = [], []
    for k in ks:
        if k > n:
            continue
        nb = n // k
        a = g.integers(0, max(1, nb), 300) * k
        b = np.minimum(n - 1, a + g.integers(1, 6, 300) * k - 1 - g.integers(0, 2, 300))
        la.append(a), ra.append(np.maximum(a, b))
    parts_l = [l, ls, c] + la
    parts_r = [r, rs, c] + ra
    return (np.concatenate(parts_l).astype(np.int32), np.concatenate(parts_r).astype(np.int32))


KS = [(32,), (64, 512), (32, 128, 1024), (128, 1024, 16384), (32, 64, 128, 256), (256, 1 << 20)]


@pytest.mark.parametrize("n,hi", [(1, 9), (777, 3), (70_001, 2**31), (300_001, 20), (1 << 20, 1000)])
@pytest.mark.parametrize("ks", KS)
def test_hlevel_matches_oracle(R, n, hi, ks):
    A = W.uniform_array(n, n + sum(ks), 0, hi)
    l, r = mixed_queries(n, ks, n + len(ks))
    got, st = run(R, A, l, r, ks)
    want, _ = oracle.hlevel_query(A, ks, l, r)
    assert np.array_equal(want, oracle.rmq_naive(A, l, r))
    assert st == R.Status.OK
    assert np.array_equal(got, want)


def test_hlevel_every_range_of_a_small_array(R):
    """All n (n + 1) / 2 ranges of an array spanning several blocks of every
    level, with a ragged last block and many ties."""
    n = 1000
    A = W.uniform_array(n, 41, 0, 6)
    i, j = np.triu_indices(n)
    l, r = i.astype(np.int32), j.astype(np.int32)
    for ks in ((32, 64, 256), (64, 128)):
        got, st = run(R, A, l, r, ks)
        assert st == R.Status.OK
        assert np.array_equal(got, oracle.rmq_naive(A, l, r)), ks


def test_hlevel_extreme_values_invalid_queries_and_unaligned_array(R):
    n = 200_003
    A = W.uniform_array(n + 1, 9, 0, 4).astype(np.int64)
    A = np.where(A == 0, -2**31, np.where(A == 3, 2**31 - 1, A)).astype(np.int32)
    ks = (32, 256, 4096)
    l, r = mixed_queries(n, ks, 12)
    l[:4], r[:4] = [5, -1, 10, 0], [4, 3, n, n - 1]   # l > r, l < 0, r >= n, the whole array
    dfull = torch.from_numpy(A).cuda()
    for off in (0, 1):                                 # off = 1: A not 16-byte aligned
        Av = A[off:off + n]
        got, st = run(R, Av, l, r, ks, dA=dfull[off:off + n])
        want = oracle.rmq_naive(Av, l, r)
        assert np.array_equal(got, want), off
        assert (got[:3] == -1).all() and st == R.Status.ERR_QUERY_RANGE
    got, st = run(R, A[:n], l[3:], r[3:], ks)
    assert st == R.Status.OK


def test_hlevel_empty_batch_and_one_block(R):
    A = W.uniform_array(5000, 3)
    dA = torch.from_numpy(A).cuda()
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    R.rmq_batch_hlevel(dA, e, e, e, (32, 64))
    assert R.rmq_stream_status() == R.Status.OK
    l, r = W.uniform_queries(5000, 2000, 4)
    got, st = run(R, A, l, r, (8192, 1 << 16))       # every level one block
    assert st == R.Status.OK and np.array_equal(got, oracle.rmq_naive(A, l, r))


def test_hlevel_rejects_bad_block_sizes(R):
    A = torch.zeros(100, dtype=torch.int32, device="cuda")
    l = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    for ks in ((48,), (16, 32), (64, 64), (128, 64), (1 << 17,)):
        with pytest.raises(R.RmqError):
            R.rmq_batch_hlevel(A, l, l, out, ks)


@pytest.mark.parametrize("workload", ["uniform", "tie_heavy_short"])
@pytest.mark.parametrize("h", [2, 3])
def test_hlevel_paper_ks_at_n_1e8(R, workload, h):
    """The n = 1e8, q = 1e7 workloads with Sec. 3.3's block sizes: a sample
    of 2000 answers against the naive scan, and every answer equal to the
    plain form's (rmq_batch_ex, itself checked against the oracle)."""
    n, q = 10**8, 10**7
    ks = R.rmq_hlevel_paper_ks(n, h)
    if workload == "uniform":
        A = W.uniform_array(n, 1)
        l, r = W.uniform_queries(n, q, 2)
    else:
        A = W.uniform_array(n, 3, 0, 1000)
        l, r = W.log_width_queries(n, q, 4, 1, 10_000)
    dA = torch.from_numpy(A).cuda()
    dl, dr = torch.from_numpy(l).cuda(), torch.from_numpy(r).cuda()
    out = torch.full((q,), -7, dtype=torch.int32, device="cuda")
    R.rmq_batch_hlevel(dA, dl, dr, out, ks)
    assert R.rmq_stream_status() == R.Status.OK
    ref = torch.full((q,), -9, dtype=torch.int32, device="cuda")
    R.rmq_batch_ex(dA, dl, dr, ref, variant=1, k=512)
    assert R.rmq_stream_status() == R.Status.OK
    assert torch.equal(out, ref)
    idx = W.rng(5).choice(q, 2000, replace=False)
    got = out.cpu().numpy()[idx]
    assert np.array_equal(got, oracle.rmq_naive(A, l[idx], r[idx]))
