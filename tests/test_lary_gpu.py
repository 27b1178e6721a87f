"""GPU parity of the l-ary block sparse table (the Sec. 3.1 variant) through
the C ABI: the same answers as the naive oracle and as the oracle's l-ary
query, for several block sizes and arities, uniform and short queries,
ties, extreme values and invalid queries."""
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


def run(R, A, l, r, k, ell):
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dl = torch.from_numpy(np.ascontiguousarray(l)).cuda()
    dr = torch.from_numpy(np.ascontiguousarray(r)).cuda()
    out = torch.full((len(l),), -7, dtype=torch.int32, device="cuda")
    R.rmq_batch_lary(dA, dl, dr, out, k=k, ell=ell)
    st = R.rmq_stream_status()
    return out.cpu().numpy(), st


@pytest.mark.parametrize("n,hi", [(1, 9), (1000, 3), (70_001, 2**31), (300_000, 1000)])
@pytest.mark.parametrize("k,ell", [(32, 2), (32, 16), (64, 4), (1024, 8), (4096, 256)])
def test_lary_matches_oracle(R, n, hi, k, ell):
    A = W.uniform_array(n, n + k + ell, 0, hi)
    l, r = W.uniform_queries(n, 3000, n + 1)
    ls, rs = W.log_width_queries(n, 2000, n + 2, 1, 5000)
    l, r = np.concatenate([l, ls, [0, n - 1]]).astype(np.int32), np.concatenate([r, rs, [n - 1, n - 1]]).astype(np.int32)
    got, st = run(R, A, l, r, k, ell)
    want = oracle.rmq_naive(A, l, r)
    assert np.array_equal(got, want), (n, k, ell, int(np.sum(got != want)))
    assert np.array_equal(got, oracle.lary_query(A, k, ell, l, r)[0])
    assert st == R.Status.OK


def test_lary_extreme_values_and_invalid_queries(R):
    n = 50_000
    A = W.uniform_array(n, 9, 0, 4).astype(np.int64)
    A = np.where(A == 0, -2**31, np.where(A == 3, 2**31 - 1, A)).astype(np.int32)
    l, r = W.uniform_queries(n, 4000, 10)
    l[:3], r[:3] = [5, -1, 10], [4, 3, n]   # l > r, l < 0, r >= n
    got, st = run(R, A, l, r, 64, 16)
    want = oracle.rmq_naive(A, l, r)
    assert np.array_equal(got, want)
    assert (got[:3] == -1).all() and st == R.Status.ERR_QUERY_RANGE


def test_lary_rejects_bad_arguments(R):
    A = torch.zeros(100, dtype=torch.int32, device="cuda")
    l = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    for k, ell in ((48, 2), (32, 3), (32, 1), (32, 512), (16, 2)):
        with pytest.raises(R.RmqError):
            R.rmq_batch_lary(A, l, l, out, k=k, ell=ell)
