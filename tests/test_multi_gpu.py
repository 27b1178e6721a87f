"""rmq_batch_multi: many arrays of uneven n with uneven q in one persistent
launch, checked array by array against the CPU oracle (exact)."""
import numpy as np
import pytest

import oracle
from paper_1706_06940_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1706_06940_gb300 import rmq
    return rmq


def make_batch(ns, qs, seed, hi=2**31, width=None):
    arrays, ls, rs = [], [], []
    for h, (n, q) in enumerate(zip(ns, qs)):
        A = W.uniform_array(max(n, 1), seed + 3 * h, 0, hi)[:n]
        if width is None:
            l, r = W.uniform_queries(max(n, 1), q, seed + 3 * h + 1)
        else:
            l, r = W.log_width_queries(max(n, 1), q, seed + 3 * h + 1, 1, width)
        arrays.append(A)
        ls.append(l)
        rs.append(r)
    return arrays, ls, rs


def run_multi(R, arrays, ls, rs, offset=0, **kw):
    dA = []
    for A in arrays:
        buf = torch.zeros(len(A) + offset, dtype=torch.int32, device=DEV)
        if len(A):
            buf[offset:] = torch.from_numpy(A).to(DEV)
        dA.append(buf[offset:])
    L = torch.from_numpy(np.concatenate(ls) if ls else np.zeros(0, np.int32)).to(DEV)
    Rr = torch.from_numpy(np.concatenate(rs) if rs else np.zeros(0, np.int32)).to(DEV)
    out = torch.full((len(L),), -7, dtype=torch.int32, device=DEV)
    R.rmq_batch_multi(dA, [len(l) for l in ls], L, Rr, out, **kw)
    st = R.rmq_stream_status()
    return out.cpu().numpy(), st


def expected(arrays, ls, rs, naive_limit=300_000):
    outs = []
    for A, l, r in zip(arrays, ls, rs):
        if len(l) == 0:
            outs.append(np.zeros(0, np.int32))
        elif len(A) <= naive_limit:
            outs.append(oracle.rmq_naive(A, l, r))
        else:
            outs.append(oracle.rmq_sparse_table(A, l, r))
    return np.concatenate(outs) if outs else np.zeros(0, np.int32)


@pytest.mark.parametrize("offset", [0, 1])
def test_mixed_small_arrays(R, offset):
    rng = np.random.default_rng(7)
    ns = [1, 2, 31, 32, 33, 1000, 4097, 100_000, 65_536, 250_001] + list(rng.integers(1, 50_000, 20))
    qs = [5, 0, 100, 33, 1, 3000, 1025, 5000, 2048, 777] + list(rng.integers(0, 3000, 20))
    arrays, ls, rs = make_batch(ns, qs, 100, hi=50)
    got, st = run_multi(R, arrays, ls, rs, offset)
    assert st == R.Status.OK
    assert np.array_equal(got, expected(arrays, ls, rs))


def test_forced_k_and_short_ranges(R):
    ns = [10_000, 200_000, 1_000_003]
    qs = [4000, 4000, 4000]
    arrays, ls, rs = make_batch(ns, qs, 200, hi=3, width=3000)
    want = expected(arrays, ls, rs)
    for k in (32, 256, 4096):
        got, st = run_multi(R, arrays, ls, rs, k=k)
        assert st == R.Status.OK and np.array_equal(got, want), k


def test_invalid_queries_and_empty_batch(R):
    arrays, ls, rs = make_batch([1000, 500], [10, 10], 300)
    ls[1][3], rs[1][3] = 400, 600                       # r >= n of its own array
    ls[0][5], rs[0][5] = 9, 8                           # l > r
    got, st = run_multi(R, arrays, ls, rs)
    assert st == R.Status.ERR_QUERY_RANGE
    want = expected(arrays, [np.clip(l, 0, len(a) - 1) for a, l in zip(arrays, ls)],
                    [np.clip(r, 0, len(a) - 1) for a, r in zip(arrays, rs)])
    want[5], want[13] = -1, -1
    assert np.array_equal(got, want)
    got, st = run_multi(R, [np.zeros(5, np.int32)], [np.zeros(0, np.int32)], [np.zeros(0, np.int32)])
    assert st == R.Status.OK and len(got) == 0


def test_withheld_ready_flag_times_out_and_context_survives(R):
    """Test hook: array 0's table is never marked ready; its queries give up
    after a short bounded wait (answers -1, RMQ_ERR_TIMEOUT), the others are
    answered, and the next call works normally."""
    arrays, ls, rs = make_batch([50_000, 70_000, 3000], [2000, 3000, 100], 400)
    got, st = run_multi(R, arrays, ls, rs, flags=R.FLAG_TEST_WITHHOLD_READY)
    assert st == R.Status.ERR_TIMEOUT
    want = expected(arrays, ls, rs)
    assert (got[:2000] == -1).all()
    assert np.array_equal(got[2000:], want[2000:])
    got, st = run_multi(R, arrays, ls, rs)
    assert st == R.Status.OK and np.array_equal(got, want)


def test_graph_capture_and_replay(R):
    arrays, ls, rs = make_batch([100_000, 30_000, 777], [5000, 100, 50], 500)
    want = expected(arrays, ls, rs)
    dA = [torch.from_numpy(A).to(DEV) for A in arrays]
    L = torch.from_numpy(np.concatenate(ls)).to(DEV)
    Rr = torch.from_numpy(np.concatenate(rs)).to(DEV)
    out = torch.full((len(L),), -7, dtype=torch.int32, device=DEV)
    qs = [len(l) for l in ls]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        R.rmq_batch_multi(dA, qs, L, Rr, out)            # first call outside capture: one-time set-up
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        R.rmq_batch_multi(dA, qs, L, Rr, out, stream=s.cuda_stream)
    for _ in range(2):
        out.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want)


def test_config4_512_uneven_arrays(R):
    ns, qs = W.uneven_batch(512, 1004)
    arrays, ls, rs = make_batch(list(ns), list(qs), 600)
    got, st = run_multi(R, arrays, ls, rs)
    assert st == R.Status.OK
    assert np.array_equal(got, expected(arrays, ls, rs))
