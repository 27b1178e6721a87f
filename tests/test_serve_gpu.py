"""The continuous-batching server: admission by memory budget, requests of
very different sizes from several threads while earlier batches run, and
every request's answers identical alone (rmq_query on the same handle) and
in the mix, and equal to the oracle."""
import threading

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


def test_results_same_alone_and_in_the_mix(R):
    ns = [3_000_000, 700_001, 20_000]
    arrays = [W.uniform_array(n, 70 + i, 0, 1000 if i == 1 else 2**31) for i, n in enumerate(ns)]
    dA = [torch.from_numpy(A).to(DEV) for A in arrays]
    srv = R.Server(inflight=3)
    ids = [srv.admit(A) for A in dA]
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(300):
        h = int(rng.integers(0, len(ns)))
        q = int(np.exp(rng.random() * np.log(100_000)))
        if i % 3 == 0:
            l, r = W.log_width_queries(ns[h], q, 1000 + i, 1, 5000)
        else:
            l, r = W.uniform_queries(ns[h], q, 1000 + i)
        reqs.append((h, l, r, np.full(q, -7, dtype=np.int32)))
    tickets = [None] * len(reqs)

    def producer(part):
        for j in range(part, len(reqs), 2):
            h, l, r, out = reqs[j]
            tickets[j] = srv.submit(ids[h], l, r, out)

    th = [threading.Thread(target=producer, args=(p,)) for p in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    lat = [srv.wait(t) for t in tickets]
    assert all(x >= 0 for x in lat)
    st = srv.stats()
    assert st["requests"] == len(reqs) and st["batches"] <= len(reqs)
    handles = [R.rmq_build(A) for A in dA]
    for (h, l, r, out) in reqs:
        alone = torch.empty(len(l), dtype=torch.int32, device=DEV)
        R.rmq_query(handles[h], torch.from_numpy(l).to(DEV), torch.from_numpy(r).to(DEV), alone)
        assert np.array_equal(out, alone.cpu().numpy())
        idx = rng.choice(len(l), min(len(l), 64), replace=False)
        assert np.array_equal(out[idx], oracle.rmq_naive(arrays[h], l[idx], r[idx]))
    for h in handles:
        h.free()
    srv.close()


def test_admission_budget_and_eviction(R):
    A = torch.from_numpy(W.uniform_array(5_000_000, 80)).to(DEV)
    B = torch.from_numpy(W.uniform_array(5_000_000, 81)).to(DEV)
    srv = R.Server(budget_bytes=30_000_000)          # room for one 20 MB array and its tables
    a = srv.admit(A)
    with pytest.raises(R.RmqError) as ei:
        srv.admit(B)
    assert ei.value.status == R.Status.ERR_BUDGET
    l, r = W.uniform_queries(5_000_000, 1000, 82)
    out = np.zeros(1000, np.int32)
    srv.wait(srv.submit(a, l, r, out))
    srv.evict(a)
    b = srv.admit(B)
    out2 = np.zeros(1000, np.int32)
    srv.wait(srv.submit(b, l, r, out2))
    assert np.array_equal(out2, oracle.rmq_naive(B.cpu().numpy(), l, r))
    with pytest.raises(R.RmqError):
        srv.submit(a, l, r, out)                      # evicted id
    srv.close()


def test_query_multi_over_handles(R):
    arrays = [W.uniform_array(n, 90 + n % 7, 0, 50) for n in (100_000, 1, 64, 333_333)]
    dA = [torch.from_numpy(A).to(DEV) for A in arrays]
    hs = [R.rmq_build(A) for A in dA]
    reqs = [(0, 500), (3, 70_000), (1, 3), (0, 1), (2, 0), (3, 5)]
    ls, rs = [], []
    for j, (h, q) in enumerate(reqs):
        l, r = W.uniform_queries(len(arrays[h]), q, 300 + j)
        ls.append(l)
        rs.append(r)
    L = torch.from_numpy(np.concatenate(ls)).to(DEV)
    Rr = torch.from_numpy(np.concatenate(rs)).to(DEV)
    out = torch.full((len(L),), -7, dtype=torch.int32, device=DEV)
    R.rmq_query_multi([hs[h] for h, _ in reqs], [q for _, q in reqs], L, Rr, out)
    got = out.cpu().numpy()
    want = np.concatenate([oracle.rmq_naive(arrays[h], l, r) for (h, _), l, r in zip(reqs, ls, rs)])
    assert np.array_equal(got, want)
    assert R.rmq_stream_status() == R.Status.OK
    for h in hs:
        h.free()


def test_evict_waits_for_its_requests_and_refuses_new_ones(R):
    """Two threads submit on two arrays while a third evicts one of them and
    re-admits its data under a new id.  Every accepted request completes with
    the right answers; once evict has begun, submits on the old id are
    refused; when evict returns, every accepted request on that id has its
    answers in its out buffer already."""
    ns = [2_000_000, 1_500_000]
    arrays = [W.uniform_array(n, 400 + i, 0, 1 << 20) for i, n in enumerate(ns)]
    dA = [torch.from_numpy(A).to(DEV) for A in arrays]
    srv = R.Server(inflight=3, max_batch_queries=1 << 16)
    ids = [srv.admit(A) for A in dA]
    rng = np.random.default_rng(11)
    accepted = []          # (array index, id, ticket, l, r, out)
    refused = []
    lock = threading.Lock()
    evict_started = threading.Event()
    evicted_done = []

    def producer(h, count, seed):
        g = np.random.default_rng(seed)
        for j in range(count):
            cur = ids[h]
            q = int(g.integers(1, 5000))
            l, r = W.uniform_queries(ns[h], q, seed * 1000 + j)
            out = np.full(q, -7, np.int32)
            try:
                t = srv.submit(cur, l, r, out)
            except R.RmqError as e:
                assert e.status == R.Status.ERR_INVALID_ARG
                with lock:
                    refused.append(cur)
                continue
            with lock:
                accepted.append((h, cur, t, l, r, out))

    def evictor():
        evict_started.wait()
        old = ids[0]
        srv.evict(old)
        # every request accepted on the old id has completed by now
        with lock:
            mine = [a for a in accepted if a[1] == old]
        evicted_done.append((old, all((a[5] != -7).all() for a in mine), len(mine)))
        ids[0] = srv.admit(dA[0])

    th = [threading.Thread(target=producer, args=(0, 300, 21)), threading.Thread(target=producer, args=(1, 300, 22)),
          threading.Thread(target=evictor)]
    for t in th:
        t.start()
    while True:
        with lock:
            if len(accepted) >= 60:
                break
    evict_started.set()
    for t in th:
        t.join()
    old, complete, n_old = evicted_done[0]
    assert complete and n_old > 0
    assert all(x == old for x in refused)
    for h, _, t, l, r, out in accepted:
        srv.wait(t)
        idx = rng.choice(len(l), min(len(l), 24), replace=False)
        assert np.array_equal(out[idx], oracle.rmq_naive(arrays[h], l[idx], r[idx]))
    with pytest.raises(R.RmqError):
        srv.evict(old)                                   # already gone
    srv.close()


def test_invalid_query_is_reported_for_its_request_only(R):
    n = 100_000
    A = W.uniform_array(n, 501, 0, 100)
    dA = torch.from_numpy(A).to(DEV)
    srv = R.Server(inflight=2)
    a = srv.admit(dA)
    reqs = []
    for j in range(6):
        l, r = W.uniform_queries(n, 300, 510 + j)
        if j == 3:
            l[7], r[7] = 50, 40           # l > r
            l[9], r[9] = 5, n             # r >= n
        reqs.append((l, r, np.full(300, -7, np.int32)))
    tickets = [srv.submit(a, l, r, out) for l, r, out in reqs]
    for j, t in enumerate(tickets):
        l, r, out = reqs[j]
        if j == 3:
            with pytest.raises(R.RmqError) as ei:
                srv.wait(t)
            assert ei.value.status == R.Status.ERR_QUERY_RANGE
            assert out[7] == -1 and out[9] == -1
            ok = np.ones(300, bool)
            ok[[7, 9]] = False
            assert np.array_equal(out[ok], oracle.rmq_naive(A, l[ok], r[ok]))
        else:
            srv.wait(t)
            assert np.array_equal(out, oracle.rmq_naive(A, l, r))
    srv.close()
    # the server's own streams reported the error; the caller's stream is clean
    assert R.rmq_stream_status() == R.Status.OK


def test_admit_wait_gets_memory_freed_by_an_eviction(R):
    A = torch.from_numpy(W.uniform_array(5_000_000, 83)).to(DEV)
    B = torch.from_numpy(W.uniform_array(5_000_000, 84)).to(DEV)
    srv = R.Server(budget_bytes=30_000_000)          # room for one of the two
    a = srv.admit(A)
    with pytest.raises(R.RmqError) as ei:
        srv.admit_wait(B, 0.2)                       # nothing is evicted: times out
    assert ei.value.status == R.Status.ERR_BUDGET
    got = []
    th = threading.Thread(target=lambda: got.append(srv.admit_wait(B, 30.0)))
    th.start()
    srv.evict(a)
    th.join()
    b = got[0]
    l, r = W.uniform_queries(5_000_000, 500, 85)
    out = np.zeros(500, np.int32)
    srv.wait(srv.submit(b, l, r, out))
    assert np.array_equal(out, oracle.rmq_naive(B.cpu().numpy(), l, r))
    srv.close()


def test_second_wait_on_a_ticket_is_refused(R):
    """A ticket is collected once: waiting on it again, or on a ticket never
    issued, returns RMQ_ERR_INVALID_ARG at once instead of blocking."""
    n = 200_000
    A = W.uniform_array(n, 520)
    srv = R.Server(inflight=2)
    a = srv.admit(torch.from_numpy(A).to(DEV))
    l, r = W.uniform_queries(n, 1000, 521)
    out = np.full(1000, -7, np.int32)
    t = srv.submit(a, l, r, out)
    srv.wait(t)
    assert np.array_equal(out, oracle.rmq_naive(A, l, r))
    for bad in (t, t + 1000):
        with pytest.raises(R.RmqError) as ei:
            srv.wait(bad)
        assert ei.value.status == R.Status.ERR_INVALID_ARG
    # the server still serves after the refused waits
    out2 = np.full(1000, -7, np.int32)
    srv.wait(srv.submit(a, l, r, out2))
    assert np.array_equal(out2, out)
    srv.close()
