"""GPU parity at the sizes of the workload configurations.

Every answer is compared with the CPU oracle: the naive scan in full where it
is affordable, otherwise the textbook sparse-table oracle on every query (it
equals the naive oracle on all pinned inputs) plus the naive scan on a random
sample.  Answers are positions, so every comparison is exact.
"""
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


def gpu_answers(R, dA, l, r, variant, k=0, k_con=0):
    dl, dr = torch.from_numpy(l).to(DEV), torch.from_numpy(r).to(DEV)
    out = torch.full((len(l),), -7, dtype=torch.int32, device=DEV)
    R.rmq_batch_ex(dA, dl, dr, out, variant=variant, k=k, k_con=k_con)
    assert R.rmq_stream_status() == R.Status.OK
    return out.cpu().numpy()


def sample_check(A, l, r, got, size, seed):
    idx = np.random.default_rng(seed).choice(len(l), size=min(size, len(l)), replace=False)
    assert np.array_equal(got[idx], oracle.rmq_naive(A, l[idx], r[idx]))


def test_config1_n1e6_q1000_naive_in_full(R):
    n, q = 10**6, 1000
    A = W.uniform_array(n, 1001)
    l, r = W.uniform_queries(n, q, 2001)
    want = oracle.rmq_naive(A, l, r)
    dA = torch.from_numpy(A).to(DEV)
    for v in (R.Variant.AUTO, R.Variant.PLAIN, R.Variant.CONTRACTED):
        assert np.array_equal(gpu_answers(R, dA, l, r, v), want), v


def test_config2_n1e8_q_sweep_both_forms(R):
    n = 10**8
    A = W.uniform_array(n, 1002)
    qs = [10**2, 10**3, 10**4, 10**5, 10**6, 10**7]
    batches = [W.uniform_queries(n, q, 2002 + i) for i, q in enumerate(qs)]
    L = np.concatenate([b[0] for b in batches])
    Rr = np.concatenate([b[1] for b in batches])
    want_all = oracle.rmq_sparse_table(A, L, Rr)          # one table build for the whole sweep
    dA = torch.from_numpy(A).to(DEV)
    off = 0
    for q, (l, r) in zip(qs, batches):
        want = want_all[off:off + q]
        off += q
        for v in (R.Variant.PLAIN, R.Variant.CONTRACTED):
            got = gpu_answers(R, dA, l, r, v)
            bad = np.nonzero(got != want)[0]
            assert len(bad) == 0, (q, v.name, len(bad), bad[:5])
        sample_check(A, l, r, got, 48, q)


def test_config2_k_range_plain_and_contracted(R):
    """k over the autotuned range 32..4096 (and beyond) gives the same answers."""
    n, q = 10**8, 10**6
    A = W.uniform_array(n, 1012)
    l, r = W.uniform_queries(n, q, 2012)
    want = oracle.rmq_sparse_table(A, l, r)
    dA = torch.from_numpy(A).to(DEV)
    for k in (32, 256, 4096, 65536):
        assert np.array_equal(gpu_answers(R, dA, l, r, R.Variant.PLAIN, k=k), want), k
    for kc in (32, 512, 4096):
        assert np.array_equal(gpu_answers(R, dA, l, r, R.Variant.CONTRACTED, k_con=kc), want), kc


def test_config3_tie_heavy_short_ranges(R):
    n, q = 10**8, 10**7
    A = W.uniform_array(n, 1003, 0, 1000)
    l, r = W.log_width_queries(n, q, 2003, 1, 10_000)
    want = oracle.rmq_naive(A, l, r)                      # sum of widths ~1.1e10: the naive scan in full
    dA = torch.from_numpy(A).to(DEV)
    for v in (R.Variant.PLAIN, R.Variant.CONTRACTED):
        got = gpu_answers(R, dA, l, r, v)
        bad = np.nonzero(got != want)[0]
        assert len(bad) == 0, (v.name, len(bad), bad[:5])


def test_paper_permutation_workload(R):
    """The paper's array (permutation of 1..n after n/2 swaps), q = 32 sqrt(n)."""
    n = 10**8
    A = W.paper_permutation(n, 1004)
    q = 32 * 10**4
    l, r = W.uniform_queries(n, q, 2004)
    want = oracle.rmq_sparse_table(A, l, r)
    dA = torch.from_numpy(A).to(DEV)
    for v in (R.Variant.PLAIN, R.Variant.CONTRACTED):
        assert np.array_equal(gpu_answers(R, dA, l, r, v), want), v
