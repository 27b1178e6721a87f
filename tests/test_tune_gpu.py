"""The autotuner measures forms and block sizes on a batch, remembers the
fastest for the shape, and the answers of every candidate are the same."""
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


def test_autotune_remembers_the_fastest_choice(R):
    R.rmq_tune_clear()
    n, q = 2_000_000, 200_000
    A = W.uniform_array(n, 5)
    l, r = W.uniform_queries(n, q, 6)
    dA, dl, dr = (torch.from_numpy(x).to(DEV) for x in (A, l, r))
    out = torch.empty(q, dtype=torch.int32, device=DEV)
    best, ms = R.rmq_autotune(dA, dl, dr, out, variant=0, k_min=64, k_max=4096)
    assert ms > 0 and 64 <= best["k"] <= 65536 and best["variant"] in (R.Variant.PLAIN, R.Variant.CONTRACTED)
    assert R.rmq_tune(n, q) == best
    want = oracle.rmq_sparse_table(A, l, r)
    assert np.array_equal(out.cpu().numpy(), want)
    out.fill_(-7)
    R.rmq_batch(dA, dl, dr, out)                      # uses the remembered choice
    assert np.array_equal(out.cpu().numpy(), want)
    plain, _ = R.rmq_autotune(dA, dl, dr, out, variant=1, k_min=32, k_max=256)
    assert plain["variant"] == R.Variant.PLAIN and 32 <= plain["k"] <= 256
    R.rmq_tune_clear()
