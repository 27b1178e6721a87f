"""Paper-scale parity (the second array size of the paper's experiments,
n = 1e9): both forms answer a uniform batch over a 4 GB array; the oracle
checks a sample of the answers (every short query, a few dozen uniform ones,
the full span), since a full naive check would scan about 1e15 cells."""
import numpy as np
import pytest

import oracle
from paper_1706_06940_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 10**9


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if torch.cuda.get_device_properties(0).total_memory < 24 * 2**30:
        pytest.skip("needs 24 GB of device memory")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1706_06940_gb300 import rmq
    return rmq


def test_n1e9_both_forms_on_sampled_answers(R):
    A = W.uniform_array(N, 2024)
    lu, ru = W.uniform_queries(N, 2_000_000, 2025)
    ls, rs = W.log_width_queries(N, 100_000, 2026, 1, 10_000)
    l = np.concatenate([lu, ls, [0, N - 1, 0]]).astype(np.int32)
    r = np.concatenate([ru, rs, [N - 1, N - 1, 0]]).astype(np.int32)
    q = len(l)
    # the sample: every short query, 48 uniform ones, the three special ones
    g = np.random.default_rng(2027)
    idx = np.concatenate([g.choice(len(lu), 48, replace=False), np.arange(len(lu), q)])
    want = oracle.rmq_naive(A, l[idx], r[idx])
    dA = torch.from_numpy(A).cuda()
    del A
    dl, dr = torch.from_numpy(l).cuda(), torch.from_numpy(r).cuda()
    answers = {}
    for variant in (R.Variant.PLAIN, R.Variant.CONTRACTED):
        out = torch.full((q,), -7, dtype=torch.int32, device="cuda")
        R.rmq_batch_ex(dA, dl, dr, out, variant=variant)
        assert R.rmq_stream_status() == R.Status.OK
        got = out.cpu().numpy()
        bad = np.nonzero(got[idx] != want)[0]
        assert len(bad) == 0, (variant.name, len(bad), idx[bad[:5]], got[idx[bad[:5]]], want[bad[:5]])
        # every answer lies in its range
        assert np.all((got >= l) & (got <= r)), variant.name
        answers[variant] = got
    # the two forms agree on every query, sampled or not
    assert np.array_equal(answers[R.Variant.PLAIN], answers[R.Variant.CONTRACTED])
