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


def test_two_width_classes_of_one_shape_keep_their_own_choices(R):
    """A uniform batch and a batch of short ranges of the same n and q are
    tuned apart (width classes 20 and 7 here); rmq_tune_batch, and so an AUTO
    rmq_batch, takes each batch's own choice, and both answer exactly."""
    R.rmq_tune_clear()
    n, q = 3_000_000, 300_000
    A = W.uniform_array(n, 15, 0, 1000)
    dA = torch.from_numpy(A).to(DEV)
    batches = {}
    for name, (l, r) in (("uniform", W.uniform_queries(n, q, 16)), ("short", W.log_width_queries(n, q, 17, 1, 10_000))):
        dl, dr = torch.from_numpy(l).to(DEV), torch.from_numpy(r).to(DEV)
        out = torch.empty(q, dtype=torch.int32, device=DEV)
        best, _ = R.rmq_autotune(dA, dl, dr, out, variant=0, k_min=32, k_max=4096)
        batches[name] = (l, r, dl, dr, best)
    wc = {name: int(round(np.log2(np.median(b[1].astype(np.int64) - b[0] + 1)))) for name, b in batches.items()}
    assert wc["uniform"] != wc["short"]
    saved = []
    for name, (l, r, dl, dr, best) in batches.items():
        assert R.rmq_tune_batch(dl, dr, n) == best, name     # the batch's own class
        saved.append(best)
        out = torch.full((q,), -7, dtype=torch.int32, device=DEV)
        R.rmq_batch(dA, dl, dr, out)                         # AUTO: samples the batch, uses its choice
        assert R.rmq_stream_status() == R.Status.OK
        assert np.array_equal(out.cpu().numpy(), oracle.rmq_sparse_table(A, l, r)), name
    # both choices survive a save and a load
    import tempfile, os
    path = os.path.join(tempfile.mkdtemp(), "tune.txt")
    R.rmq_tune_save(path)
    R.rmq_tune_clear()
    R.rmq_tune_load(path)
    for name, (l, r, dl, dr, best) in batches.items():
        assert R.rmq_tune_batch(dl, dr, n) == best, name
    R.rmq_tune_clear()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("tpq", [8, 16, 32])
def test_threads_per_query_do_not_change_answers(R, variant, tpq):
    n, q = 1_000_003, 60_000
    A = W.uniform_array(n, 30, 0, 20)
    l, r = W.log_width_queries(n, q, 31, 1, 3000)
    l[:20000], r[:20000] = W.uniform_queries(n, 20000, 32)
    dA, dl, dr = (torch.from_numpy(x).to(DEV) for x in (A, l, r))
    out = torch.full((q,), -7, dtype=torch.int32, device=DEV)
    R.rmq_batch_ex(dA, dl, dr, out, variant=variant, k=256, k_con=64, threads_per_query=tpq, k1=-1)
    assert R.rmq_stream_status() == R.Status.OK
    assert np.array_equal(out.cpu().numpy(), oracle.rmq_sparse_table(A, l, r))
