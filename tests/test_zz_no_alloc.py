"""rmq_batch_noalloc: the plain-form batch for callers that may not allocate
device memory (for example a host that has reserved all device memory for
its own allocator, or a loop that forbids allocation after start-up).

The entry point is called through the C ABI (ctypes, raw pointers) and must
give the same answers as rmq_batch_ex with the plain form and the same k on
two calls in a row; the second call uses another n and k, so its table is laid
out over whatever the first call left in the shared fixed buffer.  Answers are
positions, so the comparison is exact.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1706_06940_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1706_06940_gb300 import rmq
    return rmq, rmq.load()


def call_noalloc(lib, A, l, r, out, k):
    stream = torch.cuda.current_stream(A.device).cuda_stream
    return lib.rmq_batch_noalloc(ctypes.c_void_p(A.data_ptr()), A.numel(), ctypes.c_void_p(l.data_ptr()),
                                 ctypes.c_void_p(r.data_ptr()), l.numel(), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_int32(k), ctypes.c_void_p(stream))


def test_matches_rmq_batch_ex_on_two_calls_in_a_row(libs):
    rmq, lib = libs
    cases = [(3_000_000, 200_000, 1024, 0, 1000, 71), (777_777, 150_001, 256, 0, 7, 72)]
    for n, q, k, lo, hi, seed in cases:
        assert rmq.rmq_table_bytes(n, k) // 8 <= 1 << 19
        A = torch.from_numpy(W.uniform_array(n, seed, lo, hi)).to(DEV)
        l, r = W.uniform_queries(n, q, seed + 1)
        l[: q // 4], r[: q // 4] = W.log_width_queries(n, q // 4, seed + 2, 1, 5000)
        dl, dr = torch.from_numpy(l).to(DEV), torch.from_numpy(r).to(DEV)
        want = torch.empty(q, dtype=torch.int32, device=DEV)
        rmq.rmq_batch_ex(A, dl, dr, want, variant=rmq.Variant.PLAIN, k=k)
        got = torch.full((q,), -7, dtype=torch.int32, device=DEV)
        assert call_noalloc(lib, A, dl, dr, got, k) == rmq.Status.OK
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), want.cpu().numpy())
    assert rmq.rmq_stream_status() == rmq.Status.OK


def test_rejects_a_table_larger_than_the_fixed_buffer(libs):
    rmq, lib = libs
    n = 2_000_000                      # k = 32: 62,500 blocks x 16 levels > 2^19 entries
    assert rmq.rmq_table_bytes(n, 32) // 8 > 1 << 19
    A = torch.zeros(n, dtype=torch.int32, device=DEV)
    l = torch.zeros(4, dtype=torch.int32, device=DEV)
    out = torch.full((4,), -7, dtype=torch.int32, device=DEV)
    assert call_noalloc(lib, A, l, l, out, 32) == rmq.Status.ERR_SCRATCH_LIMIT
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == -7).all()          # nothing was enqueued
    assert call_noalloc(lib, A, l, l, out, 0) == rmq.Status.OK   # k = 0 picks a k that fits
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == 0).all()
