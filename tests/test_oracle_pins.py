"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:
  * exhaustive brute force over every tiny array (a different algorithm:
    Python's min() then list.index(), which returns the first occurrence),
  * invariants every leftmost-argmin answer must satisfy,
  * closed forms (l == r, monotone and constant arrays, a planted minimum),
  * numpy library routines (argmin -- first occurrence by specification --,
    lexsort, unique, searchsorted) for the step-level functions,
  * Table 2 of the paper for the sparse-table level count,
  * planted mutants of the oracle's arithmetic, which the pins must reject.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1706_06940_gb300 import workloads as W

I32_MIN, I32_MAX = -2**31, 2**31 - 1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute(A, l, r):
    """Leftmost argmin by min() of the slice, then the first index holding it."""
    A = list(A)
    out = []
    for lo, hi in zip(l, r):
        if lo < 0 or hi < lo or hi >= len(A):
            out.append(-1)
            continue
        m = min(A[lo:hi + 1])
        out.append(A.index(m, lo, hi + 1))
    return np.array(out, dtype=np.int32)


def all_ranges(n):
    pairs = [(i, j) for i in range(n) for j in range(i, n)]
    l = np.array([p[0] for p in pairs], dtype=np.int32)
    r = np.array([p[1] for p in pairs], dtype=np.int32)
    return l, r


def check_invariants(A, l, r, out):
    """l <= out <= r; A[out] <= A[j] on [l, r]; A[j] > A[out] on [l, out)."""
    A = np.asarray(A, dtype=np.int64)
    for lo, hi, o in zip(l, r, out):
        assert lo <= o <= hi
        seg = A[lo:hi + 1]
        assert A[o] == seg.min()
        assert (A[lo:o] > A[o]).all()


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("n", range(1, 8))
def test_exhaustive_alphabet3(n):
    l, r = all_ranges(n)
    for A in itertools.product((0, 1, 2), repeat=n):
        A = np.array(A, dtype=np.int32)
        want = brute(A, l, r)
        assert np.array_equal(oracle.rmq_naive(A, l, r, threads=1), want), A
        assert np.array_equal(oracle.rmq_sparse_table(A, l, r, threads=1), want), A
        assert np.array_equal(oracle.contracted_pipeline(A, l, r), want), A


@pytest.mark.parametrize("n", range(1, 6))
def test_exhaustive_extreme_values(n):
    l, r = all_ranges(n)
    for A in itertools.product((I32_MIN, -1, 0, I32_MAX), repeat=n):
        A = np.array(A, dtype=np.int32)
        want = brute(A, l, r)
        assert np.array_equal(oracle.rmq_naive(A, l, r), want), A
        assert np.array_equal(oracle.rmq_sparse_table(A, l, r), want), A
        assert np.array_equal(oracle.contracted_pipeline(A, l, r), want), A


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("n,q,hi,seed", [(1000, 500, 2**31, 1), (4097, 800, 7, 2),
                                         (10_000, 300, 1000, 3), (257, 1000, 2, 4)])
def test_invariants_random(n, q, hi, seed):
    A = W.uniform_array(n, seed, 0, hi)
    l, r = W.uniform_queries(n, q, seed + 100)
    out = oracle.rmq_naive(A, l, r)
    check_invariants(A, l, r, out)
    assert np.array_equal(oracle.rmq_sparse_table(A, l, r), out)
    assert np.array_equal(oracle.contracted_pipeline(A, l, r), out)


def test_invariants_negative_values():
    A = W.uniform_array(5000, 11, -2**31, 2**31)
    l, r = W.log_width_queries(5000, 2000, 12, 1, 300)
    out = oracle.rmq_naive(A, l, r)
    check_invariants(A, l, r, out)
    assert np.array_equal(oracle.rmq_sparse_table(A, l, r), out)


# ---------------------------------------------------------------- closed forms

def test_single_cell_ranges():
    A = W.uniform_array(300, 5, 0, 3)
    l = np.arange(300, dtype=np.int32)
    assert np.array_equal(oracle.rmq_naive(A, l, l), l)
    assert np.array_equal(oracle.rmq_sparse_table(A, l, l), l)
    assert np.array_equal(oracle.contracted_pipeline(A, l, l), l)


def test_monotone_and_constant_arrays():
    n = 777
    l, r = W.uniform_queries(n, 2000, 6)
    inc = np.sort(W.uniform_array(n, 7, 0, 50))            # non-decreasing, with ties
    dec = np.arange(n, 0, -1, dtype=np.int32)             # strictly decreasing
    const = np.full(n, 42, dtype=np.int32)
    for f in (oracle.rmq_naive, oracle.rmq_sparse_table, oracle.contracted_pipeline):
        assert np.array_equal(f(inc, l, r), l)
        assert np.array_equal(f(dec, l, r), r)
        assert np.array_equal(f(const, l, r), l)


def test_planted_minimum():
    n, p = 5000, 3210
    A = W.uniform_array(n, 8, 1, 1000)
    A[p] = 0
    A[p + 7] = 0                                           # a later tie must lose
    l, r = W.uniform_queries(n, 3000, 9)
    hit = (l <= p) & (r >= p)
    for f in (oracle.rmq_naive, oracle.rmq_sparse_table, oracle.contracted_pipeline):
        out = f(A, l, r)
        assert (out[hit] == p).all()
        assert (out[~hit] != p).all()


def test_invalid_queries_answer_minus_one():
    A = W.uniform_array(100, 10)
    l = np.array([-1, 5, 50, 0, 99, 10], dtype=np.int32)
    r = np.array([3, 100, 49, 99, 99, 9], dtype=np.int32)
    want = np.array([-1, -1, -1, brute(A, [0], [99])[0], 99, -1], dtype=np.int32)
    for f in (oracle.rmq_naive, oracle.rmq_sparse_table, oracle.contracted_pipeline):
        assert np.array_equal(f(A, l, r), want)


def test_empty_batch():
    A = W.uniform_array(10, 1)
    e = np.zeros(0, dtype=np.int32)
    assert len(oracle.rmq_naive(A, e, e)) == 0
    assert len(oracle.rmq_sparse_table(A, e, e)) == 0
    assert len(oracle.contracted_pipeline(A, e, e)) == 0


# ---------------------------------------------------------------- step-level pins

def np_block_argmin(A, k):
    n = len(A)
    nb = -(-n // k)
    pad = np.full(nb * k, np.iinfo(np.int64).max, dtype=np.int64)
    pad[:n] = A
    return (np.argmin(pad.reshape(nb, k), axis=1) + np.arange(nb) * k).astype(np.int32)


@pytest.mark.parametrize("n,k,hi", [(1, 32, 9), (31, 32, 9), (32, 32, 9), (33, 32, 3),
                                    (1000, 64, 5), (4096 * 3 + 17, 4096, 2**31),
                                    (10_000, 128, 2)])
def test_block_minima_vs_numpy_argmin(n, k, hi):
    A = W.uniform_array(n, n + k, 0, hi)
    assert np.array_equal(oracle.block_minima(A, k), np_block_argmin(A, k))


@pytest.mark.parametrize("n,k,hi", [(1, 32, 9), (100, 32, 4), (32 * 37 + 5, 32, 3),
                                    (5000, 64, 1000), (64 * 64, 64, 2)])
def test_block_sparse_table_vs_numpy(n, k, hi):
    A = W.uniform_array(n, 3 * n + k, 0, hi)
    T = oracle.block_sparse_table(A, k)
    nb = -(-n // k)
    assert T.shape == (int(math.floor(math.log2(nb))) + 1, nb)
    for t in range(T.shape[0]):
        span = 1 << t
        for j in range(nb):
            if j + span > nb:
                assert T[t, j] == -1
                continue
            lo, hi_ = j * k, min(n, (j + span) * k)
            assert T[t, j] == lo + int(np.argmin(A[lo:hi_]))


def test_sort_endpoints_vs_lexsort():
    n, q = 1000, 700
    l, r = W.uniform_queries(n, q, 21)
    l[:50] = r[:50]                                        # duplicate positions
    pos, tag = oracle.sort_endpoints(l, r)
    ep = np.empty(2 * q, dtype=np.int64)
    ep[0::2], ep[1::2] = l, r
    order = np.lexsort((np.arange(2 * q), ep))             # by position, then input order
    assert np.array_equal(pos, ep[order].astype(np.uint32))
    assert np.array_equal(tag, order.astype(np.uint32))


def test_rank_endpoints_vs_unique_searchsorted():
    n, q = 500, 900
    l, r = W.uniform_queries(n, q, 22)
    pos, tag = oracle.sort_endpoints(l, r)
    P, ra, rb = oracle.rank_endpoints(pos, tag, q)
    U = np.unique(np.concatenate([l, r]))
    assert np.array_equal(P, U.astype(np.uint32))
    assert np.array_equal(ra, np.searchsorted(U, l))
    assert np.array_equal(rb, np.searchsorted(U, r))


def test_contract_vs_numpy_argmin():
    n = 3000
    A = W.uniform_array(n, 23, 0, 20)
    l, r = W.uniform_queries(n, 100, 24)
    P = np.unique(np.concatenate([l, r])).astype(np.uint32)
    got = oracle.contract(A, P)
    want = [int(P[j]) + int(np.argmin(A[P[j]:P[j + 1] + 1])) for j in range(len(P) - 1)]
    assert np.array_equal(got, np.array(want, dtype=np.int32))
    assert len(oracle.contract(A, P[:1])) == 0             # one endpoint: no areas


# ---------------------------------------------------------------- Table 2

def test_table2_level_count_reproduces_paper():
    """Extra space of BbST = nb * (floor(log2 nb) + 1) entries of 8 bytes,
    nb = ceil(n / k); as % of 4n it must print as Table 2 does."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table2_memory.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for k, p8, p9 in rows:
        for n, printed in ((10**8, p8), (10**9, p9)):
            nb = -(-n // int(k))
            pct = 100.0 * nb * oracle.sparse_levels(nb) * 8 / (4 * n)
            assert abs(pct - float(printed)) <= 0.005 + 1e-9, (k, n, pct, printed)


# ---------------------------------------------------------------- l-ary block table (Sec. 3.1 variant)

@pytest.mark.parametrize("n,k,ell,hi", [(1, 1, 2, 9), (100, 1, 3, 4), (32 * 37 + 5, 32, 16, 3),
                                        (5000, 8, 4, 1000), (64 * 64, 16, 2, 2)])
def test_lary_block_table_vs_numpy(n, k, ell, hi):
    """Level t, block j: numpy's first argmin over the ell^t blocks from j."""
    A = W.uniform_array(n, 5 * n + k + ell, 0, hi)
    T = oracle.lary_block_table(A, k, ell)
    nb = -(-n // k)
    levels = 1
    while ell ** levels <= nb:
        levels += 1
    assert T.shape == (levels, nb)
    for t in range(levels):
        span = ell ** t
        for j in range(nb):
            if j + span > nb:
                assert T[t, j] == -1
                continue
            lo, hi_ = j * k, min(n, (j + span) * k)
            assert T[t, j] == lo + int(np.argmin(A[lo:hi_]))


def test_lary_with_ell_2_is_the_block_sparse_table():
    A = W.uniform_array(3000, 61, 0, 7)
    for k in (1, 4, 32):
        assert np.array_equal(oracle.lary_block_table(A, k, 2), oracle.block_sparse_table(A, k))


@pytest.mark.parametrize("n", range(1, 7))
def test_lary_query_exhaustive(n):
    """Every array of length <= 6 over {0, 1, 2}, every range, several (k, ell):
    the same answers as the brute force, with at most ell table values."""
    l, r = all_ranges(n)
    for A in itertools.product((0, 1, 2), repeat=n):
        A = np.array(A, dtype=np.int32)
        want = brute(A, l, r)
        for k in (1, 2):
            for ell in (2, 3, 4):
                got, used = oracle.lary_query(A, k, ell, l, r)
                assert np.array_equal(got, want), (A, k, ell)
                assert used.max() <= ell


@pytest.mark.parametrize("k,ell", [(1, 2), (1, 16), (3, 3), (8, 4), (64, 16)])
def test_lary_query_random_and_lookup_bound(k, ell):
    n, q = 20_000, 5_000
    A = W.uniform_array(n, 71 + k + ell, 0, 100)
    l, r = W.uniform_queries(n, q, 72)
    ls, rs = W.log_width_queries(n, 2_000, 73, 1, 3_000)
    l, r = np.concatenate([l, ls]), np.concatenate([r, rs])
    got, used = oracle.lary_query(A, k, ell, l, r)
    assert np.array_equal(got, oracle.rmq_naive(A, l, r))
    assert used.max() <= ell
    # a query whose inner span is ell^t blocks long uses exactly one value
    nb = -(-n // k)
    for t in range(1, 4):
        L = ell ** t
        if L + 2 > nb:
            break
        lo, hi = 0, (L + 1) * k   # blocks 0 and L + 1 are the end blocks
        g, u = oracle.lary_query(A, k, ell, np.array([lo], np.int32), np.array([hi], np.int32))
        assert u[0] == 1 and g[0] == oracle.rmq_naive(A, [lo], [hi])[0]


def test_lary_levels_closed_form():
    """floor(log_ell nb) + 1, the level count behind the variant's space bound."""
    for nb in (1, 2, 15, 16, 17, 255, 256, 257, 97_657, 10**9):
        for ell in (2, 3, 4, 16):
            lv = oracle.lary_levels(nb, ell)
            assert ell ** (lv - 1) <= nb < ell ** lv, (nb, ell, lv)
    assert oracle.lary_levels(0, 2) == 0 and oracle.lary_levels(5, 1) == 0


# ---------------------------------------------------------------- planted mutants

def _mutant_rightmost(A, l, r):
    out = []
    for lo, hi in zip(l, r):
        best = lo
        for t in range(lo + 1, hi + 1):
            if A[t] <= A[best]:
                best = t
        out.append(best)
    return np.array(out, dtype=np.int32)


def _mutant_exclusive_r(A, l, r):
    return np.array([lo + int(np.argmin(A[lo:max(hi, lo + 1)])) for lo, hi in zip(l, r)],
                    dtype=np.int32)


def _mutant_sparse_one_window(A, l, r):
    out = []
    for lo, hi in zip(l, r):
        if lo == hi:
            out.append(lo)
            continue
        t = int(math.floor(math.log2(hi - lo)))
        w = A[lo:lo + (1 << t)]
        out.append(lo + int(np.argmin(w)))
    return np.array(out, dtype=np.int32)


def _mutant_sparse_right_wins(A, l, r):
    out = []
    for lo, hi in zip(l, r):
        if lo == hi:
            out.append(lo)
            continue
        t = int(math.floor(math.log2(hi - lo)))
        a = lo + int(np.argmin(A[lo:lo + (1 << t)]))
        s = hi - (1 << t) + 1
        b = s + int(np.argmin(A[s:hi + 1]))
        out.append(a if A[a] < A[b] else b)
    return np.array(out, dtype=np.int32)


def _mutant_contract_open_right(A, l, r):
    """Contraction with half-open areas A[P_j .. P_{j+1}) (drops the shared end)."""
    P = np.unique(np.concatenate([l, r]))
    AQ = [P[j] + int(np.argmin(A[P[j]:P[j + 1]])) for j in range(len(P) - 1)]
    out = []
    for lo, hi in zip(l, r):
        a, b = np.searchsorted(P, lo), np.searchsorted(P, hi)
        if a == b:
            out.append(lo)
            continue
        cand = AQ[a:b]
        out.append(min(cand, key=lambda p: (A[p], p)))
    return np.array(out, dtype=np.int32)


@pytest.mark.parametrize("mutant", [_mutant_rightmost, _mutant_exclusive_r,
                                    _mutant_sparse_one_window, _mutant_sparse_right_wins,
                                    _mutant_contract_open_right])
def test_pins_reject_planted_mutants(mutant):
    """Each plausible slip in the oracle's arithmetic fails the exhaustive pin."""
    caught = False
    for n in range(1, 7):
        l, r = all_ranges(n)
        for A in itertools.product((0, 1, 2), repeat=n):
            A = np.array(A, dtype=np.int32)
            if not np.array_equal(mutant(A, l, r), brute(A, l, r)):
                caught = True
                break
        if caught:
            break
    assert caught, mutant.__name__


# ---------------------------------------------------------------- multi-level BbST (Sec. 3.3)

HLEVEL_KS = [(1,), (2,), (1, 2), (1, 3), (2, 4), (1, 2, 4), (1, 3, 6), (2, 4, 8), (1, 2, 4, 8)]


@pytest.mark.parametrize("n", range(1, 9))
def test_hlevel_query_exhaustive(n):
    """Every array of length <= 8 over {0, 1, 2}, every range, block sizes of
    one to four levels (ks with k_1 = 1 scan nothing at the bottom): the same
    answers as the brute force."""
    l, r = all_ranges(n)
    arrays = itertools.product((0, 1, 2), repeat=n)
    if n == 8:                      # 3^8 arrays: take every fifth
        arrays = itertools.islice(arrays, 0, None, 5)
    for A in arrays:
        A = np.array(A, dtype=np.int32)
        want = brute(A, l, r)
        for ks in HLEVEL_KS:
            got, _ = oracle.hlevel_query(A, ks, l, r)
            assert np.array_equal(got, want), (A, ks)


@pytest.mark.parametrize("n,ks,hi", [(50_000, (8, 64), 100), (50_000, (4, 32, 256), 3),
                                     (65_536, (16, 256, 4096), 2**31 - 1), (99_991, (32, 96, 192, 1536), 50),
                                     (7_000, (64, 128, 8192), 9), (123_457, (128, 1024), 1000)])
def test_hlevel_query_random_and_work_bound(n, ks, hi):
    """Uniform and short ranges against the (pinned) naive scan; every query
    reads at most two end parts of k_h / k_{h-1} + ... + k_2 / k_1 + k_1
    values each, plus two table values (the Sec. 3.3 cost of checking up to
    two blocks)."""
    A = W.uniform_array(n, 91 + len(ks), 0, hi)
    l, r = W.uniform_queries(n, 4_000, 92)
    ls, rs = W.log_width_queries(n, 4_000, 93, 1, 5 * ks[-1])
    l, r = np.concatenate([l, ls]), np.concatenate([r, rs])
    got, work = oracle.hlevel_query(A, ks, l, r)
    assert np.array_equal(got, oracle.rmq_naive(A, l, r))
    chain = ks[0] + sum(ks[i] // ks[i - 1] for i in range(1, len(ks)))
    assert work.max() <= 2 * chain + 2
    assert work.min() >= 1


def test_hlevel_work_on_aligned_spans():
    """A query covering whole blocks of k_h reads exactly k_h / k_{h-1}
    minima in each end block plus two table values; one covering a single
    whole block of k_1 reads its one minimum, and one inside a block of k_1
    that covers no whole block scans exactly its cells."""
    n = 1 << 15
    A = W.uniform_array(n, 97, 0, 1 << 20)
    for ks in ((4, 64), (8, 32, 512), (16, 64, 256, 2048)):
        kh, kp = ks[-1], ks[-2]
        for bl, br in ((0, 5), (3, 4), (7, n // kh - 1)):
            l = np.array([bl * kh], np.int32)
            r = np.array([(br + 1) * kh - 1], np.int32)
            got, work = oracle.hlevel_query(A, ks, l, r)
            assert got[0] == oracle.rmq_naive(A, l, r)[0]
            assert work[0] == 2 * (kh // kp) + (2 if br - bl >= 2 else 0), (ks, bl, br)
        l = np.array([3 * ks[0]], np.int32)
        got, work = oracle.hlevel_query(A, ks, l, l + ks[0] - 1)
        assert work[0] == 1 and got[0] == 3 * ks[0] + int(np.argmin(A[3 * ks[0]:4 * ks[0]]))
        got, work = oracle.hlevel_query(A, ks, l + 1, l + ks[0] - 1)
        assert work[0] == ks[0] - 1 and got[0] == 3 * ks[0] + 1 + int(np.argmin(A[3 * ks[0] + 1:4 * ks[0]]))


def test_hlevel_space_closed_form_and_bad_parameters():
    """n/k_1 + ... + n/k_{h-1} + (n/k_h)(floor(log2(n/k_h)) + 1), block counts
    rounded up; -1 when some k_i does not divide k_{i+1} or the sizes do not grow."""
    for n in (1, 1000, 10**8, 10**9):
        for ks in ((1,), (64,), (32, 1024), (512, 4096, 65536), (2, 6, 12, 48)):
            nb = -(-n // ks[-1])
            want = sum(-(-n // k) for k in ks[:-1]) + nb * (nb.bit_length())
            assert oracle.hlevel_space(n, ks) == want, (n, ks)
    # one level is the block sparse table of Sec. 3.2 (Table 2's count)
    assert oracle.hlevel_space(10**8, (4096,)) == 24415 * 15
    for bad in ((4, 6), (8, 4), (4, 4), (0, 4), ()):
        assert oracle.hlevel_space(100, bad) == -1
    with pytest.raises(ValueError):
        oracle.hlevel_query(np.zeros(10, np.int32), (3, 4), [0], [1])


def _hlevel_py(A, ks, l, r, slip):
    """The multi-level query of Sec. 3.3 in Python with one planted slip, used
    only to show that the exhaustive pin rejects each slip."""
    A = [int(x) for x in A]
    n, h = len(A), len(ks)
    M = [[b * k + min(range(min(k, n - b * k)), key=lambda t: (A[b * k + t], t))
          for b in range(-(-n // k))] for k in ks]

    def better(x, y):
        if slip == "ties_right":
            return x if A[x] < A[y] else y
        return x if (A[x], x) <= (A[y], y) else y

    def part(lev, a, b):
        if lev == 1:
            return min(range(a, b + 1), key=lambda t: (A[t], t))
        s = ks[lev - 2]
        first, last = -(-a // s), (b + 1) // s
        if slip == "last_floor":
            last = b // s + 1
        if first >= last:
            if a // s == b // s:
                return part(lev - 1, a, b)
            x = part(lev - 1, a, (a // s + 1) * s - 1)
            return x if slip == "drop_split" else better(x, part(lev - 1, (b // s) * s, b))
        best = part(lev - 1, a, first * s - 1) if a < first * s else None
        for j in range(first, last):
            best = M[lev - 2][j] if best is None else better(best, M[lev - 2][j])
        if last * s <= b and slip != "drop_tail":
            best = better(best, part(lev - 1, last * s, b))
        return best

    kh = ks[-1]
    out = []
    for lo, hi in zip(l, r):
        bl, br = lo // kh, hi // kh
        if bl == br:
            out.append(part(h, lo, hi))
            continue
        best = part(h, lo, (bl + 1) * kh - 1)
        for j in range(bl + 1, br + (1 if slip == "inner_past_end" else 0)):
            best = better(best, M[h - 1][j])
        out.append(better(best, part(h, br * kh, hi)))
    return np.array(out, dtype=np.int32)


@pytest.mark.parametrize("slip", [None, "ties_right", "last_floor", "drop_split", "drop_tail", "inner_past_end"])
def test_hlevel_pins_reject_planted_slips(slip):
    """The Python restatement agrees with the brute force without a slip, and
    each slip in the level descent fails the exhaustive pin."""
    caught = False
    for n in range(1, 9):
        l, r = all_ranges(n)
        for A in itertools.product((0, 1, 2), repeat=n):
            A = np.array(A, dtype=np.int32)
            for ks in ((1, 2), (1, 2, 4), (2, 4)):
                if not np.array_equal(_hlevel_py(A, ks, l, r, slip), brute(A, l, r)):
                    caught = True
                    break
            if caught:
                break
        if caught or (slip is None and n == 6):
            break
    assert caught == (slip is not None), slip
