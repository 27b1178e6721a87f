"""CPU oracle for batched range minimum queries -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library (``paper_1706_06940_gb300``)
never imports it, and it imports nothing from the GPU library.

The arithmetic lives in ``rmq_oracle.c`` (plain C, OpenMP over queries); this
module only compiles it with gcc and marshals numpy arrays through ctypes.
Every function follows a passage of Grabowski & Kowalski, "Faster batched
range minimum queries" (arXiv:1706.06940); see the C file for the citations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmq_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_liboracle.so`` (gcc, -O2, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_max_threads.argtypes = []
    lib.oracle_rmq_naive.restype = None
    lib.oracle_rmq_naive.argtypes = [_i32p, _i64, _i32p, _i32p, _i64, _i32p, ctypes.c_int]
    lib.oracle_rmq_sparse_table.restype = ctypes.c_int
    lib.oracle_rmq_sparse_table.argtypes = [_i32p, _i64, _i32p, _i32p, _i64, _i32p, ctypes.c_int]
    lib.oracle_sparse_levels.restype = ctypes.c_int
    lib.oracle_sparse_levels.argtypes = [_i64]
    lib.oracle_block_minima.restype = None
    lib.oracle_block_minima.argtypes = [_i32p, _i64, _i64, _i32p]
    lib.oracle_block_sparse_table.restype = None
    lib.oracle_block_sparse_table.argtypes = [_i32p, _i64, _i64, _i32p]
    lib.oracle_sort_endpoints.restype = ctypes.c_int
    lib.oracle_sort_endpoints.argtypes = [_i32p, _i32p, _i64, _u32p, _u32p]
    lib.oracle_rank_endpoints.restype = ctypes.c_int64
    lib.oracle_rank_endpoints.argtypes = [_u32p, _u32p, _i64, _u32p, _i32p, _i32p]
    lib.oracle_contract.restype = None
    lib.oracle_contract.argtypes = [_i32p, _i64, _u32p, _i64, _i32p]
    lib.oracle_contracted_query.restype = None
    lib.oracle_contracted_query.argtypes = [_i32p, _i64, _i32p, _i32p, _i32p, _i32p, _i32p,
                                            _i64, _i32p]
    lib.oracle_lary_levels.restype = ctypes.c_int
    lib.oracle_lary_levels.argtypes = [_i64, _i64]
    lib.oracle_lary_block_table.restype = None
    lib.oracle_lary_block_table.argtypes = [_i32p, _i64, _i64, _i64, _i32p]
    lib.oracle_lary_query.restype = None
    lib.oracle_lary_query.argtypes = [_i32p, _i64, _i64, _i64, _i32p, _i32p, _i32p, _i64, _i32p, _i32p]
    _i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
    lib.oracle_hlevel_space.restype = ctypes.c_int64
    lib.oracle_hlevel_space.argtypes = [_i64, _i64p, ctypes.c_int]
    lib.oracle_hlevel_query.restype = ctypes.c_int
    lib.oracle_hlevel_query.argtypes = [_i32p, _i64, _i64p, ctypes.c_int, _i32p, _i32p, _i64, _i32p, _i64p]
    _lib = lib
    return lib


def _i32(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.int32)


def max_threads() -> int:
    """OpenMP threads the oracle uses by default (the host core count it sees)."""
    return int(_load().oracle_max_threads())


def rmq_naive(A, l, r, threads: int = 0) -> np.ndarray:
    """Leftmost argmin of A[l_i .. r_i] by a plain scan per query (-1 if invalid)."""
    A, l, r = _i32(A), _i32(l), _i32(r)
    out = np.empty(len(l), dtype=np.int32)
    _load().oracle_rmq_naive(A, len(A), l, r, len(l), out, int(threads))
    return out


def rmq_sparse_table(A, l, r, threads: int = 0) -> np.ndarray:
    """Same answers as rmq_naive, via the textbook full-array sparse table."""
    A, l, r = _i32(A), _i32(l), _i32(r)
    out = np.empty(len(l), dtype=np.int32)
    rc = _load().oracle_rmq_sparse_table(A, len(A), l, r, len(l), out, int(threads))
    if rc != 0:
        raise MemoryError("oracle sparse table: allocation failed")
    return out


def sparse_levels(m: int) -> int:
    """floor(log2 m) + 1 (0 for m <= 0)."""
    return int(_load().oracle_sparse_levels(int(m)))


def block_minima(A, k: int) -> np.ndarray:
    """Position of the leftmost minimum of every k-block of A."""
    A = _i32(A)
    nb = (len(A) + k - 1) // k
    out = np.empty(nb, dtype=np.int32)
    _load().oracle_block_minima(A, len(A), int(k), out)
    return out


def block_sparse_table(A, k: int) -> np.ndarray:
    """[levels, nb] positions of the minimum over 2^t blocks from block j (-1 if absent)."""
    A = _i32(A)
    nb = (len(A) + k - 1) // k
    lv = sparse_levels(nb)
    out = np.empty(lv * nb, dtype=np.int32)
    _load().oracle_block_sparse_table(A, len(A), int(k), out)
    return out.reshape(lv, nb)


def sort_endpoints(l, r):
    """Stable sort of the 2q endpoints (pos, tag = 2i + side) by position."""
    l, r = _i32(l), _i32(r)
    q = len(l)
    pos = np.empty(2 * q, dtype=np.uint32)
    tag = np.empty(2 * q, dtype=np.uint32)
    if _load().oracle_sort_endpoints(l, r, q, pos, tag) != 0:
        raise MemoryError("oracle sort: allocation failed")
    return pos, tag


def rank_endpoints(pos_sorted, tag_sorted, q: int):
    """Distinct sorted positions P[0..m) and the ranks (a_i, b_i) of every query."""
    pos_sorted = np.ascontiguousarray(pos_sorted, dtype=np.uint32)
    tag_sorted = np.ascontiguousarray(tag_sorted, dtype=np.uint32)
    P = np.empty(max(len(pos_sorted), 1), dtype=np.uint32)
    ra = np.full(q, -1, dtype=np.int32)
    rb = np.full(q, -1, dtype=np.int32)
    m = _load().oracle_rank_endpoints(pos_sorted, tag_sorted, len(pos_sorted), P, ra, rb)
    return P[:m].copy(), ra, rb


def contract(A, P) -> np.ndarray:
    """A_Q as positions: leftmost minimum of A[P_j .. P_{j+1}], j < m-1."""
    A = _i32(A)
    P = np.ascontiguousarray(P, dtype=np.uint32)
    out = np.empty(max(len(P) - 1, 0), dtype=np.int32)
    if len(P) >= 2:
        _load().oracle_contract(A, len(A), P, len(P), out)
    return out


def contracted_query(A, AQ_pos, l, r, rank_l, rank_r) -> np.ndarray:
    """Answers from the contracted array, by the definition over A_Q."""
    A, AQ_pos, l, r = _i32(A), _i32(AQ_pos), _i32(l), _i32(r)
    rank_l, rank_r = _i32(rank_l), _i32(rank_r)
    out = np.empty(len(l), dtype=np.int32)
    aq = AQ_pos if len(AQ_pos) else np.zeros(1, dtype=np.int32)
    _load().oracle_contracted_query(A, len(A), aq, l, r, rank_l, rank_r, len(l), out)
    return out


def contracted_pipeline(A, l, r) -> np.ndarray:
    """BbST_CON's steps 1, 2 and 4 in the paper's order, each by its definition.

    Invalid queries take part in the sort as (0, 0) and answer -1.
    """
    A, l, r = _i32(A), _i32(l), _i32(r)
    ok = (l >= 0) & (r >= l) & (r < len(A))
    pos, tag = sort_endpoints(np.where(ok, l, 0), np.where(ok, r, 0))
    P, ra, rb = rank_endpoints(pos, tag, len(l))
    AQ = contract(A, P)
    return contracted_query(A, AQ, l, r, ra, rb)


def lary_levels(nb: int, ell: int) -> int:
    """floor(log_ell nb) + 1 (0 for nb <= 0 or ell < 2)."""
    return int(_load().oracle_lary_levels(int(nb), int(ell)))


def lary_block_table(A, k: int, ell: int) -> np.ndarray:
    """[levels, nb] positions of the minimum over ell^t blocks from block j (-1 if absent)."""
    A = _i32(A)
    nb = (len(A) + k - 1) // k
    lv = lary_levels(nb, ell)
    out = np.empty(max(lv * nb, 1), dtype=np.int32)
    _load().oracle_lary_block_table(A, len(A), int(k), int(ell), out)
    return out[: lv * nb].reshape(lv, nb)


def lary_query(A, k: int, ell: int, l, r):
    """Answers through the ell-ary block table (the Sec. 3.1 variant), and
    the number of table values each query used."""
    A, l, r = _i32(A), _i32(l), _i32(r)
    T = np.ascontiguousarray(lary_block_table(A, k, ell).reshape(-1), dtype=np.int32)
    T = T if len(T) else np.zeros(1, dtype=np.int32)
    out = np.empty(len(l), dtype=np.int32)
    used = np.empty(len(l), dtype=np.int32)
    _load().oracle_lary_query(A, len(A), int(k), int(ell), T, l, r, len(l), out, used)
    return out, used


def hlevel_space(n: int, ks) -> int:
    """Entries kept by the multi-level structure of Sec. 3.3 with block sizes
    ks = (k_1, ..., k_h) (-1 on bad parameters)."""
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    return int(_load().oracle_hlevel_space(int(n), ks, len(ks)))


def hlevel_query(A, ks, l, r):
    """Answers through the multi-level structure of Sec. 3.3 (block sizes ks),
    and the work of each query (cells scanned, minima and table values read)."""
    A, l, r = _i32(A), _i32(l), _i32(r)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    out = np.empty(len(l), dtype=np.int32)
    work = np.empty(len(l), dtype=np.int64)
    if _load().oracle_hlevel_query(A, len(A), ks, len(ks), l, r, len(l), out, work) != 0:
        raise ValueError("bad block sizes for the multi-level structure")
    return out, work
