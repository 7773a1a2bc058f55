"""CPU oracle for LPA and Louvain (ctypes wrapper around ``oracle.c``).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg may import this package. The product
path (the CUDA library and its binding) never imports it.

Every function takes a symmetric CSR as numpy arrays: ``off`` int64[n+1],
``cols`` int32[nnz], ``w`` int64[nnz] or ``None`` for unit weights. Loops are
stored once, as the arc v->v with the loop's weight L (paper, Sec. II-A).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DEFAULT_SCHED_SEED = 0x5EED5EED

_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_INT = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (host C only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _configure(L):
    """Declare the C signatures of oracle.h on a loaded library."""
    L.orc_degw.restype = _I64
    L.orc_degw.argtypes = [_I64, _P, _P, _P, _P]
    L.orc_modularity.restype = ctypes.c_double
    L.orc_modularity.argtypes = [_I64, _P, _P, _P, _P, _P, _P]
    L.orc_move_gain.restype = None
    L.orc_move_gain.argtypes = [_I64, _P, _P, _P, _P, _I32, _I32, _P]
    L.orc_ws_create.restype = _P
    L.orc_ws_create.argtypes = [_I64]
    L.orc_ws_free.restype = None
    L.orc_ws_free.argtypes = [_P]
    L.orc_lpa_decide.restype = _I32
    L.orc_lpa_decide.argtypes = [_I64, _P, _P, _P, _P, _I32, _INT, _P]
    L.orc_louvain_decide.restype = _I32
    L.orc_louvain_decide.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _P, _I64, _I32, _INT, _P]
    L.orc_commit.restype = _INT
    L.orc_commit.argtypes = [_U64, _I32, _I32, _I32]
    L.orc_lpa.restype = _I32
    L.orc_lpa.argtypes = [_I64, _P, _P, _P, _I32, _I64, _INT, _INT, _U64, _P, _P, _P, _P, _P, _P, _P, _P]
    L.orc_local_move.restype = _I32
    L.orc_local_move.argtypes = [_I64, _P, _P, _P, _I32, _INT, _INT, _U64, _I32, _INT, _P, _P,
                                 _P, _P, _P, _P, _P, _P, _P]
    L.orc_aggregate.restype = _I64
    L.orc_aggregate.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _P]
    L.orc_louvain.restype = _I32
    L.orc_louvain.argtypes = [_I64, _P, _P, _P, _I32, _I32, _INT, _INT, _U64, _P, _P, _P, _P, _P]
    return L


def load(path: str):
    """Load and configure an oracle library built from ``oracle.c`` at `path`
    (the tests load deliberately altered copies this way)."""
    return _configure(ctypes.CDLL(path))


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_LIB)
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(off, cols, w):
    off = np.ascontiguousarray(off, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.int64)
    return off, cols, w


def _i128(parts) -> int:
    hi, lo = int(parts[0]), int(parts[1]) & ((1 << 64) - 1)
    return (hi << 64) | lo


def degw(off, cols, w=None):
    """Sec. II-A weighted degrees; returns (deg_w int64[n], vol)."""
    off, cols, w = _csr(off, cols, w)
    n = len(off) - 1
    out = np.zeros(n, dtype=np.int64)
    vol = lib().orc_degw(n, _ptr(off), _ptr(cols), _ptr(w), _ptr(out))
    return out, int(vol)


def modularity(off, cols, w, labels):
    """Sec. II-C modularity; returns (Q fp64, exact numerator, exact denominator)."""
    off, cols, w = _csr(off, cols, w)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    n = len(off) - 1
    num = np.zeros(2, dtype=np.int64)
    den = np.zeros(2, dtype=np.int64)
    q = lib().orc_modularity(n, _ptr(off), _ptr(cols), _ptr(w), _ptr(labels), _ptr(num), _ptr(den))
    return float(q), _i128(num), _i128(den)


def move_gain(off, cols, w, labels, v: int, B: int) -> int:
    """Eq. deltaQ scaled gain G (dQ = 2 G / vol^2) of moving v into B."""
    off, cols, w = _csr(off, cols, w)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    g = np.zeros(2, dtype=np.int64)
    lib().orc_move_gain(len(off) - 1, _ptr(off), _ptr(cols), _ptr(w), _ptr(labels), v, B, _ptr(g))
    return _i128(g)


class Workspace:
    """Scratch for repeated per-vertex decisions on one graph size."""

    def __init__(self, n: int):
        self.h = lib().orc_ws_create(n)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_ws_free(self.h)
            self.h = None


def lpa_decide(off, cols, w, labels, v: int, tie_keep_current: int = 1, ws=None) -> int:
    """Algorithm 1, PLPMove decision of one vertex against `labels`."""
    off, cols, w = _csr(off, cols, w)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    ws = ws or Workspace(len(off) - 1)
    return int(lib().orc_lpa_decide(len(off) - 1, _ptr(off), _ptr(cols), _ptr(w), _ptr(labels),
                                     v, tie_keep_current, ws.h))


def louvain_decide(off, cols, w, labels, sigma_tot, csize, degw_, vol, v, singleton_rule=1, ws=None):
    """Algorithm 2, the best-move decision of one vertex against a round-start state."""
    off, cols, w = _csr(off, cols, w)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    ws = ws or Workspace(len(off) - 1)
    return int(lib().orc_louvain_decide(len(off) - 1, _ptr(off), _ptr(cols), _ptr(w), _ptr(labels),
                                         _ptr(sigma_tot), _ptr(csize), _ptr(degw_), vol, v,
                                         singleton_rule, ws.h))


def commit(level: int, rnd: int, v: int, sched_seed: int = DEFAULT_SCHED_SEED) -> int:
    """The pinned deferral coin (1 = commit the move this round)."""
    return int(lib().orc_commit(sched_seed, level, rnd, v))


@dataclass
class RunTrace:
    rounds: int
    moved: np.ndarray
    deferred: np.ndarray
    active: np.ndarray
    arcs: np.ndarray
    cands: np.ndarray       # distinct neighbour labels summed over the examined vertices
    moved_arcs: np.ndarray  # arcs of the vertices that moved


def _trace(r, *arrays):
    return RunTrace(int(r), *(a[:r].copy() for a in arrays))


def _active(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


def lpa(off, cols, w=None, max_iter=100, threshold=0, tie_keep_current=1, use_frontier=1,
        sched_seed=DEFAULT_SCHED_SEED, active_in=None):
    """Algorithm 1 with synchronous rounds; returns (labels int32[n], RunTrace).
    active_in: optional initial V_active (n bools), default all vertices."""
    off, cols, w = _csr(off, cols, w)
    active_in = _active(active_in)
    n = len(off) - 1
    labels = np.zeros(n, dtype=np.int32)
    cap = max(max_iter, 1)
    tm, td, ta, tr, tc, tk = (np.zeros(cap, dtype=np.int64) for _ in range(6))
    r = lib().orc_lpa(n, _ptr(off), _ptr(cols), _ptr(w), max_iter, threshold, tie_keep_current,
                      use_frontier, sched_seed, _ptr(active_in), _ptr(labels), _ptr(tm), _ptr(td),
                      _ptr(ta), _ptr(tr), _ptr(tc), _ptr(tk))
    return labels, _trace(r, tm, td, ta, tr, tc, tk)


def local_move(off, cols, w=None, max_iter=100, singleton_rule=1, use_frontier=1, labels_in=None,
               sched_seed=DEFAULT_SCHED_SEED, level=0, active_in=None):
    """Algorithm 2 with synchronous rounds; returns (labels, total moves, RunTrace).
    active_in: optional initial needCheck (n bools), default all vertices."""
    off, cols, w = _csr(off, cols, w)
    active_in = _active(active_in)
    n = len(off) - 1
    if labels_in is None:
        labels = np.zeros(n, dtype=np.int32)
        given = 0
    else:
        labels = np.ascontiguousarray(labels_in, dtype=np.int32).copy()
        given = 1
    cap = max(max_iter, 1)
    tm, td, ta, tr, tc, tk = (np.zeros(cap, dtype=np.int64) for _ in range(6))
    moves = np.zeros(1, dtype=np.int64)
    r = lib().orc_local_move(n, _ptr(off), _ptr(cols), _ptr(w), max_iter, singleton_rule, use_frontier,
                             sched_seed, level, given, _ptr(active_in), _ptr(labels), _ptr(moves),
                             _ptr(tm), _ptr(td), _ptr(ta), _ptr(tr), _ptr(tc), _ptr(tk))
    if r < 0:
        raise ValueError("labels out of range")
    return labels, int(moves[0]), _trace(r, tm, td, ta, tr, tc, tk)


def aggregate(off, cols, w, labels):
    """Algorithm 3, Aggregation; returns (k, newid int32[n], coarse off, cols, w)."""
    off, cols, w = _csr(off, cols, w)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    n = len(off) - 1
    nnz = int(off[-1])
    newid = np.zeros(n, dtype=np.int32)
    coff = np.zeros(n + 1, dtype=np.int64)
    ccols = np.zeros(max(nnz, 1), dtype=np.int32)
    cw = np.zeros(max(nnz, 1), dtype=np.int64)
    cnnz = np.zeros(1, dtype=np.int64)
    k = lib().orc_aggregate(n, _ptr(off), _ptr(cols), _ptr(w), _ptr(labels), _ptr(newid), _ptr(coff),
                            _ptr(ccols), _ptr(cw), _ptr(cnnz))
    if k < 0:
        raise ValueError("labels out of range")
    m = int(cnnz[0])
    return int(k), newid, coff[: k + 1].copy(), ccols[:m].copy(), cw[:m].copy()


def louvain(off, cols, w=None, max_iter=100, max_levels=64, singleton_rule=1, use_frontier=1,
            sched_seed=DEFAULT_SCHED_SEED):
    """Algorithm 3; returns (labels, levels, Q, per-level (rounds, moves, n))."""
    off, cols, w = _csr(off, cols, w)
    n = len(off) - 1
    labels = np.zeros(n, dtype=np.int32)
    q = np.zeros(1, dtype=np.float64)
    cap = max(max_levels, 1)
    tr = np.zeros(cap, dtype=np.int32)
    tm = np.zeros(cap, dtype=np.int64)
    tn = np.zeros(cap, dtype=np.int64)
    lv = lib().orc_louvain(n, _ptr(off), _ptr(cols), _ptr(w), max_iter, max_levels, singleton_rule,
                           use_frontier, sched_seed, _ptr(labels), _ptr(q), _ptr(tr), _ptr(tm), _ptr(tn))
    return labels, int(lv), float(q[0]), (tr[:lv].copy(), tm[:lv].copy(), tn[:lv].copy())
