"""Seeded synthetic graph generators (planted-partition SBM, LFR-style, R-MAT).

This module produces the inputs that both the CPU oracle and the CUDA path
consume. It holds none of the community-detection arithmetic: only random
numbers, edge sampling and the construction of a canonical symmetric CSR
(rows sorted, no duplicate arcs, no loops).

Random numbers come from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): draw number i of the stream with state ``key`` is
``mix64(key + (i + 1) * 0x9E3779B97F4A7C15)``. The same definition is written
in CUDA (``rmat_gpu.cu``) so that large R-MAT graphs can be generated on the
device with bit-identical edges.

All outputs are torch tensors so the same CSR construction runs on the host
(numpy / torch CPU) and on the GPU (torch CUDA): ``off`` int64[n+1],
``cols`` int32[nnz], ``w`` int32[nnz] or ``None`` (unit weights).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from fractions import Fraction
from typing import Optional

import numpy as np
import torch

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

TAG_SBM = 0x53424D00
TAG_PERM = 0x5045524D
TAG_RMAT = 0x524D4154
TAG_LFR = 0x4C465200
TAG_W = 0x57454947

_HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- SplitMix64

def mix64_int(z: int) -> int:
    """SplitMix64 output function on a Python int (mod 2^64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, tag: int) -> int:
    """State of an independent stream for (seed, purpose tag)."""
    return mix64_int(mix64_int(seed) ^ tag)


def mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(M1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(M2)
        z ^= z >> np.uint64(31)
    return z


def draw(key: int, ctr: np.ndarray) -> np.ndarray:
    """Draw number `ctr` (uint64 array) of the SplitMix64 stream with state `key`."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (ctr + np.uint64(1)) * np.uint64(GAMMA)
    return mix64(z)


def threshold64(p) -> int:
    """floor(p * 2^64) for a probability given as a decimal string or number."""
    return min(int(Fraction(str(p)) * (1 << 64)), MASK64)


def threshold32(p) -> int:
    return min(int(Fraction(str(p)) * (1 << 32)), (1 << 32) - 1)


def uniform_int(r: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Map uint64 draws to integers in [lo, hi] (multiply-shift on the top 32 bits)."""
    span = np.uint64(hi - lo + 1)
    return (((r >> np.uint64(32)) * span) >> np.uint64(32)).astype(np.int64) + lo


def permutation(n: int, seed: int) -> np.ndarray:
    """Seeded permutation of 0..n-1 (argsort of per-index draws)."""
    r = draw(stream_key(seed, TAG_PERM), np.arange(n, dtype=np.uint64))
    return np.argsort(r, kind="stable").astype(np.int64)


# ------------------------------------------------------ canonical CSR build

@dataclass
class Graph:
    n: int
    off: torch.Tensor          # int64[n+1]
    cols: torch.Tensor         # int32[nnz]
    w: Optional[torch.Tensor]  # int32[nnz] or None (unit weights)
    planted: Optional[np.ndarray] = None
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.off[-1])

    def numpy(self):
        """(off int64, cols int32, w int64 or None) numpy arrays for the oracle."""
        off = self.off.cpu().numpy().astype(np.int64)
        cols = self.cols.cpu().numpy().astype(np.int32)
        w = None if self.w is None else self.w.cpu().numpy().astype(np.int64)
        return off, cols, w

    def to(self, device) -> "Graph":
        return Graph(self.n, self.off.to(device), self.cols.to(device),
                     None if self.w is None else self.w.to(device), self.planted, self.name)


def csr_from_edge_keys(keys: torch.Tensor, n: int, w: Optional[torch.Tensor] = None) -> Graph:
    """Symmetric CSR from sorted unique undirected edge keys lo * 2^32 + hi (lo < hi).

    Row u lists its smaller neighbours (from the edges where u is `hi`)
    followed by its larger neighbours (edges where u is `lo`); both runs are
    ascending, so every row is sorted. Runs on whatever device `keys` is on.
    """
    dev = keys.device
    m = keys.numel()
    lo = keys >> 32
    hi = keys & 0xFFFFFFFF
    del keys
    kb = hi * (1 << 32) + lo
    order = torch.argsort(kb)
    del kb
    deg_f = torch.bincount(lo, minlength=n)[:n]
    deg_b = torch.bincount(hi, minlength=n)[:n]
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    off[1:] = torch.cumsum(deg_f + deg_b, 0)
    start_f = torch.cumsum(deg_f, 0) - deg_f
    start_b = torch.cumsum(deg_b, 0) - deg_b
    cols = torch.empty(2 * m, dtype=torch.int32, device=dev)
    j = torch.arange(m, dtype=torch.int64, device=dev)
    pos = off[:-1][lo] + deg_b[lo] + (j - start_f[lo])
    cols[pos] = hi.to(torch.int32)
    wa = None
    if w is not None:
        wa = torch.empty(2 * m, dtype=torch.int32, device=dev)
        wa[pos] = w.to(torch.int32)
    del pos
    bsrc = hi[order]
    pos = off[:-1][bsrc] + (j - start_b[bsrc])
    cols[pos] = lo[order].to(torch.int32)
    if w is not None:
        wa[pos] = w[order].to(torch.int32)
    return Graph(n, off, cols, wa)


def canonical_keys(u: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """Sorted unique undirected keys lo*2^32+hi from endpoint arrays; loops dropped."""
    u = u.to(torch.int64)
    v = v.to(torch.int64)
    lo = torch.minimum(u, v)
    hi = torch.maximum(u, v)
    keep = lo != hi
    keys = lo[keep] * (1 << 32) + hi[keep]
    return torch.unique(keys, sorted=True)


def edge_weights(keys: torch.Tensor, seed: int, wmax: int) -> torch.Tensor:
    """Per-edge integer weights uniform in [1, wmax], a function of the edge key."""
    k = keys.cpu().numpy().astype(np.uint64)
    r = draw(stream_key(seed, TAG_W), k)
    return torch.from_numpy(uniform_int(r, 1, wmax).astype(np.int32)).to(keys.device)


# -------------------------------------------------------------- SBM

def sbm(n: int, blocks: int, p_in, p_out, seed: int, permute: bool = True,
        wmax: int = 1) -> Graph:
    """Planted-partition SBM: `blocks` equal blocks, pair {u,v} (u < v) is an
    edge with probability p_in inside a block and p_out across blocks, decided
    by draw(u * n + v) < floor(p * 2^64). Vertex ids are then relabelled by a
    seeded permutation; `planted` holds each vertex's block."""
    key = stream_key(seed, TAG_SBM)
    t_in, t_out = np.uint64(threshold64(p_in)), np.uint64(threshold64(p_out))
    bsz = n // blocks
    block = np.minimum(np.arange(n) // max(bsz, 1), blocks - 1)
    us, vs = [], []
    for u in range(n - 1):
        v = np.arange(u + 1, n, dtype=np.uint64)
        r = draw(key, np.uint64(u) * np.uint64(n) + v)
        same = block[u + 1:] == block[u]
        hit = np.where(same, r < t_in, r < t_out)
        sel = v[hit].astype(np.int64)
        if sel.size:
            us.append(np.full(sel.size, u, dtype=np.int64))
            vs.append(sel)
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    planted = block.astype(np.int32)
    if permute:
        p = permutation(n, seed)        # p[new] = old
        inv = np.empty(n, dtype=np.int64)
        inv[p] = np.arange(n)
        u, v = inv[u], inv[v]
        planted = planted[p]
    keys = canonical_keys(torch.from_numpy(u), torch.from_numpy(v))
    w = edge_weights(keys, seed, wmax) if wmax > 1 else None
    g = csr_from_edge_keys(keys, n, w)
    g.planted = planted
    g.name = f"sbm_n{n}_b{blocks}"
    return g


# -------------------------------------------------------------- R-MAT

def rmat_thresholds(a, b, c):
    A = threshold32(a)
    AB = threshold32(Fraction(str(a)) + Fraction(str(b)))
    ABC = threshold32(Fraction(str(a)) + Fraction(str(b)) + Fraction(str(c)))
    return A, AB, ABC


def rmat_keys_host(scale: int, edge_factor: int, a, b, c, seed: int,
                   chunk: int = 1 << 22) -> np.ndarray:
    """Undirected edge keys lo*2^32+hi of an R-MAT graph (loops -> -1).

    Edge i descends `scale` levels; at level l the quadrant is chosen by the
    top 32 bits x of draw(i * 64 + l): x < A -> (0,0), x < AB -> (0,1),
    x < ABC -> (1,0), else (1,1), giving bit (scale-1-l) of (src, dst)."""
    A, AB, ABC = (np.uint64(t) for t in rmat_thresholds(a, b, c))
    key = stream_key(seed, TAG_RMAT)
    m = edge_factor << scale
    out = np.empty(m, dtype=np.int64)
    for s in range(0, m, chunk):
        i = np.arange(s, min(m, s + chunk), dtype=np.uint64)
        src = np.zeros(i.size, dtype=np.uint64)
        dst = np.zeros(i.size, dtype=np.uint64)
        for l in range(scale):
            x = draw(key, (i << np.uint64(6)) | np.uint64(l)) >> np.uint64(32)
            bs = (x >= AB).astype(np.uint64)
            bd = (((x >= A) & (x < AB)) | (x >= ABC)).astype(np.uint64)
            src = (src << np.uint64(1)) | bs
            dst = (dst << np.uint64(1)) | bd
        lo = np.minimum(src, dst).astype(np.int64)
        hi = np.maximum(src, dst).astype(np.int64)
        out[s:s + i.size] = np.where(lo == hi, -1, lo * (1 << 32) + hi)
    return out


_gen_lib = None


def _gpu_lib():
    global _gen_lib
    if _gen_lib is None:
        path = build_gpu_generator()
        L = ctypes.CDLL(path)
        L.synth_sbm_rows.restype = ctypes.c_int
        L.synth_sbm_rows.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L.synth_sbm_edges.restype = ctypes.c_int
        L.synth_sbm_edges.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p]
        L.synth_rmat_keys.restype = ctypes.c_int
        L.synth_rmat_keys.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p]
        _gen_lib = L
    return _gen_lib


def build_gpu_generator(force: bool = False) -> str:
    """Compile the device R-MAT edge generator (same SplitMix64 definition)."""
    src = os.path.join(_HERE, "rmat_gpu.cu")
    out = os.path.join(_HERE, "libcdsynth.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["nvcc", "-O3", "-shared", "-Xcompiler", "-fPIC",
                               "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, src])
        os.replace(tmp, out)
    return out


def rmat_keys_device(scale: int, edge_factor: int, a, b, c, seed: int, device="cuda") -> torch.Tensor:
    A, AB, ABC = rmat_thresholds(a, b, c)
    m = edge_factor << scale
    out = torch.empty(m, dtype=torch.int64, device=device)
    stream = torch.cuda.current_stream(out.device).cuda_stream
    rc = _gpu_lib().synth_rmat_keys(stream_key(seed, TAG_RMAT), scale, A, AB, ABC, 0, m,
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    if rc != 0:
        raise RuntimeError(f"synth_rmat_keys failed: {rc}")
    return out


def rmat(scale: int, edge_factor: int = 16, a="0.57", b="0.19", c="0.19", seed: int = 3,
         device: str = "cpu", permute: bool = False) -> Graph:
    """R-MAT graph, deduplicated, symmetrised, loops removed, unit weights."""
    n = 1 << scale
    if device == "cpu":
        keys = torch.from_numpy(rmat_keys_host(scale, edge_factor, a, b, c, seed))
    else:
        keys = rmat_keys_device(scale, edge_factor, a, b, c, seed, device)
    keys = keys[keys >= 0]
    if permute:
        p = torch.from_numpy(permutation(n, seed))
        inv = torch.empty(n, dtype=torch.int64)
        inv[p] = torch.arange(n)
        inv = inv.to(keys.device)
        u, v = inv[keys >> 32], inv[keys & 0xFFFFFFFF]
        del keys
        keys = canonical_keys(u, v)
    else:
        keys = torch.unique(keys, sorted=True)
    g = csr_from_edge_keys(keys, n, None)
    g.name = f"rmat{scale}_ef{edge_factor}" + ("_perm" if permute else "")
    return g


# ------------------------------------------------- served request stream

TAG_SERVE = 0x53455256
TAG_SBMS = 0x53424D53


def _pick32(r: np.ndarray, span) -> np.ndarray:
    """Uniform integer in [0, span) from the top 32 bits (multiply-shift)."""
    return ((r >> np.uint64(32)) * np.asarray(span, dtype=np.uint64)) >> np.uint64(32)


def sbm_sparse_keys_host(n: int, k: int, m: int, seed: int) -> np.ndarray:
    """Edge-sampled planted partition: m candidate edges, edge j from draws
    3j, 3j+1, 3j+2: u uniform; it stays in u's block (size s) with
    probability 100 (s-1) / (100 (s-1) + n - s), i.e. p_out = p_in / 100,
    then v is uniform in the block, else uniform over the other n - s
    vertices. Keys lo*2^32+hi, loops -> -1. Same definition as the device
    kernel in rmat_gpu.cu."""
    if not 1 <= n <= 40_000_000:
        raise ValueError("n out of range")
    key = stream_key(seed, TAG_SBMS)
    bsz = max(n // k, 1)
    j = np.arange(m, dtype=np.uint64) * np.uint64(3)
    u = _pick32(draw(key, j), n).astype(np.int64)
    bu = np.minimum(u // bsz, k - 1)
    b0 = bu * bsz
    s = np.where(bu == k - 1, n - b0, bsz)
    in_w = (100 * (s - 1)).astype(np.uint64)
    out_w = (n - s).astype(np.uint64)
    tot = in_w + out_w
    same = _pick32(draw(key, j + np.uint64(1)), tot) < in_w
    r2 = draw(key, j + np.uint64(2))
    v_in = b0 + _pick32(r2, s.astype(np.uint64)).astype(np.int64)
    x = _pick32(r2, out_w).astype(np.int64)
    v_out = np.where(x < b0, x, x + s)
    v = np.where(tot == 0, u, np.where(same, v_in, v_out))
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    return np.where(lo == hi, -1, lo * (1 << 32) + hi)


def sbm_sparse(n: int, k: int, mean_deg: int = 16, seed: int = 5, device: str = "cpu") -> Graph:
    """Sparse planted-partition graph of about mean_deg * n / 2 edges (see
    sbm_sparse_keys_host), deduplicated, loops removed, unit weights, ids
    unpermuted (blocks are contiguous id ranges)."""
    m = n * mean_deg // 2
    if device == "cpu":
        keys = torch.from_numpy(sbm_sparse_keys_host(n, k, m, seed))
    else:
        keys = torch.empty(m, dtype=torch.int64, device=device)
        stream = torch.cuda.current_stream(keys.device).cuda_stream
        rc = _gpu_lib().synth_sbm_edges(stream_key(seed, TAG_SBMS), n, k, m, ctypes.c_void_p(keys.data_ptr()),
                                        ctypes.c_void_p(stream))
        if rc != 0:
            raise RuntimeError(f"synth_sbm_edges failed: {rc}")
    keys = torch.unique(keys[keys >= 0], sorted=True)
    g = csr_from_edge_keys(keys, n, None)
    g.planted = np.minimum(np.arange(n) // max(n // k, 1), k - 1).astype(np.int32)
    g.name = f"sbms_n{n}_k{k}"
    return g


def rmat_n(n: int, edge_factor: int = 8, seed: int = 5, device: str = "cpu", a="0.57", b="0.19",
           c="0.19") -> Graph:
    """R-MAT on n vertices: edge_factor * 2^scale edges drawn at scale =
    ceil(log2 n), edges with an endpoint >= n rejected, then deduplicated,
    symmetrised, loops removed, unit weights."""
    scale = max(1, int(n - 1).bit_length())
    if device == "cpu":
        keys = torch.from_numpy(rmat_keys_host(scale, edge_factor, a, b, c, seed))
    else:
        keys = rmat_keys_device(scale, edge_factor, a, b, c, seed, device)
    keys = keys[(keys >= 0) & ((keys & 0xFFFFFFFF) < n)]
    keys = torch.unique(keys, sorted=True)
    g = csr_from_edge_keys(keys, n, None)
    g.name = f"rmatn{n}_ef{edge_factor}"
    return g


def serve_specs(count: int, seed: int = 5, nmin: int = 100, nmax: int = 2_000_000):
    """Seeded served-request recipe: per request (kind, family, n, k, graph
    seed) with n log-uniform in [nmin, nmax], kind "louvain" with probability
    0.7 else "lpa", family "rmat" or "sbm" with probability 1/2 each, k
    uniform in {2..50} (SBM blocks)."""
    key = stream_key(seed, TAG_SERVE)
    r = draw(key, np.arange(4 * count, dtype=np.uint64)).reshape(count, 4)
    u = (r[:, 0] >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    ns = np.clip(np.floor(np.exp(np.log(nmin) + u * (np.log(nmax + 1) - np.log(nmin)))), nmin, nmax).astype(np.int64)
    louv = (r[:, 1] >> np.uint64(32)) < np.uint64(threshold32("0.7"))
    rm = (r[:, 2] >> np.uint64(63)) == np.uint64(1)
    ks = uniform_int(r[:, 3], 2, 50)
    return [("louvain" if louv[i] else "lpa", "rmat" if rm[i] else "sbm", int(ns[i]), int(min(ks[i], ns[i])),
             (seed << 24) + i) for i in range(count)]


def serve_graph(spec, device: str = "cpu") -> Graph:
    """The graph of one served request (see serve_specs)."""
    _, family, n, k, sd = spec
    if family == "rmat":
        return rmat_n(n, 8, seed=sd, device=device)
    return sbm_sparse(n, k, 16, seed=sd, device=device)


# -------------------------------------------------------------- LFR-style

def _powerlaw_int(r: np.ndarray, tau: float, lo: int, hi: int) -> np.ndarray:
    """Integers in [lo, hi] with P(k) proportional to k^-tau (inverse CDF)."""
    k = np.arange(lo, hi + 1, dtype=np.float64)
    cdf = np.cumsum(k ** (-tau))
    cdf /= cdf[-1]
    u = (r >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return lo + np.searchsorted(cdf, u, side="right").clip(0, hi - lo)


def lfr(n: int = 1_000_000, tau1: float = 2.5, dmin: int = 5, dmax: int = 1000,
        tau2: float = 1.5, cmin: int = 20, cmax: int = 5000, mu: float = 0.3,
        wmax: int = 8, seed: int = 2) -> Graph:
    """LFR-style benchmark graph, written from the LFR construction (power-law
    degrees and community sizes, a mixing fraction mu of each vertex's edges
    leaving its community), wired with configuration models; loops and
    multi-edges are dropped, so realised degrees fall slightly below targets."""
    key = stream_key(seed, TAG_LFR)
    ctr = 0

    def draws(cnt):
        nonlocal ctr
        r = draw(key, np.arange(ctr, ctr + cnt, dtype=np.uint64))
        ctr += cnt
        return r

    deg = _powerlaw_int(draws(n), tau1, dmin, dmax)
    cand = _powerlaw_int(draws(n // cmin + 1), tau2, cmin, cmax)
    sizes = []
    total = 0
    for s in cand.tolist():
        if total >= n:
            break
        s = min(s, n - total)
        if 0 < n - total - s < cmin:
            s = n - total  # fold a short remainder into the last community
        sizes.append(s)
        total += s
    sizes = np.array(sizes, dtype=np.int64)
    comm_of_slot = np.repeat(np.arange(len(sizes)), sizes)
    order = np.argsort(draws(n), kind="stable")
    comm = np.empty(n, dtype=np.int64)
    comm[order] = comm_of_slot
    kin = np.rint((1.0 - mu) * deg).astype(np.int64)
    kin = np.minimum(kin, sizes[comm] - 1)
    kout = deg - kin
    # internal configuration model per community: stubs sorted by (comm, draw)
    stub_v = np.repeat(np.arange(n), kin)
    r = draws(stub_v.size)
    o = np.lexsort((r, comm[stub_v]))
    stub_v = stub_v[o]
    sc = comm[stub_v]
    # pair consecutive stubs within a community (an odd stub is dropped)
    first = np.r_[True, sc[1:] != sc[:-1]]
    rank = np.arange(sc.size) - np.maximum.accumulate(np.where(first, np.arange(sc.size), 0))
    even = (rank % 2 == 0)
    nxt_same = np.r_[sc[1:] == sc[:-1], False]
    a_idx = np.nonzero(even & nxt_same)[0]
    u_in, v_in = stub_v[a_idx], stub_v[a_idx + 1]
    # external configuration model over all external stubs
    stub_x = np.repeat(np.arange(n), kout)
    o = np.argsort(draws(stub_x.size), kind="stable")
    stub_x = stub_x[o]
    h = stub_x.size // 2
    u_x, v_x = stub_x[: 2 * h: 2], stub_x[1: 2 * h: 2]
    u = np.concatenate([u_in, u_x])
    v = np.concatenate([v_in, v_x])
    keys = canonical_keys(torch.from_numpy(u), torch.from_numpy(v))
    w = edge_weights(keys, seed, wmax) if wmax > 1 else None
    g = csr_from_edge_keys(keys, n, w)
    g.planted = comm.astype(np.int32)
    g.name = f"lfr_n{n}"
    return g


# -------------------------------------------------------------- batches

def pack_batch(graphs) -> "tuple[Graph, np.ndarray]":
    """Block-diagonal packing of independent graphs: graph b's vertex v
    becomes vstart[b] + v. Unit weights are materialised as 1 when any graph
    is weighted. Returns (packed graph, vstart int64[B+1])."""
    vstart = np.zeros(len(graphs) + 1, dtype=np.int64)
    astart = np.zeros(len(graphs) + 1, dtype=np.int64)
    for b, g in enumerate(graphs):
        vstart[b + 1] = vstart[b] + g.n
        astart[b + 1] = astart[b] + g.nnz
    weighted = any(g.w is not None for g in graphs)
    off = np.zeros(vstart[-1] + 1, dtype=np.int64)
    cols = np.zeros(astart[-1], dtype=np.int32)
    w = np.ones(astart[-1], dtype=np.int32) if weighted else None
    for b, g in enumerate(graphs):
        go = g.off.cpu().numpy()
        off[vstart[b] + 1: vstart[b + 1] + 1] = go[1:] + astart[b]
        cols[astart[b]: astart[b + 1]] = g.cols.cpu().numpy() + vstart[b]
        if weighted and g.w is not None:
            w[astart[b]: astart[b + 1]] = g.w.cpu().numpy()
    packed = Graph(int(vstart[-1]), torch.from_numpy(off), torch.from_numpy(cols),
                   None if w is None else torch.from_numpy(w))
    packed.name = f"batch{len(graphs)}"
    return packed, vstart


def batch_specs(count: int = 4096, seed: int = 4, nmin: int = 50, nmax: int = 5000,
                kmin: int = 2, kmax: int = 50):
    """Seeded recipe of a batch: per graph (n log-uniform in [nmin, nmax],
    k uniform in {kmin..kmax}, seed + b)."""
    key = stream_key(seed, TAG_SBM ^ 0xBA7C4)
    r = draw(key, np.arange(2 * count, dtype=np.uint64))
    u = (r[:count] >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    ns = np.floor(np.exp(np.log(nmin) + u * (np.log(nmax + 1) - np.log(nmin)))).astype(np.int64)
    ns = np.clip(ns, nmin, nmax)
    ks = uniform_int(r[count:], kmin, kmax)
    ks = np.minimum(ks, ns)
    return [(int(n), int(k), seed + b) for b, (n, k) in enumerate(zip(ns, ks))]


def sbm_batch_device(specs, p_in="0.2", p_out="0.002", wmax: int = 4, device: str = "cuda"):
    """The planted-partition graphs of `specs` [(n, k, seed), ...] generated on
    the device with the same definition as `sbm` (identical edges, the same
    seeded relabelling and weights), packed block-diagonally.
    Returns (packed Graph on `device`, vstart int64[B+1], planted int32[n])."""
    B = len(specs)
    ns = np.array([n for n, _, _ in specs], dtype=np.int64)
    vstart = np.zeros(B + 1, dtype=np.int64)
    vstart[1:] = np.cumsum(ns)
    rows = int(vstart[-1])
    row_graph = np.repeat(np.arange(B, dtype=np.int32), ns)
    blocks = np.array([k for _, k, _ in specs], dtype=np.int32)
    keys = np.array([stream_key(sd, TAG_SBM) for _, _, sd in specs], dtype=np.uint64)
    t_in, t_out = threshold64(p_in), threshold64(p_out)
    pin = float(Fraction(str(p_in)))
    pairs = float(sum(n * (n - 1) // 2 for n in ns))
    cap = int(pairs * max(pin, float(Fraction(str(p_out)))) * 1.2) + 1024
    d = lambda a: torch.from_numpy(a).to(device)
    t_vstart, t_rg, t_blocks, t_keys = d(vstart), d(row_graph), d(blocks), d(keys.view(np.int64))
    out = torch.empty(cap, dtype=torch.int64, device=device)
    cnt = torch.zeros(1, dtype=torch.int64, device=device)
    stream = torch.cuda.current_stream(out.device).cuda_stream
    rc = _gpu_lib().synth_sbm_rows(t_vstart.data_ptr(), t_rg.data_ptr(), t_blocks.data_ptr(), t_keys.data_ptr(),
                                   t_in, t_out, rows, out.data_ptr(), cnt.data_ptr(), cap, stream)
    if rc != 0:
        raise RuntimeError("synth_sbm_rows failed")
    m = int(cnt.item())
    if m > cap:
        raise RuntimeError("SBM edge buffer too small")
    e = out[:m]
    b = e >> 40
    u = (e >> 20) & 0xFFFFF
    v = e & 0xFFFFF
    # the per-graph seeded relabelling of `sbm`: new id of old vertex x
    inv = np.empty(rows, dtype=np.int64)
    planted = np.empty(rows, dtype=np.int32)
    for gi, (n, k, sd) in enumerate(specs):
        p = permutation(n, sd)
        loc = np.empty(n, dtype=np.int64)
        loc[p] = np.arange(n)
        inv[vstart[gi]:vstart[gi + 1]] = loc
        bsz = max(n // k, 1)
        planted[vstart[gi]:vstart[gi + 1]] = np.minimum(np.arange(n) // bsz, k - 1)[p]
    t_inv = d(inv)
    base = t_vstart[b]
    nu = t_inv[base + u]
    nv = t_inv[base + v]
    lo = torch.minimum(nu, nv)
    hi = torch.maximum(nu, nv)
    local = torch.unique(b * (1 << 40) + lo * (1 << 20) + hi, sorted=True)
    b = local >> 40
    lo = (local >> 20) & 0xFFFFF
    hi = local & 0xFFFFF
    gkeys = (t_vstart[b] + lo) * (1 << 32) + (t_vstart[b] + hi)
    w = None
    if wmax > 1:
        wkeys = np.array([stream_key(sd, TAG_W) for _, _, sd in specs], dtype=np.uint64)
        bk = wkeys[b.cpu().numpy()]
        ctr = (lo * (1 << 32) + hi).cpu().numpy().astype(np.uint64)
        with np.errstate(over="ignore"):
            z = bk + (ctr + np.uint64(1)) * np.uint64(GAMMA)
        w = torch.from_numpy(uniform_int(mix64(z), 1, wmax).astype(np.int32)).to(device)
    g = csr_from_edge_keys(gkeys, rows, w)
    g.planted = planted
    g.name = f"sbm_batch{B}"
    return g, vstart, planted


def unpack_batch(packed: Graph, vstart) -> "list[Graph]":
    """The member graphs of a block-diagonal batch, with local vertex ids."""
    out = []
    off = packed.off
    for b in range(len(vstart) - 1):
        a0, a1 = int(off[vstart[b]]), int(off[vstart[b + 1]])
        o = off[vstart[b]:vstart[b + 1] + 1] - a0
        c = packed.cols[a0:a1] - int(vstart[b])
        w = None if packed.w is None else packed.w[a0:a1]
        out.append(Graph(int(vstart[b + 1] - vstart[b]), o, c.to(torch.int32), w))
    return out


# -------------------------------------------------------------- small helpers

def from_edge_list(n: int, edges, weights=None, loops=None) -> Graph:
    """Symmetric CSR from an explicit undirected edge list (test fixtures).

    `edges` are (u, v) pairs with u != v, `weights` their weights, `loops` a
    dict {v: L} of loop weights (stored once as the arc v->v)."""
    adj = [dict() for _ in range(n)]
    for i, (a, b) in enumerate(edges):
        wt = 1 if weights is None else int(weights[i])
        assert a != b
        adj[a][b] = adj[a].get(b, 0) + wt
        adj[b][a] = adj[b].get(a, 0) + wt
    for v, L in (loops or {}).items():
        adj[v][v] = adj[v].get(v, 0) + int(L)
    off = np.zeros(n + 1, dtype=np.int64)
    cols, ws = [], []
    for v in range(n):
        for u in sorted(adj[v]):
            cols.append(u)
            ws.append(adj[v][u])
        off[v + 1] = len(cols)
    unit = weights is None and not loops
    w = None if unit else torch.tensor(ws, dtype=torch.int32)
    return Graph(n, torch.from_numpy(off), torch.tensor(cols, dtype=torch.int32), w)
