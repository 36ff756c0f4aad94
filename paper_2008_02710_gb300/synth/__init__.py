"""Seeded synthetic Markov-chain inputs.

This module generates graphs and raw edge weights only. It performs no step
of the RLGL method: weights are not normalised to transition probabilities
here, and nothing about cash or history is computed. The CUDA library and the
CPU oracle each turn these inputs into transition probabilities on their own.

Workloads (sizes and distributions follow the RLGL experiments' scale: web
graphs of 1e5..1e6 nodes with heavy-tailed degrees, Sec. 6, Table 1):

* ``tiny_chain``: n nodes, out-degree U{1..8} to uniform targets, plus the
  cycle i->i+1 and a self-loop, weights U(0,1] (strongly connected and
  aperiodic).
* ``rmat_chain``: R-MAT (a,b,c,d) = (.57,.19,.19,.05) with a seeded random
  relabelling, then the cycle and self-loops; unit weights (p_ij =
  multiplicity/out-degree) or weights U(0,1]; optionally symmetrised.
* ``two_wheels``: the 12-node, 21-edge undirected graph of the paper's
  two-wheels figure (Sec. 6).
* dense fixtures for the mean-field stochastic block models (Sec. 4, 5) and
  doubly-stochastic permutation mixtures.
* ``rmat_chain_n_device``: the same R-MAT recipe at any size drawn on a CUDA
  device with PyTorch's seeded generator (a stream of requests needs
  thousands of graphs of up to millions of nodes; the host generator takes
  about a microsecond per node). Its graphs are not those of
  ``rmat_chain_n`` for the same seed: the device generator is its own
  seeded stream.

The C part (``synth.c``) uses a counter-based generator, so every graph is a
pure function of (sizes, seed) on any machine.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import NamedTuple, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libsynth.so`` next to it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, u64, i32, dbl, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_void_p)
            lib.synth_tiny_edges.restype = i64
            lib.synth_tiny_edges.argtypes = [i64, u64, vp, vp, vp, i64]
            lib.synth_rmat_edges.restype = None
            lib.synth_rmat_edges.argtypes = [i32, i64, dbl, dbl, dbl, u64, vp, vp]
            lib.synth_rmat_edges_n.restype = None
            lib.synth_rmat_edges_n.argtypes = [i64, i64, dbl, dbl, dbl, u64, vp, vp]
            lib.synth_batch_sizes.restype = i64
            lib.synth_batch_sizes.argtypes = [i64, u64, dbl, dbl, dbl, dbl, vp]
            lib.synth_batch_degrees.restype = i64
            lib.synth_batch_degrees.argtypes = [i64, u64, dbl, dbl, dbl, dbl, vp, vp]
            lib.synth_batch_fill.restype = ctypes.c_int
            lib.synth_batch_fill.argtypes = [i64, u64, vp, vp, vp]
            lib.synth_permutation.restype = None
            lib.synth_permutation.argtypes = [i64, u64, vp]
            lib.synth_relabel.restype = None
            lib.synth_relabel.argtypes = [i64, vp, vp, vp]
            lib.synth_weights.restype = None
            lib.synth_weights.argtypes = [i64, u64, u64, vp]
            lib.synth_cycle_selfloops.restype = None
            lib.synth_cycle_selfloops.argtypes = [i64, vp, vp]
            lib.synth_to_csr.restype = ctypes.c_int
            lib.synth_to_csr.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp]
            lib.synth_powerlaw_chain_edges.restype = i64
            lib.synth_powerlaw_chain_edges.argtypes = [i64, dbl, u64, vp, vp, i64]
            lib.synth_u64.restype = u64
            lib.synth_u64.argtypes = [u64, u64, u64]
            lib.synth_unit.restype = dbl
            lib.synth_unit.argtypes = [u64, u64, u64]
            _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


class CSR(NamedTuple):
    """A chain's raw graph: row i's out-edges are col[row_ptr[i]:row_ptr[i+1]].

    ``w`` holds positive raw weights (FP32) or is None for unit weights, in
    which case p_ij = multiplicity(i->j) / out-degree(i).
    """
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    w: Optional[np.ndarray]  # float32 [nnz] or None

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def nbytes(self) -> int:
        b = self.row_ptr.nbytes + self.col.nbytes
        return b + (self.w.nbytes if self.w is not None else 0)


def edges_to_csr(n: int, src: np.ndarray, dst: np.ndarray,
                 w: Optional[np.ndarray] = None) -> CSR:
    """Stable counting sort of an edge list by source into CSR."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = src.shape[0]
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(m, dtype=np.int32)
    wout = None
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float32)
        wout = np.empty(m, dtype=np.float32)
    rc = lib.synth_to_csr(n, m, _p(src), _p(dst), _p(w), _p(row_ptr), _p(col), _p(wout))
    if rc != 0:
        raise ValueError(f"edge list to CSR failed (code {rc})")
    return CSR(n, row_ptr, col, wout)


def tiny_chain(n: int = 1000, seed: int = 1) -> CSR:
    """n nodes; out-degree U{1..8} to uniform targets + cycle + self-loop; w ~ U(0,1]."""
    lib = _load()
    cap = 10 * n
    src = np.empty(cap, dtype=np.int32)
    dst = np.empty(cap, dtype=np.int32)
    w = np.empty(cap, dtype=np.float32)
    m = lib.synth_tiny_edges(n, seed, _p(src), _p(dst), _p(w), cap)
    if m < 0:
        raise RuntimeError("tiny chain generator overflow")
    return edges_to_csr(n, src[:m], dst[:m], w[:m])


def rmat_edges(scale: int, m: int, seed: int, a: float = 0.57, b: float = 0.19,
               c: float = 0.19, permute: bool = True):
    """m R-MAT edges on 2^scale nodes, optionally relabelled by a seeded permutation."""
    lib = _load()
    n = 1 << scale
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    lib.synth_rmat_edges(scale, m, a, b, c, seed, _p(src), _p(dst))
    if permute:
        perm = np.empty(n, dtype=np.int32)
        lib.synth_permutation(n, seed, _p(perm))
        lib.synth_relabel(m, _p(perm), _p(src), _p(dst))
    return src, dst


def cycle_selfloop_edges(n: int):
    lib = _load()
    src = np.empty(2 * n, dtype=np.int32)
    dst = np.empty(2 * n, dtype=np.int32)
    lib.synth_cycle_selfloops(n, _p(src), _p(dst))
    return src, dst


def weights(m: int, seed: int, stream: int = 0) -> np.ndarray:
    lib = _load()
    w = np.empty(m, dtype=np.float32)
    lib.synth_weights(m, seed, stream, _p(w))
    return w


def rmat_chain(scale: int, edge_factor: int = 16, seed: int = 1, a: float = 0.57,
               b: float = 0.19, c: float = 0.19, weighted: bool = False,
               undirected: bool = False, permute: bool = True) -> CSR:
    """R-MAT chain: 2^scale nodes, edge_factor*2^scale R-MAT edges, relabelled,
    plus the cycle i->i+1 and self-loops.

    ``undirected`` adds every R-MAT edge reversed and the cycle in both
    directions (unit weights). ``weighted`` draws weights U(0,1] per edge.
    """
    n = 1 << scale
    m = edge_factor * n
    src, dst = rmat_edges(scale, m, seed, a, b, c, permute)
    cs, cd = cycle_selfloop_edges(n)
    if undirected:
        if weighted:
            raise ValueError("the undirected variant uses unit weights")
        cyc_s, cyc_d = cs[0::2], cd[0::2]
        loop = cs[1::2]
        s_all = np.concatenate([src, dst, cyc_s, cyc_d, loop])
        d_all = np.concatenate([dst, src, cyc_d, cyc_s, loop])
        return edges_to_csr(n, s_all, d_all, None)
    src = np.concatenate([src, cs])
    dst = np.concatenate([dst, cd])
    w = weights(src.shape[0], seed, stream=1) if weighted else None
    return edges_to_csr(n, src, dst, w)


def rmat_chain_n(n: int, edge_factor: int = 16, seed: int = 1, a: float = 0.57,
                 b: float = 0.19, c: float = 0.19) -> CSR:
    """R-MAT chain on n nodes (any n): scale ceil(log2 n), out-of-range
    endpoints drawn again, seeded relabelling, cycle and self-loops; unit
    weights."""
    lib = _load()
    m = edge_factor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    lib.synth_rmat_edges_n(n, m, a, b, c, seed, _p(src), _p(dst))
    perm = np.empty(n, dtype=np.int32)
    lib.synth_permutation(n, seed, _p(perm))
    lib.synth_relabel(m, _p(perm), _p(src), _p(dst))
    cs, cd = cycle_selfloop_edges(n)
    return edges_to_csr(n, np.concatenate([src, cs]), np.concatenate([dst, cd]), None)


def two_wheels() -> CSR:
    """The 12-node two-wheels graph (Sec. 6, two-wheels figure), undirected,
    unit weights, each edge stored in both directions, no self-loops.

    Wheel 1: rim 1-2-3-4-5-6-1 with hub 7 joined to 1..6. Wheel 2 hangs off
    node 3: path 3-8-9-10-11-12 with hub 12 joined to 8, 9, 10 and the chord
    8-11. Nodes are numbered 0..11 here (paper label minus one).
    """
    und = [(1, 2), (2, 3), (3, 4), (4, 5), (5, 6), (6, 1), (1, 7),
           (3, 8), (8, 9), (9, 10), (10, 11), (11, 12),
           (2, 7), (3, 7), (4, 7), (5, 7), (6, 7),
           (8, 12), (9, 12), (10, 12), (8, 11)]
    s = [a - 1 for a, b in und] + [b - 1 for a, b in und]
    d = [b - 1 for a, b in und] + [a - 1 for a, b in und]
    return edges_to_csr(12, np.array(s), np.array(d), None)


def from_dense(A: np.ndarray) -> CSR:
    """CSR of the positive entries of a dense non-negative weight matrix."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    rows, cols = np.nonzero(A > 0)
    w = A[rows, cols].astype(np.float32)
    if not np.array_equal(w.astype(np.float64), A[rows, cols]):
        raise ValueError("weights must be exactly representable in FP32")
    return edges_to_csr(n, rows.astype(np.int32), cols.astype(np.int32), w)


def sbm_mean_field(sizes: Sequence[int], p: float, q: float) -> np.ndarray:
    """Dense adjacency of the mean-field SBM (Sec. 4.1, Sec. 5): weight p
    inside a block and q across blocks (every pair of nodes, self included)."""
    lab = np.repeat(np.arange(len(sizes)), sizes)
    return np.where(lab[:, None] == lab[None, :], p, q).astype(np.float64)


def doubly_stochastic(n: int, k: int, seed: int = 1) -> CSR:
    """P = sum_m alpha_m Pi_m over the identity, the cycle shift and k-2
    seeded random permutations; every row carries the same weights in the
    same order, so P is doubly stochastic and its stationary law is uniform."""
    lib = _load()
    perms = [np.arange(n, dtype=np.int32), ((np.arange(n) + 1) % n).astype(np.int32)]
    for r in range(k - 2):
        pm = np.empty(n, dtype=np.int32)
        lib.synth_permutation(n, seed * 1000 + r, _p(pm))
        perms.append(pm)
    alpha = weights(k, seed, stream=7)
    src = np.concatenate([np.arange(n, dtype=np.int32)] * k)
    dst = np.concatenate(perms)
    w = np.repeat(alpha, n)
    # Row order must be (perm 0, perm 1, ...) for every row: a stable sort by
    # source keeps the concatenation order.
    return edges_to_csr(n, src, dst, w)


def powerlaw_chain(n: int, delta: float, seed: int) -> CSR:
    """One chain of the many-chain mix (Poisson(delta) out-degrees, power-law
    targets, cycle, self-loops), unit weights."""
    lib = _load()
    cap = int(n * (delta + 12 * np.sqrt(delta) + 30)) + 64
    src = np.empty(cap, dtype=np.int32)
    dst = np.empty(cap, dtype=np.int32)
    m = lib.synth_powerlaw_chain_edges(n, float(delta), seed, _p(src), _p(dst), cap)
    if m < 0:
        raise RuntimeError("power-law chain generator overflow")
    return edges_to_csr(n, src[:m], dst[:m], None)


def u64(seed: int, stream: int, i: int) -> int:
    return int(_load().synth_u64(seed, stream, i))


def unit(seed: int, stream: int, i: int) -> float:
    return float(_load().synth_unit(seed, stream, i))


def stack_chains(chains):
    """Block-diagonal stack of several chains (node ids shifted): returns
    (CSR of the batch, node_ptr int64 [k+1]). Mixing weighted and unit-weight
    chains gives unit weights 1.0 to the latter."""
    n_off = np.cumsum([0] + [c.n for c in chains]).astype(np.int64)
    e_off = np.cumsum([0] + [c.nnz for c in chains]).astype(np.int64)
    row_ptr = np.concatenate([c.row_ptr[:-1] + e_off[k] for k, c in enumerate(chains)] +
                             [np.array([e_off[-1]], np.int64)])
    col = np.concatenate([c.col.astype(np.int64) + n_off[k] for k, c in enumerate(chains)]).astype(np.int32)
    if all(c.w is None for c in chains):
        w = None
    else:
        w = np.concatenate([c.w if c.w is not None else np.ones(c.nnz, np.float32) for c in chains])
    return CSR(int(n_off[-1]), row_ptr, col, w), n_off


def powerlaw_batch(nchains: int = 4096, seed: int = 1, lo: float = 100, hi: float = 1e5,
                   dlo: float = 4.0, dhi: float = 32.0):
    """The many-chain mix: nchains chains of log-uniform size in [lo, hi),
    mean out-degree U(dlo, dhi), Poisson out-degrees, power-law targets,
    cycle and self-loops, as one block-diagonal CSR (unit weights).
    Returns (CSR, node_ptr)."""
    lib = _load()
    node_ptr = np.empty(nchains + 1, dtype=np.int64)
    n = int(lib.synth_batch_sizes(nchains, seed, lo, hi, dlo, dhi, _p(node_ptr)))
    row_ptr = np.empty(n + 1, dtype=np.int64)
    nnz = int(lib.synth_batch_degrees(nchains, seed, lo, hi, dlo, dhi, _p(node_ptr), _p(row_ptr)))
    col = np.empty(nnz, dtype=np.int32)
    if lib.synth_batch_fill(nchains, seed, _p(node_ptr), _p(row_ptr), _p(col)) != 0:
        raise MemoryError("batch generator")
    return CSR(n, row_ptr, col, None), node_ptr


def pagerank_chain(csr: CSR, c_num: int = 17, c_den: int = 20) -> CSR:
    """The augmented chain P^(0) on n+1 nodes through which RLGL computes
    PageRank with damping c = c_num/c_den and uniform restart (Sec. 2.3.2,
    the Gauss-Southwell comparison): node 0 is the auxiliary node, original
    node i becomes i+1. Weights (FP32-exact integers; rows are normalised by
    the solver):
      row 0   : c_num * n to itself and c_den - c_num to every node, so
                p_00 = c and p_0j = (1 - c) / n;
      row i+1 : (c_den - c_num) * deg_i to node 0 and c_num per out-edge,
                so p_{i0} = 1 - c and p_ij = c / deg_i (unit-weight P);
                a node without out-edges sends everything to node 0.
    Without such dangling nodes the stationary law is (1/2, pi*/2), pi* the
    PageRank vector. With them, the original nodes' part, normalised, is
    PageRank with each dangling row replaced by the restart law s (the
    normalised solution of y = c y P + (1 - c) s with those rows zero).
    """
    if csr.w is not None:
        raise ValueError("pagerank_chain expects unit weights")
    n = csr.n
    a = float(c_num * n)
    if float(np.float32(a)) != a:
        raise ValueError("c_num * n is not exact in FP32")
    deg = np.diff(csr.row_ptr)
    rest = c_den - c_num
    row_ptr = np.empty(n + 2, dtype=np.int64)
    row_ptr[0] = 0
    row_ptr[1] = n + 1
    row_ptr[2:] = (n + 1) + np.cumsum(deg + 1)
    col = np.empty(int(row_ptr[-1]), dtype=np.int32)
    w = np.empty(int(row_ptr[-1]), dtype=np.float32)
    col[:n + 1] = np.arange(n + 1)
    w[0] = a
    w[1:n + 1] = rest
    starts = row_ptr[1:-1]
    col[starts] = 0
    w[starts] = np.where(deg > 0, rest * deg, 1).astype(np.float32)
    body = np.ones(int(row_ptr[-1]), dtype=bool)
    body[:n + 1] = False
    body[starts] = False
    col[body] = csr.col + 1
    w[body] = float(c_num)
    return CSR(n + 1, row_ptr, col, w)


def rmat_chain_n_device(n: int, edge_factor: int = 16, seed: int = 1, a: float = 0.57, b: float = 0.19,
                        c: float = 0.19, device="cuda") -> CSR:
    """R-MAT chain on n nodes drawn on a CUDA device: edge_factor * n R-MAT
    edges at scale ceil(log2 n) (one quadrant per bit, endpoints outside
    [0, n) drawn again), a seeded relabelling, then the cycle i -> i+1 and
    self-loops; unit weights. Returns a CSR of device tensors (row_ptr int64,
    col int32), in node order by source, stable in the draw order."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    m = int(edge_factor) * int(n)
    scale = max(1, int(np.ceil(np.log2(max(n, 2)))))

    def draw(k):
        src = torch.zeros(k, dtype=torch.int64, device=device)
        dst = torch.zeros(k, dtype=torch.int64, device=device)
        for level in range(scale):
            r = torch.rand(k, generator=g, device=device)
            bit = 1 << (scale - 1 - level)
            src += (r >= a + b).to(torch.int64) * bit
            dst += (((r >= a) & (r < a + b)) | (r >= a + b + c)).to(torch.int64) * bit
        return src, dst

    src, dst = draw(m)
    for _ in range(64):
        bad = (src >= n) | (dst >= n)
        k = int(bad.sum().item())
        if k == 0:
            break
        s2, d2 = draw(k)
        src[bad] = s2
        dst[bad] = d2
    else:
        keep = (src < n) & (dst < n)
        src, dst = src[keep], dst[keep]
    perm = torch.randperm(n, generator=g, device=device)
    src, dst = perm[src], perm[dst]
    ids = torch.arange(n, dtype=torch.int64, device=device)
    src = torch.cat([src, ids, ids])
    dst = torch.cat([dst, (ids + 1) % n, ids])
    order = torch.argsort(src, stable=True)
    col = dst[order].to(torch.int32)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(torch.bincount(src, minlength=n), 0)
    return CSR(int(n), row_ptr, col, None)


def stack_chains_device(chains):
    """Block-diagonal stack of several chains of device (or host) tensors:
    returns (CSR of device tensors, node_ptr int64 numpy [k+1]). Unit
    weights only."""
    import torch
    dev = chains[0].row_ptr.device if hasattr(chains[0].row_ptr, "device") else torch.device("cuda")
    n_off = np.cumsum([0] + [c.n for c in chains]).astype(np.int64)
    e_off = np.cumsum([0] + [int(c.row_ptr[-1]) for c in chains]).astype(np.int64)
    rp = [torch.as_tensor(c.row_ptr, device=dev)[:-1] + int(e_off[k]) for k, c in enumerate(chains)]
    rp.append(torch.tensor([int(e_off[-1])], dtype=torch.int64, device=dev))
    col = [(torch.as_tensor(c.col, device=dev).to(torch.int64) + int(n_off[k])).to(torch.int32)
           for k, c in enumerate(chains)]
    return CSR(int(n_off[-1]), torch.cat(rp), torch.cat(col), None), n_off
