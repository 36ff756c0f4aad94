"""RLGL oracle -- TEST INFRASTRUCTURE, not part of the product.

ctypes wrapper around ``rlgl_oracle.c``: a plain FP64 CPU restatement of
the Red Light Green Light method (Alg. 1; Eqs. init, recursion_M/H/C,
pi_hat). Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import it. It shares no code with the CUDA library and
never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlgl_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALL_GREEN, THRESHOLD, TOPFRAC, MASK, LINK_THRESHOLD, BLOCK_RR, PC = 0, 1, 2, 3, 4, 5, 6
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOTSTOCHASTIC", 5: "EDEGENERATE", 6: "ENOCONV"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, so x86 and Arm agree)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            L.oracle_transition_probs.restype = ctypes.c_int
            L.oracle_transition_probs.argtypes = [i64, vp, vp, vp, vp]
            L.oracle_move.restype = None
            L.oracle_move.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
            L.oracle_initial_step.restype = None
            L.oracle_initial_step.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            L.oracle_select.restype = dbl
            L.oracle_select.argtypes = [i64, vp, vp, i32, dbl, i32, dbl, dbl, vp, i64, i64, dbl,
                                        ctypes.c_uint64, vp, vp]
            L.oracle_pc_uniform.restype = dbl
            L.oracle_pc_uniform.argtypes = [ctypes.c_uint64, i64, i64]
            L.oracle_sm64_next.restype = ctypes.c_uint64
            L.oracle_sm64_next.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
            L.oracle_l1.restype = dbl
            L.oracle_l1.argtypes = [i64, vp]
            L.oracle_sum.restype = dbl
            L.oracle_sum.argtypes = [i64, vp]
            L.oracle_invariant_residual.restype = dbl
            L.oracle_invariant_residual.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            L.oracle_solve.restype = ctypes.c_int
            L.oracle_solve.argtypes = [i64, vp, vp, vp, i32, dbl, i32, dbl, dbl, vp, i64,
                                       i64, dbl, i64, vp, vp, i64, vp, vp, i64, i64, dbl,
                                       ctypes.c_uint64, i32]
            L.oracle_estimate.restype = ctypes.c_int
            L.oracle_estimate.argtypes = [i64, vp, vp]
            L.oracle_power_iteration.restype = i64
            L.oracle_power_iteration.argtypes = [i64, vp, vp, vp, dbl, i64, i32, vp, vp]
            L.oracle_gth.restype = ctypes.c_int
            L.oracle_gth.argtypes = [i64, vp, vp]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def transition_probs(csr) -> np.ndarray:
    """p_e = w_e / row sum (or 1/deg for unit weights), FP64."""
    L = _load()
    p = np.empty(csr.nnz, dtype=np.float64)
    rc = L.oracle_transition_probs(csr.n, _p(csr.row_ptr), _p(csr.col), _p(csr.w), _p(p))
    if rc != 0:
        raise ValueError(f"not stochastic ({STATUS.get(rc, rc)})")
    return p


def initial_step(csr, p, m0: Optional[np.ndarray] = None):
    """Step 0: returns (C_1, H_1) = (-M_0 (I-P), M_0)."""
    L = _load()
    C = np.empty(csr.n)
    H = np.empty(csr.n)
    m0 = None if m0 is None else _f64(m0)
    L.oracle_initial_step(csr.n, _p(csr.row_ptr), _p(csr.col), _p(p), _p(m0), _p(C), _p(H))
    return C, H


def select(C, sched: int, theta_scale: float = 1.0, r: int = 1, abs_theta: float = 0.0,
           top_frac: float = 0.01, mask=None, row_ptr=None, move: int = 0, rr_blocks: int = 8,
           pc_frac: float = 0.05, seed: int = 0, cstat=None):
    """Green set of the schedule for cash C: returns (green uint8[n], theta).
    row_ptr (the CSR offsets) is needed by LINK_THRESHOLD only; move (t,
    counted from step 0), rr_blocks, pc_frac and seed by BLOCK_RR and PC.
    cstat: the cash whose statistics set theta and the PC constant (default
    C itself; the stale threshold passes the previous move's cash)."""
    L = _load()
    C = _f64(C)
    cs = None if cstat is None else _f64(cstat)
    green = np.empty(C.shape[0], dtype=np.uint8)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    rp = None if row_ptr is None else np.ascontiguousarray(row_ptr, dtype=np.int64)
    if sched == LINK_THRESHOLD and rp is None:
        raise ValueError("LINK_THRESHOLD needs row_ptr")
    th = L.oracle_select(C.shape[0], _p(rp), _p(C), sched, theta_scale, r, abs_theta, top_frac,
                         _p(mk), move, rr_blocks, pc_frac, seed, _p(cs), _p(green))
    return green, th


def move(csr, p, green, C, H):
    """One synchronous move in place; returns (|G|, sum deg, sum |M|)."""
    L = _load()
    st = np.zeros(3)
    g = np.ascontiguousarray(green, dtype=np.uint8)
    assert C.dtype == np.float64 and H.dtype == np.float64
    L.oracle_move(csr.n, _p(csr.row_ptr), _p(csr.col), _p(p), _p(g), _p(C), _p(H), _p(st))
    return st


def l1(x) -> float:
    x = _f64(x)
    return _load().oracle_l1(x.shape[0], _p(x))


def total(x) -> float:
    x = _f64(x)
    return _load().oracle_sum(x.shape[0], _p(x))


def invariant_residual(csr, p, C, H, c0=None) -> float:
    """||C - C_0 - H(P - I)||_1 (Eq. recursion_H_res)."""
    L = _load()
    C, H = _f64(C), _f64(H)
    c0 = None if c0 is None else _f64(c0)
    return L.oracle_invariant_residual(csr.n, _p(csr.row_ptr), _p(csr.col), _p(p),
                                       _p(C), _p(H), _p(c0))


def solve(csr, p, C, H, sched: int = THRESHOLD, theta_scale: float = 1.0, r: int = 1,
          abs_theta: float = 0.0, top_frac: float = 0.01, masks=None, safety_every: int = 0,
          tol: float = 1e-12, max_steps: int = 100000, check_every: int = 0, move0: int = 0,
          rr_blocks: int = 8, pc_frac: float = 0.05, seed: int = 0, theta_lag: int = 0):
    """Algorithm 1 from state (C, H) (modified in place). Returns a dict with
    status, moves, resid (||C||_1/|H 1|), pushes, hsum and the worst
    per-step invariant values when check_every >= 0. theta_lag = 1: every
    move after the first takes its threshold from the cash before the
    previous move and is made before its stop test takes effect (the stale
    threshold of Sec. 6; see oracle_solve)."""
    L = _load()
    assert C.dtype == np.float64 and H.dtype == np.float64
    mk, period = None, 1
    if masks is not None:
        mk = np.ascontiguousarray(masks, dtype=np.uint8).reshape(-1, csr.n)
        period = mk.shape[0]
    chk = np.zeros(3) if check_every >= 0 else None
    out = np.zeros(4)
    st = L.oracle_solve(csr.n, _p(csr.row_ptr), _p(csr.col), _p(p), sched, theta_scale, r,
                        abs_theta, top_frac, _p(mk), period, safety_every, tol, max_steps,
                        _p(C), _p(H), check_every, _p(chk), _p(out), move0, rr_blocks,
                        pc_frac, seed, theta_lag)
    res = dict(status=STATUS.get(st, st), moves=int(out[0]), resid=float(out[1]),
               pushes=float(out[2]), hsum=float(out[3]))
    if chk is not None:
        res.update(sum_cash=float(chk[0]), l1_growth=float(chk[1]), invariant=float(chk[2]))
    return res


def sm64_outputs(state: int, count: int):
    """The first `count` outputs of SplitMix64 from `state` (sequential form)."""
    L = _load()
    st = ctypes.c_uint64(state)
    return [L.oracle_sm64_next(ctypes.byref(st)) for _ in range(count)]


def pc_uniform(seed: int, t: int, i: int) -> float:
    """u_{t,i} of the PC schedule (SplitMix64, counter-based)."""
    return _load().oracle_pc_uniform(seed, t, i)


def estimate(H) -> np.ndarray:
    """pi_hat = H / (H 1) (Eq. pi_hat); raises on a degenerate history."""
    L = _load()
    H = _f64(H)
    pi = np.empty_like(H)
    rc = L.oracle_estimate(H.shape[0], _p(H), _p(pi))
    if rc != 0:
        raise ArithmeticError("degenerate history: H 1 = 0")
    return pi


def power_iteration(csr, p, tol: float = 1e-10, maxit: int = 100000, nthreads: int = 1,
                    start=None):
    """Reference pi by power iteration to ||pi_t - pi_{t+1}||_1 <= tol.
    Returns (pi, iterations, last delta)."""
    L = _load()
    pi = np.full(csr.n, -1.0) if start is None else _f64(start).copy()
    delta = ctypes.c_double(0.0)
    it = L.oracle_power_iteration(csr.n, _p(csr.row_ptr), _p(csr.col), _p(p), tol, maxit,
                                  nthreads, _p(pi), ctypes.addressof(delta))
    return pi, int(it), float(delta.value)


def gth(A) -> np.ndarray:
    """Stationary law of a dense row-stochastic matrix by GTH elimination."""
    L = _load()
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    pi = np.empty(A.shape[0])
    rc = L.oracle_gth(A.shape[0], _p(A), _p(pi))
    if rc != 0:
        raise ValueError("GTH: reducible chain")
    return pi


def degree_law(csr) -> np.ndarray:
    """pi_i = d_i / sum_k d_k (d_i = row length with multiplicity): the
    stationary law of the random walk on an undirected graph (each edge
    stored in both directions, unit weights)."""
    d = np.diff(np.asarray(csr.row_ptr)).astype(np.float64)
    return d / d.sum()


def dense_P(csr, p) -> np.ndarray:
    """Dense P from CSR probabilities (duplicates add)."""
    P = np.zeros((csr.n, csr.n))
    rows = np.repeat(np.arange(csr.n), np.diff(csr.row_ptr))
    np.add.at(P, (rows, csr.col), p)
    return P


def run(csr, sched: int = THRESHOLD, m0=None, **kw):
    """Step 0 + Algorithm 1 + estimate. Returns (pi_hat, C, H, info)."""
    p = transition_probs(csr)
    C, H = initial_step(csr, p, m0)
    info = solve(csr, p, C, H, sched=sched, **kw)
    pi = estimate(H) if info["status"] != "EDEGENERATE" else None
    return pi, C, H, info
