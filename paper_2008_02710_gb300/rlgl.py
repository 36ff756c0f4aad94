"""Python binding of librlgl (include/rlgl.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts
numpy arrays / torch tensors into pointers and status codes into
exceptions. It never computes any part of a move itself and has no CPU
fallback: if the library cannot be loaded, importing the functions raises.

Names follow the C ABI: ``create``, ``step``, ``solve``, ``estimate``, ...
and the ``Chain`` class wraps one context.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import _build

ALL_GREEN, THRESHOLD, TOPFRAC, MASK, LINK_THRESHOLD, BLOCK_RR, PC = 0, 1, 2, 3, 4, 5, 6
FP64, MIXED = 0, 1
HOST, DEVICE = 0, 1
SCHEDULES = {"all_green": ALL_GREEN, "threshold": THRESHOLD, "topfrac": TOPFRAC, "mask": MASK,
             "link_threshold": LINK_THRESHOLD, "block_rr": BLOCK_RR, "pc": PC}
PRECISIONS = {"fp64": FP64, "mixed": MIXED}
KERNEL_CLASSES = ("stats", "select", "push", "pull", "topk", "refresh", "sweep")

_STATUS = {0: "RLGL_OK", 1: "RLGL_EINVAL", 2: "RLGL_ENOTSTOCHASTIC", 3: "RLGL_ENOMEM",
           4: "RLGL_ECUDA", 5: "RLGL_EDEGENERATE", 6: "RLGL_ENOCONV", 7: "RLGL_ETIMEOUT"}


class RLGLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = _STATUS.get(status, str(status))


class Params(ctypes.Structure):
    _fields_ = [("theta_scale", ctypes.c_double), ("r", ctypes.c_int32),
                ("top_frac", ctypes.c_double), ("pull_crossover", ctypes.c_double),
                ("safety_every", ctypes.c_int32), ("refresh_factor", ctypes.c_double),
                ("time_limit_s", ctypes.c_double), ("rr_blocks", ctypes.c_int64),
                ("pc_frac", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("persistent", ctypes.c_int32), ("barrier_limit_s", ctypes.c_double),
                ("test_skip_barrier", ctypes.c_int32), ("stall_moves", ctypes.c_int32),
                ("theta_lag", ctypes.c_int32), ("batch_block", ctypes.c_int32)]


class StepInfo(ctypes.Structure):
    _fields_ = [("green", ctypes.c_int64), ("edges_pushed", ctypes.c_int64),
                ("mode", ctypes.c_int32), ("theta", ctypes.c_double),
                ("l1_cash", ctypes.c_double), ("sum_cash", ctypes.c_double),
                ("sum_hist", ctypes.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveInfo(ctypes.Structure):
    _fields_ = [("moves", ctypes.c_int64), ("edges_pushed", ctypes.c_int64),
                ("green_total", ctypes.c_int64), ("push_moves", ctypes.c_int64),
                ("pull_moves", ctypes.c_int64), ("refreshes", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("resid", ctypes.c_double), ("l1_cash", ctypes.c_double),
                ("sum_hist", ctypes.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MoveRecord(ctypes.Structure):
    _fields_ = [("move", ctypes.c_int64), ("green", ctypes.c_int64),
                ("edges_pushed", ctypes.c_int64), ("mode", ctypes.c_int32),
                ("theta", ctypes.c_double), ("l1_cash", ctypes.c_double),
                ("sum_hist", ctypes.c_double), ("phase_us", ctypes.c_float * 6)]

    def asdict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_us"] = list(self.phase_us)
        return d


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_I64, _I32, _D, _VP = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
_ST = ctypes.c_int
SIGNATURES = {
    "rlgl_default_params": (_ST, [ctypes.POINTER(Params)]),
    "rlgl_create": (_ST, [_I64, _I64, _VP, _VP, _VP, _VP, _I32, _I32, _VP, ctypes.POINTER(_VP)]),
    "rlgl_create_from_state": (_ST, [_I64, _I64, _VP, _VP, _VP, _VP, _VP, _I32, _I32, _VP,
                                     ctypes.POINTER(_VP)]),
    "rlgl_batch_create": (_ST, [_I64, _VP, _I64, _I64, _VP, _VP, _VP, _I32, _I32, _VP,
                                ctypes.POINTER(_VP)]),
    "rlgl_batch_set_tol": (_ST, [_VP, _VP]),
    "rlgl_batch_chains": (_ST, [_VP, _VP, _VP, _VP]),
    "rlgl_reset": (_ST, [_VP, _VP, _I32]),
    "rlgl_set_masks": (_ST, [_VP, _VP, _I64, _I32]),
    "rlgl_step": (_ST, [_VP, _I32, _D, ctypes.POINTER(StepInfo)]),
    "rlgl_solve": (_ST, [_VP, _I32, _D, _D, _I64, ctypes.POINTER(SolveInfo)]),
    "rlgl_solve_async": (_ST, [_VP, _I32, _D, _D, _I64]),
    "rlgl_query": (_ST, [_VP, ctypes.POINTER(_I32)]),
    "rlgl_wait": (_ST, [_VP, ctypes.POINTER(SolveInfo)]),
    "rlgl_estimate": (_ST, [_VP, _VP, _I32]),
    "rlgl_estimate_range": (_ST, [_VP, _I64, _I64, _VP, _I32]),
    "rlgl_get_state": (_ST, [_VP, _VP, _VP, _I32]),
    "rlgl_invariant_residual": (_ST, [_VP, ctypes.POINTER(_D)]),
    "rlgl_refresh": (_ST, [_VP, ctypes.POINTER(_D)]),
    "rlgl_set_params": (_ST, [_VP, ctypes.POINTER(Params)]),
    "rlgl_get_params": (_ST, [_VP, ctypes.POINTER(Params)]),
    "rlgl_profile": (_ST, [_VP, _I32]),
    "rlgl_kernel_times": (_ST, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "rlgl_profile_moves": (_ST, [_VP, _I32, _D, _I64]),
    "rlgl_profile_sweep": (_ST, [_VP, _I32, _D, _I64]),
    "rlgl_move_log": (_ST, [_VP, ctypes.POINTER(MoveRecord), _I64, ctypes.POINTER(_I64)]),
    "rlgl_invariant_residual_noalloc": (_ST, [_I64, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                              _VP]),
    "rlgl_footprint": (_I64, [_I64, _I64, _I32, _I32, _I64]),
    "rlgl_release_retired": (_I64, []),
    "rlgl_stream": (_VP, [_VP]),
    "rlgl_last_error": (ctypes.c_char_p, [_VP]),
    "rlgl_status_string": (ctypes.c_char_p, [_ST]),
    "rlgl_destroy": (None, [_VP]),
}


def load(build_if_missing: bool = True):
    """Loads librlgl.so (building it with nvcc when missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise ImportError(f"CUDA library not built: {_build.LIB}")
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(lib, ctx, status):
    if status != 0:
        msg = lib.rlgl_last_error(ctx)
        raise RLGLError(status, msg.decode() if msg else "")


def _ptr(a, dtype=None):
    """(pointer, memspace, keepalive) of a numpy array or torch tensor."""
    if a is None:
        return None, HOST, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if dtype is not None:
                if not isinstance(dtype, torch.dtype):
                    dtype = _np_dtype(np.dtype(dtype).type)
                a = a.to(dtype=dtype)
            a = a.contiguous()
            return a.data_ptr(), (DEVICE if a.is_cuda else HOST), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, HOST, arr


def _like(x, ref):
    """x (numpy array or torch tensor, or None) in the memory space of ref."""
    if x is None:
        return None
    if _is_torch(ref):
        import torch
        t = x if _is_torch(x) else torch.from_numpy(np.ascontiguousarray(x))
        return t.to(device=ref.device)
    if _is_torch(x):
        return x.detach().cpu().numpy()
    return x


def _np_dtype(t):
    import torch
    return {np.int64: torch.int64, np.int32: torch.int32, np.float32: torch.float32,
            np.float64: torch.float64, np.uint8: torch.uint8}[t]


class Chain:
    """One chain on the GPU: wraps an rlgl_ctx.

    csr: an object with n, row_ptr (int64), col (int32), w (float32 or None);
    numpy arrays (copied from host) or CUDA torch tensors (copied on device).
    """

    def __init__(self, csr, m0=None, precision="fp64", stream=None, c=None, h=None,
                 node_ptr=None):
        self.lib = load()
        self.n = int(csr.n)
        self.nnz = int(csr.row_ptr[-1])
        self.precision = precision
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        is_torch = _is_torch(csr.row_ptr)
        cv = (lambda t: _np_dtype(t)) if is_torch else (lambda t: t)
        # m0 / c / h are read from the CSR's memory space: bring them there
        m0, c, h = (_like(x, csr.row_ptr) for x in (m0, c, h))
        rp, sp, k1 = _ptr(csr.row_ptr, cv(np.int64))
        cp, _, k2 = _ptr(csr.col, cv(np.int32))
        wp, _, k3 = _ptr(csr.w, cv(np.float32))
        sptr = _stream_ptr(stream)
        out = _VP()
        self.nchains = 1
        if node_ptr is not None:
            npp, _, k6 = _ptr(_like(node_ptr, csr.row_ptr), cv(np.int64))
            self.nchains = int(len(node_ptr)) - 1
            st = self.lib.rlgl_batch_create(self.nchains, npp, self.n, self.nnz, rp, cp, wp, prec, sp,
                                            sptr, ctypes.byref(out))
        elif c is not None:
            c_p, _, k4 = _ptr(c, cv(np.float64))
            h_p, _, k5 = _ptr(h, cv(np.float64))
            st = self.lib.rlgl_create_from_state(self.n, self.nnz, rp, cp, wp, c_p, h_p, prec, sp,
                                                 sptr, ctypes.byref(out))
        else:
            m_p, _, k4 = _ptr(m0, cv(np.float64))
            st = self.lib.rlgl_create(self.n, self.nnz, rp, cp, wp, m_p, prec, sp, sptr,
                                      ctypes.byref(out))
        _check(self.lib, None, st)
        self.ctx = out.value

    # ---------------------------------------------------------------- API
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.rlgl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _c(self, st):
        _check(self.lib, self.ctx, st)

    @property
    def stream(self) -> int:
        return int(self.lib.rlgl_stream(self.ctx) or 0)

    def reset(self, m0=None):
        p, sp, keep = _ptr(m0, np.float64 if not _is_torch(m0) else None)
        self._c(self.lib.rlgl_reset(self.ctx, p, sp))

    def set_masks(self, masks):
        masks = masks if _is_torch(masks) else np.ascontiguousarray(masks, dtype=np.uint8)
        period = int(np.prod(masks.shape)) // self.n
        p, sp, keep = _ptr(masks)
        self._c(self.lib.rlgl_set_masks(self.ctx, p, period, sp))

    def step(self, schedule="threshold", theta: float = 0.0, info: bool = True):
        si = StepInfo()
        self._c(self.lib.rlgl_step(self.ctx, _sched(schedule), float(theta),
                                   ctypes.byref(si) if info else None))
        return si.asdict() if info else None

    def solve(self, schedule="threshold", theta: float = 0.0, tol: float = 1e-12,
              max_steps: int = 100000, raise_on_noconv: bool = True):
        si = SolveInfo()
        st = self.lib.rlgl_solve(self.ctx, _sched(schedule), float(theta), float(tol),
                                 int(max_steps), ctypes.byref(si))
        res = si.asdict()
        res["status"] = _STATUS.get(st, st)
        # ENOCONV / EDEGENERATE / ETIMEOUT end a solve normally; raise only
        # when asked to
        if st != 0 and (raise_on_noconv or st not in (5, 6, 7)):
            self._c(st)
        return res

    def solve_async(self, schedule="threshold", theta: float = 0.0, tol: float = 1e-12,
                    max_steps: int = 100000):
        self._c(self.lib.rlgl_solve_async(self.ctx, _sched(schedule), float(theta), float(tol),
                                          int(max_steps)))

    def query(self) -> bool:
        f = ctypes.c_int32()
        self._c(self.lib.rlgl_query(self.ctx, ctypes.byref(f)))
        return bool(f.value)

    def wait(self, raise_on_noconv: bool = True):
        si = SolveInfo()
        st = self.lib.rlgl_wait(self.ctx, ctypes.byref(si))
        res = si.asdict()
        res["status"] = _STATUS.get(st, st)
        if st != 0 and (raise_on_noconv or st not in (5, 6, 7)):
            self._c(st)
        return res

    def estimate(self, out=None):
        if out is None:
            out = np.empty(self.n, dtype=np.float64)
        p, sp, keep = _ptr(out)
        self._c(self.lib.rlgl_estimate(self.ctx, p, sp))
        return out

    def estimate_range(self, lo: int, hi: int, out=None):
        """pi_hat over the nodes [lo, hi), normalised over them."""
        if out is None:
            out = np.empty(hi - lo, dtype=np.float64)
        p, sp, keep = _ptr(out)
        self._c(self.lib.rlgl_estimate_range(self.ctx, lo, hi, p, sp))
        return out

    def set_chain_tol(self, tol):
        t = np.ascontiguousarray(tol, dtype=np.float64)
        self._c(self.lib.rlgl_batch_set_tol(self.ctx, t.ctypes.data))

    def chains(self):
        """Per chain of a batch: (status, moves, residual)."""
        stt = np.empty(self.nchains, np.int32)
        mv = np.empty(self.nchains, np.int64)
        rs = np.empty(self.nchains, np.float64)
        self._c(self.lib.rlgl_batch_chains(self.ctx, stt.ctypes.data, mv.ctypes.data, rs.ctypes.data))
        return stt, mv, rs

    def get_state(self):
        c = np.empty(self.n)
        h = np.empty(self.n)
        self._c(self.lib.rlgl_get_state(self.ctx, c.ctypes.data, h.ctypes.data, HOST))
        return c, h

    def invariant_residual(self) -> float:
        v = ctypes.c_double()
        self._c(self.lib.rlgl_invariant_residual(self.ctx, ctypes.byref(v)))
        return v.value

    def refresh(self) -> float:
        v = ctypes.c_double()
        self._c(self.lib.rlgl_refresh(self.ctx, ctypes.byref(v)))
        return v.value

    def get_params(self) -> Params:
        p = Params()
        self._c(self.lib.rlgl_get_params(self.ctx, ctypes.byref(p)))
        return p

    def set_params(self, **kw):
        p = self.get_params()
        for k, v in kw.items():
            setattr(p, k, v)
        self._c(self.lib.rlgl_set_params(self.ctx, ctypes.byref(p)))

    def profile(self, mode: int):
        self._c(self.lib.rlgl_profile(self.ctx, int(mode)))

    def profile_moves(self, schedule, theta: float, moves: int):
        """Eager moves with exact per-kernel CUDA-event timings; returns
        kernel_times() accumulated so far."""
        self._c(self.lib.rlgl_profile_moves(self.ctx, _sched(schedule), float(theta), int(moves)))
        return self.kernel_times()

    def profile_sweep(self, schedule, theta: float, moves: int):
        """`moves` moves of the persistent sweep launched eagerly, each launch
        timed with CUDA events (class "sweep"); returns kernel_times()."""
        self._c(self.lib.rlgl_profile_sweep(self.ctx, _sched(schedule), float(theta), int(moves)))
        return self.kernel_times()

    def move_log(self, count: int):
        buf = (MoveRecord * int(count))()
        n = ctypes.c_int64()
        self._c(self.lib.rlgl_move_log(self.ctx, buf, int(count), ctypes.byref(n)))
        return [buf[i].asdict() for i in range(n.value)]

    def kernel_times(self):
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        n = (ctypes.c_int64 * len(KERNEL_CLASSES))()
        self._c(self.lib.rlgl_kernel_times(self.ctx, ms, n))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_CLASSES)}


def _is_torch(a) -> bool:
    try:
        import torch
        return isinstance(a, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _sched(s) -> int:
    return SCHEDULES[s] if isinstance(s, str) else int(s)


def status_name(code: int) -> str:
    """The rlgl_status name of a status code (a chain's, from Chain.chains())."""
    return _STATUS.get(code, str(code))


def footprint(n: int, nnz: int, weighted: bool, precision="mixed", n_chains: int = 1) -> int:
    """Device bytes a context holds (rlgl_footprint)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return int(load().rlgl_footprint(n, nnz, int(weighted), prec, n_chains))


def release_retired() -> int:
    """Destroys the solve graphs of destroyed contexts (rlgl_release_retired)."""
    return int(load().rlgl_release_retired())


def default_params() -> Params:
    p = Params()
    _check(load(), None, load().rlgl_default_params(ctypes.byref(p)))
    return p
