"""rlgl_invariant_residual_noalloc: the cash-balance residual for callers
that may not allocate device memory (device memory owned by another
framework's pool, for example). It is called here through the C
ABI on plain device buffers and checked against the oracle's residual
||C - C_0 - H (P - I)||_1 (Eq. recursion_H_res) and against the context's
own rlgl_invariant_residual, on calls in a row on different chains (a call
must not see an earlier call's data), with and without weights and C_0.
Inputs the kernels must refuse (a column index out of range, an empty row,
a row whose weights sum to zero) give NaN; every such index is one the
kernels check before any access."""
import numpy as np
import pytest

import oracle
from paper_2008_02710_gb300 import rlgl, synth

pytestmark = pytest.mark.gpu

MAX_NODES = 1 << 20


def _budget(csr, c, h, c0=None):
    """FP64 rounding budget of the residual: every node j sums indeg_j + 4
    terms whose magnitudes add up to |c_j| + |c0_j| + |h_j| + (|h| P)_j."""
    p = oracle.transition_probs(csr)
    rows = np.repeat(np.arange(csr.n), np.diff(csr.row_ptr))
    hp_abs = np.zeros(csr.n)
    np.add.at(hp_abs, csr.col, np.abs(h[rows]) * p)
    indeg = np.bincount(csr.col, minlength=csr.n)
    mag = np.abs(c) + np.abs(h) + hp_abs + (0.0 if c0 is None else np.abs(c0))
    return float(np.sum((indeg + 5) * 2.0 ** -53 * mag))


def _call(lib, torch, n, nnz, row_ptr, col, w, c, h, c0, out):
    dev = torch.device("cuda")
    rp = torch.from_numpy(np.ascontiguousarray(row_ptr)).to(dev)
    cl = torch.from_numpy(np.ascontiguousarray(col)).to(dev)
    wd = None if w is None else torch.from_numpy(np.ascontiguousarray(w)).to(dev)
    cd = torch.from_numpy(c).to(dev)
    hd = torch.from_numpy(h).to(dev)
    c0d = None if c0 is None else torch.from_numpy(c0).to(dev)
    out.fill_(-1.0)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    free0 = torch.cuda.mem_get_info()[0]
    st = lib.rlgl_invariant_residual_noalloc(n, nnz, rp.data_ptr(), cl.data_ptr(),
                                             None if wd is None else wd.data_ptr(), cd.data_ptr(),
                                             hd.data_ptr(), None if c0d is None else c0d.data_ptr(),
                                             out.data_ptr(), stream)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    return st, float(out.item()), free0 - free1


def _state(csr, prec, moves):
    with rlgl.Chain(csr, precision=prec) as ch:
        ch.set_params(refresh_factor=0.0, theta_scale=0.5)
        for _ in range(moves):
            ch.step("link_threshold", info=False)
        c, h = ch.get_state()
        ctx_resid = ch.invariant_residual()  # the context's own entry point
    return c, h, ctx_resid


def test_noalloc_residual_matches_oracle_calls_in_a_row():
    import torch
    lib = rlgl.load()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    a = synth.rmat_chain(14, 16, seed=5, weighted=True)   # 16384 nodes, weighted
    b = synth.tiny_chain(3000, seed=2)                    # smaller chain, different size
    u = synth.rmat_chain(12, 8, seed=3)                   # unit weights (w = NULL)
    rng = np.random.default_rng(11)
    cases = [(a, "mixed", 15, None, None), (b, "fp64", 10, 17, None), (u, "mixed", 6, None, "c0"),
             (a, "fp64", 4, None, "c0")]
    leaked = []
    for k, (csr, prec, moves, plant, with_c0) in enumerate(cases):
        c, h, ctx_resid = _state(csr, prec, moves)
        c0 = None
        if with_c0:
            c0 = rng.standard_normal(csr.n) * 1e-3
            c0 -= c0.mean()
            c = c + c0  # a state resumed from C_0 != 0: the residual is unchanged
        if plant is not None:
            # a planted defect makes the FP64 residual large and known
            c = c.copy()
            c[plant] += 3e-9
        p = oracle.transition_probs(csr)
        want = oracle.invariant_residual(csr, p, c, h, c0)
        st, got, used = _call(lib, torch, csr.n, csr.nnz, csr.row_ptr, csr.col, csr.w, c, h, c0, out)
        assert st == 0
        tol = _budget(csr, c, h, c0)
        assert np.isfinite(got) and abs(got - want) <= tol, (k, got, want, tol)
        if plant is None and with_c0 is None:
            # the context's residual of the same state
            assert abs(got - ctx_resid) <= tol, k
        if plant is not None:
            assert abs(got - 3e-9) <= 1e-12
        if k > 0:
            leaked.append(used)
    # after the first call (which may load the library's device code and
    # its fixed array), no call takes device memory
    assert leaked == [0] * len(leaked)


def test_noalloc_flags_bad_rows_with_nan():
    """An out-of-range column index, an empty row and a row whose weights sum
    to zero each give NaN; a clean call after them is exact again."""
    import torch
    lib = rlgl.load()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    csr = synth.tiny_chain(500, seed=4)
    p = oracle.transition_probs(csr)
    C, H = oracle.initial_step(csr, p)
    bad_col = csr.col.copy()
    bad_col[7] = csr.n  # checked against [0, n) before any access
    empty = csr.row_ptr.copy()
    empty[3] = empty[2]  # row 2 empty, every offset still inside [0, nnz]
    zero_w = csr.w.copy()
    zero_w[csr.row_ptr[5]:csr.row_ptr[6]] = 0.0
    for rp, col, w in ((csr.row_ptr, bad_col, csr.w), (empty, csr.col, csr.w),
                       (csr.row_ptr, csr.col, zero_w)):
        st, got, _ = _call(lib, torch, csr.n, csr.nnz, rp, col, w, C, H, None, out)
        assert st == 0 and np.isnan(got)
    st, got, _ = _call(lib, torch, csr.n, csr.nnz, csr.row_ptr, csr.col, csr.w, C, H, None, out)
    assert st == 0 and abs(got - oracle.invariant_residual(csr, p, C, H)) <= _budget(csr, C, H)


def test_noalloc_rejects_too_many_nodes():
    import torch
    lib = rlgl.load()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.rlgl_invariant_residual_noalloc(MAX_NODES + 1, 10, x.data_ptr(), x.data_ptr(), None,
                                             x.data_ptr(), x.data_ptr(), None, x.data_ptr(), None)
    assert st == 1  # RLGL_EINVAL, nothing queued
