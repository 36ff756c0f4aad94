"""rlgl_invariant_residual_noalloc: the cash-balance residual for callers
that may not allocate device memory (a stream capture in progress, or device
memory owned by another framework's pool). It is called here through the C
ABI on plain device buffers and must agree with the context's own
rlgl_invariant_residual on the same state, on two calls in a row on
different chains (the second call must not see the first call's data)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2008_02710_gb300 import rlgl, synth

pytestmark = pytest.mark.gpu

MAX_NODES = 1 << 20


def _budget(csr, c, h):
    """FP64 rounding budget of the residual: every node j sums indeg_j + 3
    terms whose magnitudes add up to |c_j| + |h_j| + (|h| P)_j."""
    p = oracle.transition_probs(csr)
    rows = np.repeat(np.arange(csr.n), np.diff(csr.row_ptr))
    hp_abs = np.zeros(csr.n)
    np.add.at(hp_abs, csr.col, np.abs(h[rows]) * p)
    indeg = np.bincount(csr.col, minlength=csr.n)
    return float(np.sum((indeg + 4) * 2.0 ** -53 * (np.abs(c) + np.abs(h) + hp_abs)))


def _call(lib, csr, c, h, out, torch):
    dev = torch.device("cuda")
    rp = torch.from_numpy(csr.row_ptr).to(dev)
    col = torch.from_numpy(csr.col).to(dev)
    w = None if csr.w is None else torch.from_numpy(csr.w).to(dev)
    cd = torch.from_numpy(c).to(dev)
    hd = torch.from_numpy(h).to(dev)
    out.fill_(-1.0)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.rlgl_invariant_residual_noalloc(csr.n, csr.nnz, rp.data_ptr(), col.data_ptr(),
                                             None if w is None else w.data_ptr(), cd.data_ptr(),
                                             hd.data_ptr(), None, out.data_ptr(), stream)
    torch.cuda.synchronize()
    return st, float(out.item())


def test_noalloc_residual_matches_context_residual_two_calls():
    import torch
    lib = rlgl.load()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    a = synth.rmat_chain(14, 16, seed=5, weighted=True)   # 16384 nodes, weighted
    b = synth.tiny_chain(3000, seed=2)                    # smaller chain, different size
    cases = [(a, "mixed", 15, None), (b, "fp64", 10, 17)]
    for csr, prec, moves, plant in cases:
        with rlgl.Chain(csr, precision=prec) as ch:
            ch.set_params(refresh_factor=0.0, theta_scale=0.5)
            for _ in range(moves):
                ch.step("link_threshold", info=False)
            c, h = ch.get_state()
            expected = ch.invariant_residual()  # the context's entry point
        if plant is not None:
            # a planted defect makes the FP64 residual large and known
            c = c.copy()
            c[plant] += 3e-9
            expected += 3e-9
        st, got = _call(lib, csr, c, h, out, torch)
        assert st == 0
        tol = _budget(csr, c, h)
        assert np.isfinite(got) and abs(got - expected) <= tol, (got, expected, tol)
        if plant is not None:
            assert abs(got - 3e-9) <= 1e-12


def test_noalloc_rejects_too_many_nodes():
    import torch
    lib = rlgl.load()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.rlgl_invariant_residual_noalloc(MAX_NODES + 1, 10, x.data_ptr(), x.data_ptr(), None,
                                             x.data_ptr(), x.data_ptr(), None, x.data_ptr(), None)
    assert st == 1  # RLGL_EINVAL, nothing queued
