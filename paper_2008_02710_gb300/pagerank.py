"""PageRank through the RLGL sweep (Sec. 2.3.2).

PageRank with damping c and restart law s is the stationary law of the
chain that follows P with probability c and restarts from s otherwise
(Eq. 7). The paper embeds it in a stochastic chain P^(0) on N+1 nodes with
an auxiliary node 0: p_00 = c, p_0j = (1-c) s_j, p_i0 = 1-c and the cP
block for the original nodes. Starting from M_0 = e_0 and C_0 = 0, step 0
leaves exactly the Gauss-Southwell initial residual (1-c)s on the original
nodes and -(1-c) on node 0, and any RLGL schedule then runs on P^(0) with
the same kernels as any other chain. The PageRank vector is the original
nodes' part of the estimate, normalised.

A schedule that greens node 0 alone while the original nodes' cash stays
below the threshold moves only node 0's negative cash, which cancels the
positive cash it sends out: H 1 then falls towards 0 and the estimate
H / H 1 degenerates (the solve ends without convergence). The threshold
schedules avoid that when the first threshold lies below (1-c) s_i, as the
per-link threshold at scale 1/2 does on R-MAT graphs.
"""
from __future__ import annotations

import numpy as np

from . import rlgl
from .synth import CSR, pagerank_chain


def augmented(csr: CSR, c_num: int = 17, c_den: int = 20) -> CSR:
    """P^(0) for damping c = c_num / c_den and uniform s (integer weights,
    exact in FP32)."""
    return pagerank_chain(csr, c_num, c_den)


def solve(csr: CSR, c_num: int = 17, c_den: int = 20, tol: float = 1e-9,
          schedule: str = "link_threshold", theta_scale: float = 0.5, precision: str = "mixed",
          max_steps: int = 100000, stream=None, theta_lag: int = 0):
    """PageRank of the unit-weight graph csr: returns (pi*, solve info).
    theta_lag = 1 takes the stale threshold (see rlgl_params)."""
    aug = augmented(csr, c_num, c_den)
    m0 = np.zeros(aug.n)
    m0[0] = 1.0
    with rlgl.Chain(aug, m0=m0, precision=precision, stream=stream) as ch:
        ch.set_params(theta_scale=theta_scale, theta_lag=theta_lag)
        info = ch.solve(schedule, tol=tol, max_steps=max_steps)
        # the original nodes' part of the estimate, normalised over them
        pr = ch.estimate_range(1, aug.n)
    return pr, info
