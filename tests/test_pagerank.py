"""PageRank through the RLGL sweep on the augmented chain P^(0) (Sec.
2.3.2): pins of the construction on the CPU oracle, then the GPU."""
import numpy as np
import pytest

import oracle
from paper_2008_02710_gb300 import synth


def _pagerank_closed_form(csr, c):
    """pi* = (1 - c) s (I - c P)^-1 with uniform s (dense solve)."""
    P = oracle.dense_P(csr, oracle.transition_probs(csr))
    n = csr.n
    s = np.full(n, 1.0 / n)
    return np.linalg.solve((np.eye(n) - c * P).T, (1 - c) * s)


def test_augmented_step0_is_gauss_southwell_initialisation():
    """With M_0 = e_0, step 0 gives C_1 = (-(1-c), (1-c) s), H_1 = (1, 0):
    the initialisation of Alg. 2 on the original nodes (Sec. 2.3.2)."""
    g = synth.tiny_chain(64, seed=3)
    g = synth.CSR(g.n, g.row_ptr, g.col, None)
    aug = synth.pagerank_chain(g)
    p = oracle.transition_probs(aug)
    m0 = np.zeros(aug.n)
    m0[0] = 1.0
    C, H = oracle.initial_step(aug, p, m0)
    assert abs(C[0] + 0.15) < 1e-16
    assert np.abs(C[1:] - 0.15 / 64).max() < 1e-17
    assert H[0] == 1.0 and not H[1:].any()


@pytest.mark.parametrize("sched", [oracle.ALL_GREEN, oracle.LINK_THRESHOLD, oracle.THRESHOLD])
def test_augmented_chain_gives_pagerank(sched):
    g = synth.rmat_chain(9, 8, seed=4)
    aug = synth.pagerank_chain(g)
    m0 = np.zeros(aug.n)
    m0[0] = 1.0
    pi, C, H, info = oracle.run(aug, sched=sched, m0=m0, theta_scale=0.5, tol=1e-13,
                                max_steps=100000)
    assert info["status"] == "OK"
    ref = _pagerank_closed_form(g, 0.85)
    assert abs(pi[0] - 0.5) < 1e-12          # x_0 = sum y when p_00 = c
    y = pi[1:] / pi[1:].sum()
    assert np.abs(y - ref).sum() < 1e-11


@pytest.mark.gpu
@pytest.mark.parametrize("prec,bound", [("fp64", 1e-11), ("mixed", 1e-6)])
def test_pagerank_on_gpu(prec, bound):
    from paper_2008_02710_gb300 import pagerank
    g = synth.rmat_chain(12, 16, seed=5)
    y, info = pagerank.solve(g, tol=1e-13 if prec == "fp64" else 1e-9, precision=prec)
    assert info["status"] == "RLGL_OK"
    assert np.abs(y - _pagerank_closed_form(g, 0.85)).sum() <= bound


@pytest.mark.gpu
def test_pagerank_degenerate_schedule_on_gpu():
    """The GPU path ends the degenerate run (node 0 alone green, H 1 -> 0)
    the way the oracle does: without convergence, H 1 vanishing."""
    from paper_2008_02710_gb300.rlgl import Chain
    g = synth.tiny_chain(40, seed=2)
    aug = synth.pagerank_chain(synth.CSR(g.n, g.row_ptr, g.col, None))
    m0 = np.zeros(aug.n)
    m0[0] = 1.0
    with Chain(aug, m0=m0, precision="fp64") as ch:
        for t in range(1, 11):
            ch.step("threshold", info=False)
        _, h = ch.get_state()
        assert abs(h.sum() - 0.85 ** 10) < 1e-14
        info = ch.solve("threshold", tol=1e-12, max_steps=3000, raise_on_noconv=False)
    # The device tests |H 1| against an upper bound of sum |H| (the moved
    # mass), the oracle against sum |H| itself: the device may call the run
    # degenerate where the oracle runs out of moves. Neither converges.
    assert info["status"] in ("RLGL_ENOCONV", "RLGL_EDEGENERATE")
    assert abs(info["sum_hist"]) < 1e-9


def test_dangling_nodes_follow_restart_law():
    """Dangling rows: the normalised original-node part equals the
    eigenvector of the Google matrix whose dangling rows are s."""
    n = 40
    rng = np.random.default_rng(8)
    src, dst = [], []
    for i in range(n):
        if i % 7 == 3:
            continue                       # dangling
        for j in rng.choice(n, size=3, replace=False):
            src.append(i)
            dst.append(int(j))
    g = synth.edges_to_csr(n, np.array(src, np.int32), np.array(dst, np.int32), None)
    aug = synth.pagerank_chain(g)
    m0 = np.zeros(aug.n)
    m0[0] = 1.0
    pi, C, H, info = oracle.run(aug, sched=oracle.LINK_THRESHOLD, m0=m0, theta_scale=0.5,
                                tol=1e-14, max_steps=100000)
    assert info["status"] == "OK" and info["hsum"] > 0.1
    y = pi[1:] / pi[1:].sum()
    P = np.zeros((n, n))
    for i, j in zip(src, dst):
        P[i, j] += 1.0
    deg = P.sum(1)
    P[deg > 0] /= deg[deg > 0, None]
    P[deg == 0] = 1.0 / n
    G = 0.85 * P + 0.15 / n
    w, v = np.linalg.eig(G.T)
    ref = np.real(v[:, np.argmin(np.abs(w - 1))])
    ref /= ref.sum()
    assert np.abs(y - ref).sum() < 1e-11


def test_aux_node_alone_green_degenerates():
    """With uniform s and the |C| threshold at scale 1, only node 0 passes at
    first (|C_0| = 1 - c against a mean of 2(1 - c)/(N + 1)). Moving node 0
    alone keeps a share c of its negative cash on itself and sends the rest
    to cancel the positive cash: H 1 = c^t after t such moves, so H tends to
    0 and the estimate H / H 1 degenerates; the solve ends without
    convergence."""
    g = synth.tiny_chain(40, seed=2)
    g = synth.CSR(g.n, g.row_ptr, g.col, None)
    aug = synth.pagerank_chain(g)
    p = oracle.transition_probs(aug)
    m0 = np.zeros(aug.n)
    m0[0] = 1.0
    C, H = oracle.initial_step(aug, p, m0)
    for t in range(1, 21):
        green, _ = oracle.select(C, oracle.THRESHOLD, 1.0)
        assert green[0] == 1 and green.sum() == 1
        oracle.move(aug, p, green, C, H)
        assert abs(H.sum() - 0.85 ** t) < 1e-14
    pi, C, H, info = oracle.run(aug, sched=oracle.THRESHOLD, m0=m0, tol=1e-12, max_steps=3000)
    assert info["status"] == "ENOCONV" and abs(info["hsum"]) < 1e-9


@pytest.mark.gpu
@pytest.mark.parametrize("persistent", [1, 0])
def test_pagerank_mixed_large_hub_converges(persistent):
    """The auxiliary node takes an addition from every other node at every
    move, so its FP32 cash carries a rounding floor above the re-derivation
    trigger; the stall rule re-derives anyway and the MIXED solve reaches
    its tolerance (L1 <= 1e-6 against the oracle's power iteration)."""
    from paper_2008_02710_gb300.rlgl import Chain
    g = synth.rmat_chain(17, 16, seed=1)
    aug = synth.pagerank_chain(g)
    p = oracle.transition_probs(aug)
    ref, _, _ = oracle.power_iteration(aug, p, tol=1e-14, maxit=100000, nthreads=8)
    m0 = np.zeros(aug.n)
    m0[0] = 1.0
    with Chain(aug, m0=m0, precision="mixed") as ch:
        ch.set_params(theta_scale=0.5, persistent=persistent)
        info = ch.solve("link_threshold", tol=1e-9, max_steps=5000)
        pi = ch.estimate()
        inv = ch.invariant_residual()
    assert info["status"] == "RLGL_OK" and info["refreshes"] >= 1
    assert np.abs(pi - ref).sum() <= 1e-6
    assert inv <= 1e-8


@pytest.mark.gpu
def test_pagerank_hot_node_push_matches_oracle_moves():
    """The auxiliary node's in-links are summed per block before they reach
    its cash: one FP64 move from the GPU's state equals the oracle's move of
    that state within the FP64 rounding budget, node by node."""
    from paper_2008_02710_gb300.rlgl import Chain
    g = synth.rmat_chain(14, 16, seed=3)
    aug = synth.pagerank_chain(g)
    p = oracle.transition_probs(aug)
    m0 = np.zeros(aug.n)
    m0[0] = 1.0
    with Chain(aug, m0=m0, precision="fp64") as ch:
        ch.set_params(theta_scale=0.5, pull_crossover=10.0)  # always push
        hot_moves = 0
        for _ in range(8):
            c, h = ch.get_state()
            info = ch.step("link_threshold")
            c2, h2 = ch.get_state()
            g_ = (h2 != h).astype(np.uint8)
            assert info["mode"] == 1
            hot_moves += int(g_[0])
            C, H = c.copy(), h.copy()
            oracle.move(aug, p, g_, C, H)
            A, HA = np.abs(c), np.zeros(aug.n)
            oracle.move(aug, p, g_, A, HA)
            deg_in = np.bincount(aug.col, minlength=aug.n).astype(float)
            budget = (deg_in + 4) * 2.0 ** -53 * A + 1e-300
            assert np.all(np.abs(c2 - C) <= budget)
    assert hot_moves >= 1  # the auxiliary node was pushed at least once


@pytest.mark.gpu
@pytest.mark.parametrize("persistent", [0, 1])
def test_relabelled_hub_push_matches_oracle_moves(persistent):
    """A hub anywhere in the id range: the PageRank chain's auxiliary node
    (fed by every node) moved to a random id by a seeded relabelling. Its
    in-links are summed per block through the push's hub table; FP64 push
    moves, single steps and persistent sweeps, equal the oracle's moves node
    by node within the FP64 rounding budget."""
    from paper_2008_02710_gb300.rlgl import Chain
    aug = synth.pagerank_chain(synth.rmat_chain(14, 16, seed=3))
    n = aug.n
    perm = np.random.default_rng(4).permutation(n)  # old id -> new id
    rows = np.repeat(np.arange(n), np.diff(aug.row_ptr))
    src, dst = perm[rows], perm[aug.col]
    order = np.argsort(src, kind="stable")
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    g = synth.CSR(n, row_ptr, dst[order].astype(np.int32), aug.w[order])
    hub = int(perm[0])
    assert hub > 100
    deg_in = np.bincount(g.col, minlength=n).astype(float)
    assert deg_in[hub] == n
    grow = np.repeat(np.arange(n), np.diff(g.row_ptr))
    into_hub = g.col == hub
    p = oracle.transition_probs(g)
    m0 = np.zeros(n)
    m0[hub] = 1.0
    with Chain(g, m0=m0, precision="fp64") as ch:
        ch.set_params(theta_scale=0.5, pull_crossover=10.0, persistent=persistent)  # always push
        hub_pushes = 0
        for _ in range(8):
            c, h = ch.get_state()
            if persistent:
                ch.solve("link_threshold", tol=0.0, max_steps=1, raise_on_noconv=False)
            else:
                assert ch.step("link_threshold")["mode"] == 1
            c2, h2 = ch.get_state()
            g_ = (h2 != h).astype(np.uint8)
            hub_pushes += int(g_[grow[into_hub]].sum())  # green rows' links into the hub
            C, H = c.copy(), h.copy()
            oracle.move(g, p, g_, C, H)
            A, HA = np.abs(c), np.zeros(n)
            oracle.move(g, p, g_, A, HA)
            budget = (deg_in + 4) * 2.0 ** -53 * A + 1e-300
            assert np.all(np.abs(c2 - C) <= budget)
            assert np.array_equal(h2, H)
    assert hub_pushes > n // 4  # many links into the hub were pushed
