"""Batch mode (many independent chains in one context, one launch per
kernel over a block-diagonal CSR) against the FP64 oracle run on each chain
alone."""
import numpy as np
import pytest

import oracle
from paper_2008_02710_gb300 import synth

pytestmark = pytest.mark.gpu


def Chain(*a, **k):
    from paper_2008_02710_gb300.rlgl import Chain as C
    return C(*a, **k)


@pytest.fixture(scope="module")
def parts():
    chains = [synth.tiny_chain(n, seed=s) for n, s in ((50, 1), (700, 2), (7, 3), (1000, 4), (300, 5))]
    chains.append(synth.two_wheels())
    return chains


def _weighted(c):
    return c if c.w is not None else synth.CSR(c.n, c.row_ptr, c.col, np.ones(c.nnz, np.float32))


@pytest.mark.parametrize("sched", ["link_threshold", "threshold", "all_green"])
def test_batch_solve_matches_each_chain_alone_fp64(parts, sched):
    parts = [_weighted(c) for c in parts]
    batch, node_ptr = synth.stack_chains(parts)
    with Chain(batch, node_ptr=node_ptr) as ch:
        ch.set_params(theta_scale=0.5)
        info = ch.solve(sched, tol=1e-12, max_steps=100000)
        pi = ch.estimate()
        status, moves, resid = ch.chains()
    assert info["status"] == "RLGL_OK"
    assert np.all(status == 0) and np.all(resid < 1e-12)
    sc = {"link_threshold": oracle.LINK_THRESHOLD, "threshold": oracle.THRESHOLD,
          "all_green": oracle.ALL_GREEN}[sched]
    for k, c in enumerate(parts):
        seg = pi[node_ptr[k]:node_ptr[k + 1]]
        p = oracle.transition_probs(c)
        ref = oracle.gth(oracle.dense_P(c, p))
        pi_or, C, H, info_or = oracle.run(c, sched=sc, theta_scale=0.5, tol=1e-12, max_steps=100000)
        assert abs(seg.sum() - 1) < 1e-13
        assert np.abs(seg - ref).sum() <= 1e-10, k  # residual 1e-12 times the mixing factor
        assert abs(int(moves[k]) - info_or["moves"]) <= 1, (k, moves[k], info_or["moves"])
        assert np.abs(seg - pi_or).sum() <= 1e-11, k


def test_batch_same_as_alone_gpu(parts):
    """Each chain's result in the mix equals its result solved alone."""
    parts = [_weighted(c) for c in parts]
    batch, node_ptr = synth.stack_chains(parts)
    with Chain(batch, node_ptr=node_ptr) as ch:
        ch.set_params(theta_scale=0.5)
        ch.solve("link_threshold", tol=1e-12, max_steps=100000)
        pi = ch.estimate()
        _, moves, _ = ch.chains()
    for k, c in enumerate(parts):
        with Chain(c) as one:
            one.set_params(theta_scale=0.5)
            inf = one.solve("link_threshold", tol=1e-12, max_steps=100000)
            alone = one.estimate()
        assert abs(inf["moves"] - int(moves[k])) <= 1
        assert np.abs(alone - pi[node_ptr[k]:node_ptr[k + 1]]).sum() <= 1e-11


def test_batch_per_chain_tolerance_and_mixed(parts):
    parts = [_weighted(c) for c in parts]
    batch, node_ptr = synth.stack_chains(parts)
    tols = np.array([1e-4, 1e-6, 1e-8, 1e-9, 1e-6, 1e-10])
    with Chain(batch, node_ptr=node_ptr, precision="mixed") as ch:
        ch.set_chain_tol(tols)
        info = ch.solve("link_threshold", tol=-1.0, max_steps=100000)
        pi = ch.estimate()
        status, moves, resid = ch.chains()
    assert info["status"] == "RLGL_OK" and np.all(status == 0)
    assert np.all(resid < tols)
    # looser tolerances stop earlier
    assert moves[0] < moves[3]
    for k, c in enumerate(parts):
        ref = oracle.gth(oracle.dense_P(c, oracle.transition_probs(c)))
        if tols[k] <= 1e-8:
            assert np.abs(pi[node_ptr[k]:node_ptr[k + 1]] - ref).sum() <= 1e-6


def test_batch_one_move_per_chain_threshold(parts):
    """One move of the batch = one oracle move of each chain with its own
    threshold."""
    parts = [_weighted(c) for c in parts]
    batch, node_ptr = synth.stack_chains(parts)
    with Chain(batch, node_ptr=node_ptr) as ch:
        for _ in range(4):
            ch.step("threshold", info=False)
        c0, h0 = ch.get_state()
        ch.step("threshold", info=False)
        c1, h1 = ch.get_state()
    for k, c in enumerate(parts):
        a, b = node_ptr[k], node_ptr[k + 1]
        p = oracle.transition_probs(c)
        g, th = oracle.select(c0[a:b], oracle.THRESHOLD)
        C, H = c0[a:b].copy(), h0[a:b].copy()
        oracle.move(c, p, g, C, H)
        assert np.abs(h1[a:b] - H).max() <= 1e-15 * max(1.0, np.abs(H).max())
        assert np.abs(c1[a:b] - C).max() <= 1e-13 * max(1e-300, np.abs(c0[a:b]).max())


def test_batch_rejects_edges_between_chains(parts):
    from paper_2008_02710_gb300.rlgl import RLGLError
    batch, node_ptr = synth.stack_chains([_weighted(c) for c in parts[:2]])
    col = batch.col.copy()
    col[0] = batch.n - 1  # an edge of chain 0 into chain 1
    bad = synth.CSR(batch.n, batch.row_ptr, col, batch.w)
    with pytest.raises(RLGLError) as e:
        Chain(bad, node_ptr=node_ptr)
    assert e.value.name == "RLGL_EINVAL"
    with pytest.raises(RLGLError):
        with Chain(batch, node_ptr=node_ptr) as ch:
            ch.step("topfrac", 0.1)


def test_persistent_batch_matches_phase_kernels_and_block_sizes(parts):
    """The whole batch solve in one persistent launch (each chain its own
    stop, per-chain frontier regions and merge-path tiles) gives, for every
    block size it is built for, the result of the one-kernel-per-phase batch
    path, chain by chain."""
    parts = [_weighted(c) for c in parts]
    batch, node_ptr = synth.stack_chains(parts)
    with Chain(batch, node_ptr=node_ptr) as ch:
        ch.set_params(theta_scale=0.5, persistent=0)
        ch.solve("link_threshold", tol=1e-12, max_steps=100000)
        ref = ch.estimate()
        _, ref_moves, _ = ch.chains()
        for bb in (128, 256, 512):
            ch.reset()
            ch.set_params(persistent=1, batch_block=bb)
            info = ch.solve("link_threshold", tol=1e-12, max_steps=100000)
            pi = ch.estimate()
            status, moves, resid = ch.chains()
            assert info["status"] == "RLGL_OK" and np.all(status == 0), bb
            assert np.all(np.abs(moves - ref_moves) <= 1), (bb, moves, ref_moves)
            assert info["moves"] == moves.max()
            for k in range(len(parts)):
                a, b = node_ptr[k], node_ptr[k + 1]
                assert np.abs(pi[a:b] - ref[a:b]).sum() <= 1e-11, (bb, k)


@pytest.fixture(scope="module")
def lopsided():
    """One chain much larger than the rest (it gets a group of several
    blocks in the persistent launch) among small ones."""
    big = synth.rmat_chain_n(120000, 12, seed=9)
    small = [synth.tiny_chain(n, seed=s) for n, s in ((100, 1), (333, 2), (57, 3), (1000, 4))]
    return [_weighted(c) for c in [small[0], big] + small[1:]]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_persistent_batch_large_chain_in_a_group(lopsided, prec):
    batch, node_ptr = synth.stack_chains(lopsided)
    with Chain(batch, node_ptr=node_ptr, precision=prec) as ch:
        ch.set_params(theta_scale=0.5)
        info = ch.solve("link_threshold", tol=1e-12 if prec == "fp64" else 1e-9, max_steps=100000)
        pi = ch.estimate()
        status, moves, resid = ch.chains()
    assert info["status"] == "RLGL_OK" and np.all(status == 0)
    for k, c in enumerate(lopsided):
        a, b = node_ptr[k], node_ptr[k + 1]
        p = oracle.transition_probs(c)
        law, _, _ = oracle.power_iteration(c, p, tol=1e-14, maxit=200000)
        bound = 1e-10 if prec == "fp64" else 1e-6
        assert np.abs(pi[a:b] - law).sum() <= bound, (k, np.abs(pi[a:b] - law).sum())
        if prec == "fp64":
            pi_or, _, _, info_or = oracle.run(c, sched=oracle.LINK_THRESHOLD, theta_scale=0.5, tol=1e-12,
                                              max_steps=100000)
            assert abs(int(moves[k]) - info_or["moves"]) <= max(1, info_or["moves"] // 1000), k


def test_persistent_batch_group_wait_is_bounded(lopsided):
    """A member of the large chain's group leaves before its first barrier
    (test hook): the others give up after the limit, that chain ends with
    RLGL_ETIMEOUT, the other chains converge, and the context solves
    normally afterwards."""
    batch, node_ptr = synth.stack_chains(lopsided)
    with Chain(batch, node_ptr=node_ptr) as ch:
        ch.set_params(theta_scale=0.5, barrier_limit_s=0.05, test_skip_barrier=1)
        info = ch.solve("link_threshold", tol=1e-10, max_steps=100000, raise_on_noconv=False)
        status, _, _ = ch.chains()
        assert info["status"] == "RLGL_ETIMEOUT"
        # the large chain's group lost a member; chains of one block are
        # untouched (the 1000-node chain may get a small group too)
        assert status[1] == 7 and np.all(status[[0, 2, 3]] == 0) and status[4] in (0, 7)
        ch.set_params(test_skip_barrier=0, barrier_limit_s=2.0)
        ch.reset()
        info = ch.solve("link_threshold", tol=1e-10, max_steps=100000)
        status, _, _ = ch.chains()
        assert info["status"] == "RLGL_OK" and np.all(status == 0)
