"""The stale threshold (params.theta_lag = 1; Sec. 6 lets the threshold of
RLGL_Theta be updated less often) on the persistent sweep, through the
C-ABI, against the oracle's variant of Alg. 1 (oracle_solve with
theta_lag = 1) on the same seeded chains. FP64 trajectories agree up to the
order of floating-point additions; the MIXED path re-derives its cash and
starts each re-launch with a fresh threshold, so it is held to the
stationary law instead."""
import numpy as np
import pytest

import oracle
from paper_2008_02710_gb300 import synth

pytestmark = pytest.mark.gpu

FP64_PI_TOL = 1e-12
SCHEDS = {"all_green": oracle.ALL_GREEN, "threshold": oracle.THRESHOLD,
          "link_threshold": oracle.LINK_THRESHOLD, "pc": oracle.PC, "block_rr": oracle.BLOCK_RR}


def Chain(*a, **k):
    from paper_2008_02710_gb300.rlgl import Chain as C
    return C(*a, **k)


@pytest.fixture(scope="module")
def tiny():
    csr = synth.tiny_chain(1000, seed=1)
    p = oracle.transition_probs(csr)
    return csr, p, oracle.gth(oracle.dense_P(csr, p))


@pytest.fixture(scope="module")
def medium():
    # 2^14 nodes, ~300k weighted edges: many push chunks, hub rows
    csr = synth.rmat_chain(14, 16, seed=5, weighted=True)
    return csr, oracle.transition_probs(csr)


KW = dict(theta_scale=0.5, pc_frac=0.2, seed=3, rr_blocks=5)


@pytest.mark.parametrize("sched", ["threshold", "link_threshold", "pc", "all_green", "block_rr"])
def test_solve_tiny_fp64_vs_oracle(tiny, sched):
    csr, p, ref = tiny
    pi_or, C, H, info_or = oracle.run(csr, sched=SCHEDS[sched], tol=1e-12, max_steps=200000,
                                      theta_lag=1, **KW)
    with Chain(csr) as ch:
        ch.set_params(theta_lag=1, **KW)
        info = ch.solve(sched, tol=1e-12, max_steps=200000)
        pi_tol = ch.estimate()
        ch.reset()
        ch.solve(sched, tol=0.0, max_steps=info_or["moves"], raise_on_noconv=False)
        pi = ch.estimate()
        assert ch.get_params().persistent == 1
    assert info["status"] == "RLGL_OK"
    assert abs(info["moves"] - info_or["moves"]) <= max(1, info_or["moves"] // 1000)
    if info["moves"] == info_or["moves"]:
        # the reported residual is the tested ||C_t||_1 over H_{t+1} 1
        assert info["resid"] == pytest.approx(info_or["resid"], rel=1e-6)
    assert np.abs(pi - pi_or).sum() <= FP64_PI_TOL
    assert np.abs(pi_tol - ref).sum() <= 1e-11


@pytest.mark.parametrize("sched", ["threshold", "link_threshold"])
def test_solve_medium_fp64_vs_oracle(medium, sched):
    csr, p = medium
    # tol as in the plain-rule test: both sides end close enough to pi* that
    # a green set flipped by rounding early on has died out
    pi_or, C, H, info_or = oracle.run(csr, sched=SCHEDS[sched], tol=1e-12, max_steps=200000,
                                      theta_lag=1, theta_scale=0.5)
    with Chain(csr) as ch:
        ch.set_params(theta_lag=1, theta_scale=0.5)
        info = ch.solve(sched, tol=1e-12, max_steps=200000)
        ch.reset()
        ch.solve(sched, tol=0.0, max_steps=info_or["moves"], raise_on_noconv=False)
        pi = ch.estimate()
        inv = ch.invariant_residual()
    assert info["status"] == "RLGL_OK"
    assert abs(info["moves"] - info_or["moves"]) <= max(1, info_or["moves"] // 1000)
    assert np.abs(pi - pi_or).sum() <= FP64_PI_TOL
    assert inv <= 1e-13 * np.abs(H).sum()


def test_first_moves_share_theta_and_skip_the_statistics_pass(medium):
    """Moves 1 and 2 take their threshold from the same cash (C_1): equal
    thetas to the bit; later moves run without a statistics pass (no stats
    time, no wait at its barrier in the move log); the state after 5 moves
    is the oracle's."""
    csr, p = medium
    C, H = oracle.initial_step(csr, p)
    oracle.solve(csr, p, C, H, sched=oracle.LINK_THRESHOLD, theta_scale=0.5, tol=0.0, max_steps=5,
                 theta_lag=1)
    with Chain(csr) as ch:
        ch.set_params(theta_lag=1, theta_scale=0.5)
        ch.profile(2)
        ch.profile_sweep("link_threshold", 0.0, 5)
        log = ch.move_log(5)
        pi = ch.estimate()
    assert [r["move"] for r in log] == list(range(5))
    assert log[1]["theta"] == log[0]["theta"] > 0
    assert log[2]["theta"] != log[1]["theta"]
    assert log[0]["phase_us"][0] > 0
    assert all(r["phase_us"][0] == 0.0 and r["phase_us"][1] == 0.0 for r in log[1:])
    assert np.abs(pi - H / H.sum()).sum() <= FP64_PI_TOL


def test_exact_move_count_and_resume(tiny):
    """tol 0 stops after exactly max_steps moves; the second call starts with
    a fresh threshold, as the oracle's second call does."""
    csr, p, _ = tiny
    C, H = oracle.initial_step(csr, p)
    oracle.solve(csr, p, C, H, sched=oracle.LINK_THRESHOLD, theta_scale=0.5, tol=0.0, max_steps=13,
                 theta_lag=1)
    oracle.solve(csr, p, C, H, sched=oracle.LINK_THRESHOLD, theta_scale=0.5, tol=0.0, max_steps=17,
                 theta_lag=1, move0=13)
    with Chain(csr) as ch:
        ch.set_params(theta_lag=1, theta_scale=0.5)
        i1 = ch.solve("link_threshold", tol=0.0, max_steps=13, raise_on_noconv=False)
        i2 = ch.solve("link_threshold", tol=0.0, max_steps=17, raise_on_noconv=False)
        c, h = ch.get_state()
    assert (i1["moves"], i2["moves"]) == (13, 17)
    assert i1["status"] == i2["status"] == "RLGL_ENOCONV"
    assert np.abs(h - H).max() <= 1e-13 * np.abs(H).max()
    assert np.abs(c - C).max() <= 1e-13 * np.abs(C).max() + 1e-18


@pytest.mark.parametrize("sched", ["threshold", "link_threshold", "pc"])
def test_mixed_converges_to_the_stationary_law(tiny, medium, sched):
    csr, p, ref = tiny
    with Chain(csr, precision="mixed") as ch:
        ch.set_params(theta_lag=1, **KW)
        info = ch.solve(sched, tol=1e-9, max_steps=200000)
        pi = ch.estimate()
        resid = ch.invariant_residual()
    assert info["status"] == "RLGL_OK"
    assert np.abs(pi - ref).sum() <= 1e-6
    assert resid <= 1e-6
    csr, p = medium
    law, _, delta = oracle.power_iteration(csr, p, tol=1e-13, maxit=200000)
    assert delta <= 1e-13
    with Chain(csr, precision="mixed") as a:
        a.set_params(theta_lag=1, **KW)
        ia = a.solve(sched, tol=1e-10, max_steps=200000)
        assert ia["status"] == "RLGL_OK"
        assert np.abs(a.estimate() - law).sum() <= 1e-6


def test_rejected_where_the_sweep_does_not_run(tiny):
    from paper_2008_02710_gb300.rlgl import RLGLError
    csr, _, _ = tiny
    with Chain(csr) as ch:
        ch.set_params(theta_lag=1, persistent=0)
        with pytest.raises(RLGLError) as e:
            ch.solve("threshold", tol=1e-9)
        assert e.value.name == "RLGL_EINVAL"
        ch.set_params(persistent=1)
        with pytest.raises(RLGLError) as e:
            ch.solve("topfrac", 0.05, tol=1e-9)
        assert e.value.name == "RLGL_EINVAL"
        with pytest.raises(RLGLError):
            ch.set_params(theta_lag=2)
        # single steps ignore it
        ch.step("threshold")
    big, node_ptr = synth.stack_chains([synth.tiny_chain(200, seed=s) for s in (1, 2)])
    with Chain(big, node_ptr=node_ptr) as ch:
        ch.set_params(theta_lag=1)
        with pytest.raises(RLGLError) as e:
            ch.solve("threshold", tol=1e-9)
        assert e.value.name == "RLGL_EINVAL"
