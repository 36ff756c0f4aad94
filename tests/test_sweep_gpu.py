"""The persistent sweep (one cooperative kernel per stretch of a solve,
grid barriers between the phases of a move) against the path with one
kernel per phase, on the same seeded chains, and its profiling entry point.
Both paths make the moves of Alg. 1; they differ only in the order in
which floating-point atomic additions land, so trajectories agree up to
rounding and the stop test may fire a move apart."""
import numpy as np
import pytest

from paper_2008_02710_gb300 import synth

pytestmark = pytest.mark.gpu


def Chain(*a, **k):
    from paper_2008_02710_gb300.rlgl import Chain as C
    return C(*a, **k)


@pytest.fixture(scope="module")
def weighted():
    # 2^14 nodes, ~300k weighted edges: many push chunks and merge-path tiles
    return synth.rmat_chain(14, 16, seed=5, weighted=True)


@pytest.fixture(scope="module")
def unweighted():
    # ragged size: not a multiple of the vector width or of a block-iteration
    return synth.rmat_chain_n(10007, 8, seed=3)


def _solve(csr, prec, sched, persistent, tol, max_steps=100000, **params):
    with Chain(csr, precision=prec) as ch:
        ch.set_params(persistent=persistent, **params)
        info = ch.solve(sched, tol=tol, max_steps=max_steps, raise_on_noconv=False)
        # the sweep was not turned off for want of a cooperative graph node
        assert ch.get_params().persistent == persistent, ch.lib.rlgl_last_error(ch.ctx)
        pi = ch.estimate()
        log = ch.move_log(min(info["moves"], 65536))
        inv = ch.invariant_residual()
    return info, pi, log, inv


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("sched", ["all_green", "threshold", "link_threshold"])
@pytest.mark.parametrize("which", ["weighted", "unweighted"])
def test_sweep_matches_phase_kernels(request, which, sched, prec):
    csr = request.getfixturevalue(which)
    tol = 1e-12 if prec == "fp64" else 1e-9
    ia, pa, la, inva = _solve(csr, prec, sched, 1, tol, theta_scale=0.5)
    ib, pb, lb, invb = _solve(csr, prec, sched, 0, tol, theta_scale=0.5)
    assert ia["status"] == ib["status"] == "RLGL_OK"
    # FP32 atomics on the MIXED path round differently with every order, so
    # long MIXED solves drift apart by a few green sets; FP64 ones hardly
    slack = 1000 if prec == "fp64" else 50
    assert abs(ia["moves"] - ib["moves"]) <= max(1, ib["moves"] // slack)
    assert abs(ia["refreshes"] - ib["refreshes"]) <= 1
    # the first moves choose the same green sets up to nodes within
    # rounding of the threshold
    for ra, rb in list(zip(la, lb))[:20]:
        assert abs(ra["green"] - rb["green"]) <= max(2, rb["green"] // 10000)
        assert ra["mode"] == rb["mode"] or abs(ra["green"] - rb["green"]) > 0
        if prec == "fp64":
            assert abs(ra["theta"] - rb["theta"]) <= 1e-12 * max(rb["theta"], 1e-300)
    bound = 1e-10 if prec == "fp64" else 2e-6
    assert np.abs(pa - pb).sum() <= bound
    assert abs(pa.sum() - 1) < 1e-12
    assert inva <= max(10 * invb, 1e-12)


def test_sweep_relaunches_for_each_rederivation(weighted):
    """MIXED with a large refresh factor re-derives the cash many times: the
    sweep returns for each and the graph launches it again."""
    ia, pa, _, inva = _solve(weighted, "mixed", "link_threshold", 1, 1e-10, refresh_factor=0.1,
                             theta_scale=0.5)
    ib, pb, _, invb = _solve(weighted, "mixed", "link_threshold", 0, 1e-10, refresh_factor=0.1,
                             theta_scale=0.5)
    assert ia["status"] == ib["status"] == "RLGL_OK"
    assert ia["refreshes"] >= 5
    assert abs(ia["refreshes"] - ib["refreshes"]) <= 1
    assert np.abs(pa - pb).sum() <= 1e-7
    assert inva <= 1e-9


def test_sweep_exact_move_count_and_resume(unweighted):
    """tol 0 stops after exactly max_steps moves; a second solve continues
    from the state the first one left."""
    with Chain(unweighted, precision="fp64") as a, Chain(unweighted, precision="fp64") as b:
        for ch in (a, b):
            ch.set_params(theta_scale=0.5)
        b.set_params(theta_scale=0.5, persistent=0)
        i1 = a.solve("link_threshold", tol=0.0, max_steps=13, raise_on_noconv=False)
        i2 = a.solve("link_threshold", tol=0.0, max_steps=17, raise_on_noconv=False)
        i3 = b.solve("link_threshold", tol=0.0, max_steps=30, raise_on_noconv=False)
        assert i1["status"] == i2["status"] == "RLGL_ENOCONV"
        assert (i1["moves"], i2["moves"], i3["moves"]) == (13, 17, 30)
        ca, ha = a.get_state()
        cb, hb = b.get_state()
    assert np.abs(ha - hb).max() <= 1e-12 * np.abs(hb).max()
    assert np.abs(ca - cb).max() <= 1e-12 * np.abs(cb).max()


def test_profile_sweep_times_the_kernel(weighted):
    with Chain(weighted, precision="mixed") as a, Chain(weighted, precision="mixed") as b:
        for ch in (a, b):
            ch.set_params(theta_scale=0.5)
        a.profile(2)
        kt = a.profile_sweep("link_threshold", 0.0, 25)
        b.solve("link_threshold", tol=0.0, max_steps=25, raise_on_noconv=False)
        assert kt["sweep"][1] >= 1 and kt["sweep"][0] > 0
        log = a.move_log(100)
        assert [r["move"] for r in log] == list(range(25))
        # every move of the sweep carries its phase timings
        assert all(min(r["phase_us"]) >= 0 and sum(r["phase_us"]) > 0 for r in log)
        _, ha = a.get_state()
        _, hb = b.get_state()
    assert np.abs(ha - hb).sum() <= 1e-6 * np.abs(hb).sum()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("which", ["weighted", "unweighted"])
def test_sweep_topfrac_threshold_is_the_kth_largest(request, which, prec):
    """TOPFRAC in the sweep (radix passes with a grid barrier each): move
    after move, theta is exactly the k-th largest |C| of the state before
    the move (k = ceil(f N)), and the green set is every nonzero node at or
    above it, ties included."""
    csr = request.getfixturevalue(which)
    f = 0.05
    k = int(np.ceil(f * csr.n))
    with Chain(csr, precision=prec) as ch:
        for m in range(12):
            c, _ = ch.get_state()
            ac = np.abs(c)
            kth = np.sort(ac)[::-1][k - 1]
            green = int(((ac >= kth) & (c != 0)).sum())
            ch.solve("topfrac", f, tol=0.0, max_steps=1, raise_on_noconv=False)
            assert ch.get_params().persistent == 1
            rec = ch.move_log(1)[-1]
            assert rec["theta"] == kth, (m, rec["theta"], kth)
            assert rec["green"] == green, (m, rec["green"], green)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sweep_topfrac_solves_like_phase_kernels(weighted, prec):
    """The same TOPFRAC solve through the sweep and through the phase
    kernels: both stop, a few moves apart at most, at the same law."""
    tol = 1e-11 if prec == "fp64" else 1e-8
    with Chain(weighted, precision=prec) as a, Chain(weighted, precision=prec) as b:
        b.set_params(persistent=0)
        ia = a.solve("topfrac", 0.05, tol=tol, max_steps=100000)
        ib = b.solve("topfrac", 0.05, tol=tol, max_steps=100000)
        pa, pb = a.estimate(), b.estimate()
    assert ia["status"] == ib["status"] == "RLGL_OK"
    # ties at the k-th value split differently once rounding differs, so
    # the two trajectories part after a few moves
    assert abs(ia["moves"] - ib["moves"]) <= max(3, ib["moves"] // 20)
    assert np.abs(pa - pb).sum() <= (1e-9 if prec == "fp64" else 2e-6)


def test_sweep_not_used_where_it_does_not_apply(weighted):
    """The stale threshold does not apply to TOPFRAC, and batches keep their
    own launch: asking for either is an error."""
    from paper_2008_02710_gb300.rlgl import RLGLError
    with Chain(weighted) as ch:
        ch.set_params(theta_lag=1)
        with pytest.raises(RLGLError) as e:
            ch.solve("topfrac", 0.05, tol=1e-10, max_steps=100000)
        assert e.value.name == "RLGL_EINVAL"
        ch.set_params(theta_lag=0)
        kt = ch.profile_sweep("topfrac", 0.05, 5)
        assert kt["sweep"][1] >= 1
    big, node_ptr = synth.stack_chains([synth.tiny_chain(300, seed=s) for s in (1, 2, 3)])
    with Chain(big, node_ptr=node_ptr) as ch:
        with pytest.raises(RLGLError):
            ch.profile_sweep("threshold", 0.0, 5)


def test_barrier_wait_is_bounded_and_context_survives(weighted):
    """One block leaves before its first barrier (test hook): the others'
    wait runs out after the limit, the solve ends with RLGL_ETIMEOUT, and
    the next solve on the same context runs normally."""
    import time
    with Chain(weighted, precision="mixed") as ch:
        ch.set_params(theta_scale=0.5, barrier_limit_s=0.05, test_skip_barrier=1)
        t0 = time.perf_counter()
        info = ch.solve("link_threshold", tol=1e-9, raise_on_noconv=False)
        dt = time.perf_counter() - t0
        assert info["status"] == "RLGL_ETIMEOUT"
        assert dt < 5.0
        assert "barrier" in ch.lib.rlgl_last_error(ch.ctx).decode()
        ch.set_params(test_skip_barrier=0, barrier_limit_s=2.0)
        ch.reset()
        info = ch.solve("link_threshold", tol=1e-9)
        assert info["status"] == "RLGL_OK"
        assert ch.get_params().persistent == 1


def test_sweep_large_chain_single_pass_select():
    """More nodes than the sweep's select cache covers (n > blocks x 1024 for FP64 cash):
    the one-pass select. 25 FP64 moves agree with the oracle's 25 moves and
    with the one-kernel-per-phase path."""
    import oracle
    csr = synth.rmat_chain_n((1 << 21) + 12345, 2, seed=11)
    p = oracle.transition_probs(csr)
    C, H = oracle.initial_step(csr, p)
    info_or = oracle.solve(csr, p, C, H, sched=oracle.LINK_THRESHOLD, theta_scale=0.5, tol=0.0,
                           max_steps=25, check_every=-1)
    pi_or = oracle.estimate(H)
    pis = []
    for persistent in (1, 0):
        with Chain(csr, precision="fp64") as ch:
            ch.set_params(theta_scale=0.5, persistent=persistent)
            info = ch.solve("link_threshold", tol=0.0, max_steps=25, raise_on_noconv=False)
            assert info["moves"] == 25 and ch.get_params().persistent == persistent
            pis.append(ch.estimate())
    assert np.abs(pis[0] - pi_or).sum() <= 1e-12
    assert np.abs(pis[0] - pis[1]).sum() <= 1e-12
    assert abs(info["edges_pushed"] - info_or["pushes"]) <= 1e-4 * info_or["pushes"]


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("theta_lag", [0, 1])
def test_sweep_large_chain_mixed_pipelined_select(theta_lag, weighted):
    """MIXED cash on more nodes than the select cache covers (n > blocks x
    2048): node ranges stream through the two shared-memory stages, handed
    out by a counter after the first two per block (with weights, s_i is
    staged beside 1/d). After 25 moves (no re-derivation yet) the FP32 cash
    has drifted from the oracle's FP64 trajectory by rounding only (~1e-6
    relative per node); a range skipped or moved twice would leave ~2e-4 of
    the mass out. Without the stale threshold the sweep also agrees with the
    one-kernel-per-phase path (both FP32) move by move."""
    import oracle
    csr = synth.rmat_chain_n((1 << 21) + 54321, 3, seed=12)
    if weighted:
        rng = np.random.default_rng(12)
        w = (rng.integers(1, 1 << 24, csr.nnz) * 2.0 ** -24).astype(np.float32)
        csr = synth.CSR(csr.n, csr.row_ptr, csr.col, w)
    p = oracle.transition_probs(csr)
    C, H = oracle.initial_step(csr, p)
    info_or = oracle.solve(csr, p, C, H, sched=oracle.LINK_THRESHOLD, theta_scale=0.5, tol=0.0,
                           max_steps=25, theta_lag=theta_lag)
    pi_or = oracle.estimate(H)
    res = []
    for persistent in ((1, 0) if theta_lag == 0 else (1,)):
        with Chain(csr, precision="mixed") as ch:
            ch.set_params(theta_scale=0.5, theta_lag=theta_lag, persistent=persistent)
            info = ch.solve("link_threshold", tol=0.0, max_steps=25, raise_on_noconv=False)
            assert info["moves"] == 25 and ch.get_params().persistent == persistent
            res.append((ch.estimate(), ch.move_log(25), info))
    pi, log, info = res[0]
    assert np.abs(pi - pi_or).sum() <= 1e-5
    assert abs(info["edges_pushed"] - info_or["pushes"]) <= 1e-3 * info_or["pushes"]
    assert all(r["green"] > 0 for r in log)
    if theta_lag == 0:
        pib, logb, _ = res[1]
        assert np.abs(pi - pib).sum() <= 2e-6
        for ra, rb in zip(log[:10], logb[:10]):
            assert abs(ra["green"] - rb["green"]) <= max(2, rb["green"] // 10000)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_power_sweep_makes_the_oracle_moves(prec):
    """The all-green sweep (one pass over the in-links a move; rows whose
    in-links cross merge-path tiles are finished after a barrier) makes the
    oracle's all-green moves: after 40 moves from step 0 the state is the
    oracle's up to rounding, on a chain whose auxiliary node's in-links span
    many tiles, and the move log shows the fused moves (no statistics or
    select pass)."""
    import oracle
    csr = synth.pagerank_chain(synth.rmat_chain(14, 16, seed=7))  # node 0: 16385 in-links
    p = oracle.transition_probs(csr)
    C, H = oracle.initial_step(csr, p)
    c1 = np.abs(C).max()  # the cash the moves start from: the scale of their rounding
    oracle.solve(csr, p, C, H, sched=oracle.ALL_GREEN, tol=0.0, max_steps=40, check_every=-1)
    with Chain(csr, precision=prec) as ch:
        info = ch.solve("all_green", tol=0.0, max_steps=40, raise_on_noconv=False)
        c, h = ch.get_state()
        log = ch.move_log(40)
        assert ch.get_params().persistent == 1
    assert info["moves"] == 40 and info["pull_moves"] == 40
    assert info["edges_pushed"] == 40 * csr.nnz
    assert all(r["phase_us"][0] == 0.0 and r["phase_us"][1] == 0.0 and r["phase_us"][4] > 0 for r in log)
    assert [r["move"] for r in log] == list(range(40))
    if prec == "fp64":
        # FP64 rounding of 40 moves' in-link sums, in another order than the
        # oracle's: a budget per node from its in-degree (16385 at node 0)
        indeg = np.bincount(csr.col, minlength=csr.n)
        budget = 40 * (indeg + 4) * 2.0 ** -53
        assert np.all(np.abs(h - H) <= budget * np.abs(H).max())
        # the cash after 40 moves is what is left of sums that cancel: its
        # error scales with the cash the moves started from
        assert np.all(np.abs(c - C) <= budget * c1)
    else:
        # FP32 cash: the history drifts by FP32 rounding of the moved cash
        assert np.abs(h / h.sum() - H / H.sum()).sum() <= 1e-5


def test_power_sweep_barrier_wait_is_bounded(weighted):
    """The all-green sweep's grid barriers are bounded too (test hook: one
    block leaves before its first barrier)."""
    with Chain(weighted, precision="mixed") as ch:
        ch.set_params(barrier_limit_s=0.05, test_skip_barrier=1)
        info = ch.solve("all_green", tol=1e-9, raise_on_noconv=False)
        assert info["status"] == "RLGL_ETIMEOUT"
        ch.set_params(test_skip_barrier=0, barrier_limit_s=2.0)
        ch.reset()
        info = ch.solve("all_green", tol=1e-9)
        assert info["status"] == "RLGL_OK"
