"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs. Tolerances: FP64 path L1 <= 1e-12 on pi; MIXED path
L1 <= 1e-6 on pi; per-move states within the rounding of the arithmetic
(see each test)."""
import numpy as np
import pytest

import oracle
from paper_2008_02710_gb300 import synth
from tests.golden_io import read_example3, read_example9

pytestmark = pytest.mark.gpu

FP64_PI_TOL = 1e-12
MIXED_PI_TOL = 1e-6
SCHEDS = {"all_green": oracle.ALL_GREEN, "threshold": oracle.THRESHOLD, "topfrac": oracle.TOPFRAC,
          "link_threshold": oracle.LINK_THRESHOLD, "block_rr": oracle.BLOCK_RR, "pc": oracle.PC}


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
    # 2^14 nodes, ~300k edges: many merge-path tiles and push chunks, and
    # hub rows far longer than a chunk.
    csr = synth.rmat_chain(14, 16, seed=5, weighted=True)
    return csr, oracle.transition_probs(csr)


def green_of(h_before, h_after):
    return np.nonzero(h_after != h_before)[0]


# ------------------------------------------------------------ step 0

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_step0(tiny, prec):
    csr, p, _ = tiny
    C, H = oracle.initial_step(csr, p)
    with Chain(csr, precision=prec) as ch:
        c, h = ch.get_state()
    assert np.array_equal(h, H)
    scale = np.abs(C).max()
    tol = 1e-15 if prec == "fp64" else 2 ** -23
    assert np.abs(c - C).max() <= tol * scale


def test_step0_given_m0(medium):
    csr, p = medium
    m0 = synth.weights(csr.n, 9).astype(np.float64)
    m0 /= m0.sum()
    C, H = oracle.initial_step(csr, p, m0)
    with Chain(csr, m0=m0) as ch:
        c, h = ch.get_state()
    assert np.array_equal(h, m0)
    # step 0 is a move of M_0 from zero cash: node-wise rounding budget
    budget = rounding_budget(csr, p, m0, np.ones(csr.n, np.uint8), 2.0 ** -53) + 4 * 2.0 ** -53 * m0
    assert np.all(np.abs(c - C) <= budget)


# ------------------------------------------------- one move at a time

def rounding_budget(csr, p, c, green, unit):
    """First-order bound on |GPU - oracle| per node after one move from the
    same state: every node j ends as a sum of (adds_j) terms whose magnitudes
    add up to A_j (the same move applied to |C|); each add and each product
    (m_i s_i, then times w_ij) rounds once at `unit` relative."""
    A = np.abs(c).astype(np.float64)
    HA = np.zeros_like(A)
    oracle.move(csr, p, green, A, HA)
    rows = np.repeat(np.arange(csr.n), np.diff(csr.row_ptr))
    adds = np.zeros(csr.n)
    np.add.at(adds, csr.col, green[rows].astype(float))
    return (adds + 4.0) * unit * A + 1e-300


def _one_move_parity(csr, p, ch, sched, theta=0.0, top_frac=0.01, move=0):
    """From the GPU's current state, one oracle move and one GPU move must
    agree: the same green set (up to ties within rounding of theta) and, node
    by node, the same new cash within the rounding budget. `move` is the
    number of moves made since step 0 (BLOCK_RR and PC)."""
    unit = 2.0 ** -53 if ch.precision == "fp64" else 2.0 ** -24
    c, h = ch.get_state()
    prm = ch.get_params()
    g_or, th = oracle.select(c, SCHEDS[sched], abs_theta=theta, top_frac=top_frac,
                             theta_scale=prm.theta_scale, row_ptr=csr.row_ptr, move=move,
                             rr_blocks=prm.rr_blocks, pc_frac=prm.pc_frac, seed=prm.seed)
    info = ch.step(sched, theta if sched != "topfrac" else top_frac)
    c2, h2 = ch.get_state()
    # green sets: nodes whose history changed on the GPU vs the oracle's set
    # (zero-cash nodes move nothing, so they are compared by count only)
    gpu_set = set(green_of(h, h2).tolist())
    or_set = set(np.nonzero(g_or & (c != 0))[0].tolist())
    diff = gpu_set ^ or_set
    # Ties: nodes whose test value is within the rounding of theta may go
    # either way. The FP64 path decides in FP64 (band 1e-12 relative); the
    # MIXED path sums the statistics in FP32 within blocks and takes the
    # per-link test in FP32 (band 1e-4 relative).
    band = 1e-12 if ch.precision == "fp64" else 1e-4
    deg = np.diff(csr.row_ptr)
    for i in diff:
        if sched == "pc":
            # u_{t,i} against k |C_i| / ||C||_1, with ||C||_1 summed in
            # another order
            pr = prm.pc_frac * csr.n * abs(c[i]) / np.abs(c).sum()
            u = oracle.pc_uniform(prm.seed, move, int(i))
            assert abs(u - pr) <= band * pr, (i, u, pr)
            continue
        assert sched != "block_rr", i  # no arithmetic: exact
        v = abs(c[i]) / deg[i] if sched == "link_threshold" else abs(c[i])
        assert abs(v - th) <= band * max(th, 1e-300), (i, c[i], th)
    if not diff:
        assert info["green"] == int(g_or.sum())
        deg = np.diff(csr.row_ptr)
        assert info["edges_pushed"] == int(deg[g_or.astype(bool)].sum())
    if sched in ("threshold", "link_threshold"):
        assert abs(info["theta"] - th) <= (1e-13 if ch.precision == "fp64" else 1e-5) * th
    if sched == "topfrac":
        assert info["theta"] == th  # a selection, not arithmetic: exact
    C, H = c.copy(), h.copy()
    if diff:
        g_or = np.zeros(csr.n, np.uint8)
        g_or[list(gpu_set)] = 1
    oracle.move(csr, p, g_or, C, H)
    assert np.array_equal(h2, H)  # H_i += m_i adds one exact value per node
    budget = rounding_budget(csr, p, c, g_or, unit)
    err = np.abs(c2 - C)
    bad = np.nonzero(err > budget)[0]
    assert bad.size == 0, (bad[:5], err[bad[:5]], budget[bad[:5]])
    return info


@pytest.mark.parametrize("sched", ["all_green", "threshold", "topfrac", "link_threshold"])
def test_moves_tiny_fp64(tiny, sched):
    csr, p, _ = tiny
    with Chain(csr) as ch:
        for _ in range(25):
            _one_move_parity(csr, p, ch, sched, top_frac=0.05)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", ["push", "pull"])
@pytest.mark.parametrize("sched", ["threshold", "topfrac", "link_threshold"])
def test_moves_medium_push_pull(medium, sched, mode, prec):
    csr, p = medium
    with Chain(csr, precision=prec) as ch:
        ch.set_params(pull_crossover=0.0 if mode == "pull" else 10.0, theta_scale=0.5)
        for _ in range(12):
            info = _one_move_parity(csr, p, ch, sched, top_frac=0.02)
            if info["green"]:
                assert info["mode"] == (2 if mode == "pull" else 1)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("sched,kw", [("block_rr", dict(rr_blocks=7)), ("block_rr", dict(rr_blocks=1)),
                                      ("pc", dict(pc_frac=0.02, seed=9)), ("pc", dict(pc_frac=0.5, seed=1))])
def test_moves_block_rr_and_pc(medium, sched, kw, prec):
    """Block round robin and PC sampling, one move at a time from the GPU's
    state: the same green sets (PC: the same counter-based draws) and cash."""
    csr, p = medium
    with Chain(csr, precision=prec) as ch:
        ch.set_params(**kw)
        for t in range(10):
            info = _one_move_parity(csr, p, ch, sched, move=t)
            if sched == "block_rr" and kw["rr_blocks"] == 1:
                assert info["green"] == csr.n


@pytest.mark.parametrize("sched,kw", [("block_rr", dict(rr_blocks=5)), ("pc", dict(pc_frac=0.2, seed=3))])
@pytest.mark.parametrize("persistent", [0, 1])
def test_solve_block_rr_and_pc_vs_oracle(tiny, sched, kw, persistent):
    csr, p, ref = tiny
    pi_or, C, H, info_or = oracle.run(csr, sched=SCHEDS[sched], tol=1e-12, max_steps=200000, **kw)
    with Chain(csr) as ch:
        ch.set_params(persistent=persistent, **kw)
        info = ch.solve(sched, tol=1e-12, max_steps=200000)
        pi_tol = ch.estimate()
        ch.reset()
        ch.solve(sched, tol=0.0, max_steps=info_or["moves"], raise_on_noconv=False)
        pi = ch.estimate()
    assert info["status"] == "RLGL_OK"
    assert abs(info["moves"] - info_or["moves"]) <= max(1, info_or["moves"] // 1000)
    assert np.abs(pi - pi_or).sum() <= FP64_PI_TOL
    assert np.abs(pi_tol - ref).sum() <= 1e-11


def test_block_rr_and_pc_rejected_for_a_batch():
    from paper_2008_02710_gb300.rlgl import RLGLError
    big, node_ptr = synth.stack_chains([synth.tiny_chain(200, seed=s) for s in (1, 2)])
    with Chain(big, node_ptr=node_ptr) as ch:
        for sched in ("block_rr", "pc"):
            with pytest.raises(RLGLError) as e:
                ch.solve(sched, tol=1e-9)
            assert e.value.name == "RLGL_EINVAL"


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_moves_medium_all_green(medium, prec):
    csr, p = medium
    with Chain(csr, precision=prec) as ch:
        for _ in range(6):
            info = _one_move_parity(csr, p, ch, "all_green")
            assert info["mode"] == 2 and info["green"] == csr.n


# ------------------------------------------------------------ solves

@pytest.mark.parametrize("sched", ["all_green", "threshold", "topfrac", "link_threshold"])
def test_solve_tiny_fp64_vs_oracle_and_gth(tiny, sched):
    csr, p, ref = tiny
    pi_or, C, H, info_or = oracle.run(csr, sched=SCHEDS[sched], top_frac=0.01, tol=1e-12,
                                      max_steps=200000)
    th = 0.01 if sched == "topfrac" else 0.0
    with Chain(csr) as ch:
        info = ch.solve(sched, th, tol=1e-12, max_steps=200000)
        pi_tol = ch.estimate()
        # the same number of moves as the oracle: the same trajectory up to
        # the order of FP64 additions
        ch.reset()
        ch.solve(sched, th, tol=0.0, max_steps=info_or["moves"], raise_on_noconv=False)
        pi = ch.estimate()
    assert info["status"] == "RLGL_OK"
    assert abs(info["moves"] - info_or["moves"]) <= 1
    assert np.abs(pi - pi_or).sum() <= FP64_PI_TOL
    assert np.abs(pi_tol - ref).sum() <= 1e-11
    assert abs(pi.sum() - 1) < 1e-13


@pytest.mark.parametrize("sched", ["all_green", "threshold", "topfrac", "link_threshold"])
def test_solve_tiny_mixed_vs_gth(tiny, sched):
    csr, p, ref = tiny
    with Chain(csr, precision="mixed") as ch:
        info = ch.solve(sched, 0.01 if sched == "topfrac" else 0.0, tol=1e-9, max_steps=200000)
        pi = ch.estimate()
        resid = ch.invariant_residual()
    assert info["status"] == "RLGL_OK"
    assert np.abs(pi - ref).sum() <= MIXED_PI_TOL
    assert resid <= 1e-6


@pytest.mark.parametrize("sched", ["threshold", "link_threshold"])
def test_solve_medium_fp64_vs_oracle(medium, sched):
    csr, p = medium
    pi_or, C, H, info_or = oracle.run(csr, sched=SCHEDS[sched], tol=1e-12, max_steps=200000)
    ref, it, delta = oracle.power_iteration(csr, p, tol=1e-14, maxit=200000, nthreads=8)
    with Chain(csr) as ch:
        info = ch.solve(sched, tol=1e-12, max_steps=200000)
        ch.reset()
        ch.solve(sched, tol=0.0, max_steps=info_or["moves"], raise_on_noconv=False)
        pi = ch.estimate()
        inv = ch.invariant_residual()
    assert info["status"] == "RLGL_OK"
    assert np.abs(pi - pi_or).sum() <= FP64_PI_TOL
    # the stop test fires on a residual that both sides compute with their
    # own rounding: over ~1e4 moves it may fire a few moves apart
    assert abs(info["moves"] - info_or["moves"]) <= max(1, info_or["moves"] // 1000)
    # residual 1e-12 bounds the error by 1e-12 * ||Z|| (Eq. convergence)
    assert np.abs(pi - ref).sum() <= 1e-8
    assert inv <= 1e-13 * np.abs(H).sum()


def test_solve_exact_move_count_with_zero_tol(tiny):
    csr, p, _ = tiny
    with Chain(csr) as ch:
        info = ch.solve("threshold", tol=0.0, max_steps=37, raise_on_noconv=False)
    assert info["status"] == "RLGL_ENOCONV" and info["moves"] == 37


def test_reset_restores_step0(tiny):
    csr, p, _ = tiny
    with Chain(csr) as ch:
        c0, h0 = ch.get_state()
        ch.solve("threshold", tol=1e-6)
        ch.reset()
        c1, h1 = ch.get_state()
        info = ch.solve("threshold", tol=1e-6)
        info2 = None
        ch.reset()
        info2 = ch.solve("threshold", tol=1e-6)
    assert np.array_equal(h0, h1) and np.abs(c0 - c1).max() <= 1e-18
    assert info["moves"] == info2["moves"]


# --------------------------------------------- the paper's examples

def test_example3_degenerate_on_gpu():
    ex = read_example3()
    A = np.array([[float(x) for x in r] for r in ex["P"]])
    csr = synth.from_dense(A)
    with Chain(csr, m0=np.array([1.0, 0, 0, 0])) as ch:
        c, h = ch.get_state()
        assert np.array_equal(c, [float(x) for x in ex["C1"]])
        ch.set_masks(np.array([[1, 0, 0, 0]], np.uint8))
        info = ch.solve("mask", tol=1e-12, max_steps=10, raise_on_noconv=False)
        assert info["status"] == "RLGL_EDEGENERATE"
        from paper_2008_02710_gb300.rlgl import RLGLError
        with pytest.raises(RLGLError) as e:
            ch.estimate()
        assert e.value.name == "RLGL_EDEGENERATE"


@pytest.mark.parametrize("table", ["example9_table1.txt", "example9_table2.txt"])
def test_example9_tables_on_gpu(table):
    from fractions import Fraction
    M = (Fraction(1, 8), Fraction(1, 4), Fraction(1, 4), Fraction(3, 8))
    ex = read_example3()
    A = np.array([[float(x) for x in r] for r in ex["P"]])
    csr = synth.from_dense(A)
    rows = read_example9(table, M)
    masks = np.zeros((len(rows), 4), np.uint8)
    for k, (_, _, _, g) in enumerate(rows):
        masks[k, g - 1] = 1
    for prec in ("fp64", "mixed"):
        with Chain(csr, m0=np.array([float(x) for x in M]), precision=prec) as ch:
            ch.set_masks(masks)
            for t, Ht, Ct, g in rows:
                c, h = ch.get_state()
                assert np.array_equal(h, [float(x) for x in Ht]), (prec, t)
                assert np.array_equal(c, [float(x) for x in Ct]), (prec, t)
                ch.step("mask")


def test_two_wheels_and_doubly_stochastic_on_gpu():
    tw = synth.two_wheels()
    d = tw.degrees().astype(float)
    with Chain(tw) as ch:
        ch.solve("threshold", tol=1e-14)
        assert np.abs(ch.estimate() - d / d.sum()).sum() < 1e-12
    ds = synth.doubly_stochastic(3000, 5, seed=3)
    with Chain(ds) as ch:
        ch.solve("threshold", tol=1e-13)
        assert np.abs(ch.estimate() - 1 / 3000).sum() < 1e-11


def test_two_block_contraction_on_gpu():
    K, n = 4, 25
    csr = synth.from_dense(synth.sbm_mean_field([K * n, n], 10.0, 1.0))
    p, q = 0.1, 0.01
    with Chain(csr) as ch:
        mask = np.zeros((1, csr.n), np.uint8)
        mask[0, K * n:] = 1
        ch.set_masks(mask)
        c, _ = ch.get_state()
        before = np.abs(c).sum()
        for _ in range(8):
            info = ch.step("mask")
            assert abs(info["l1_cash"] - p / (q * K + p) * before) <= 1e-13 * before + 1e-16
            before = info["l1_cash"]


def test_three_block_single_block_does_not_converge_on_gpu():
    sizes = [50, 20, 10]
    csr = synth.from_dense(synth.sbm_mean_field(sizes, 10.0, 1.0))
    with Chain(csr) as ch:
        m = np.zeros((1, 80), np.uint8)
        m[0, :50] = 1
        ch.set_masks(m)
        info = ch.solve("mask", tol=1e-12, max_steps=3000, raise_on_noconv=False)
    assert info["status"] == "RLGL_ENOCONV" and info["resid"] > 1e-4


# ---------------------------------------- state, resume, device input

def test_resume_from_state_continues_identically(medium):
    csr, p = medium
    with Chain(csr) as a:
        a.solve("threshold", tol=0.0, max_steps=15, raise_on_noconv=False)
        c, h = a.get_state()
        with Chain(csr, c=c, h=h) as b:
            assert b.invariant_residual() <= 1e-15
            cb, hb = b.get_state()
            assert np.array_equal(cb, c) and np.array_equal(hb, h)
            # the same moves from the same state: equal up to the order of
            # the FP64 atomic additions
            a.solve("threshold", tol=0.0, max_steps=200, raise_on_noconv=False)
            b.solve("threshold", tol=0.0, max_steps=200, raise_on_noconv=False)
            assert np.abs(a.estimate() - b.estimate()).sum() <= 1e-13
            # to the tolerance: the stop test may fire a move apart, and two
            # estimates that both meet tol 1e-12 differ by O(tol)
            ia = a.solve("threshold", tol=1e-12, max_steps=100000)
            ib = b.solve("threshold", tol=1e-12, max_steps=100000)
            assert np.abs(a.estimate() - b.estimate()).sum() <= 1e-11
    # this chain mixes slowly (~3e4 moves to 1e-12): the residual shrinks by
    # ~1e-3 relative per move, so residuals that differ in the last bits can
    # cross tol a few moves apart
    assert abs(ia["moves"] - ib["moves"]) <= max(1, ib["moves"] // 1000)


def test_device_input_same_as_host(tiny):
    import torch
    csr, p, ref = tiny
    dev = synth.CSR(csr.n, torch.from_numpy(csr.row_ptr).cuda(), torch.from_numpy(csr.col).cuda(),
                    torch.from_numpy(csr.w).cuda())
    with Chain(dev) as a, Chain(csr) as b:
        ca, ha = a.get_state()
        cb, hb = b.get_state()
        assert np.array_equal(ha, hb) and np.abs(ca - cb).max() <= 1e-18
        a.solve("threshold", tol=1e-12)
        out = torch.empty(csr.n, dtype=torch.float64, device="cuda")
        a.estimate(out)
        assert np.abs(out.cpu().numpy() - ref).sum() <= 1e-11


def test_invariant_and_refresh_mixed(medium):
    csr, p = medium
    with Chain(csr, precision="mixed") as ch:
        ch.set_params(refresh_factor=0.0)
        for _ in range(20):
            ch.step("threshold", info=False)
        drift = ch.invariant_residual()
        removed = ch.refresh()
        after = ch.invariant_residual()
        c, h = ch.get_state()
    assert drift > 0 and abs(removed - drift) <= 1e-3 * drift + 1e-18
    # after re-derivation only the FP32 rounding of C itself remains
    assert after <= 2 ** -23 * np.abs(c).sum() + 1e-16
    assert oracle.invariant_residual(csr, p, c, h) <= 2 ** -23 * np.abs(c).sum() + 1e-15


def test_single_node_chain():
    csr = synth.edges_to_csr(1, np.array([0]), np.array([0]), None)
    with Chain(csr) as ch:
        info = ch.solve("threshold", tol=1e-12, max_steps=10)
        assert info["moves"] == 1
        assert np.array_equal(ch.estimate(), [1.0])


# --------------------------------------------------------- errors

def test_invalid_inputs_are_rejected():
    from paper_2008_02710_gb300.rlgl import RLGLError
    bad_col = synth.CSR(3, np.array([0, 1, 2, 3], np.int64), np.array([1, 2, 3], np.int32), None)
    with pytest.raises(RLGLError) as e:
        Chain(bad_col)
    assert e.value.name == "RLGL_EINVAL"
    empty_row = synth.CSR(3, np.array([0, 1, 1, 2], np.int64), np.array([1, 0], np.int32), None)
    with pytest.raises(RLGLError) as e:
        Chain(empty_row)
    assert e.value.name == "RLGL_ENOTSTOCHASTIC"
    neg_w = synth.CSR(2, np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32),
                      np.array([1.0, -1.0], np.float32))
    with pytest.raises(RLGLError) as e:
        Chain(neg_w)
    assert e.value.name == "RLGL_ENOTSTOCHASTIC"
    bad_ptr = synth.CSR(2, np.array([0, 2, 1], np.int64), np.array([1, 0], np.int32), None)
    with pytest.raises(RLGLError) as e:
        Chain(bad_ptr)
    assert e.value.name == "RLGL_EINVAL"
    good = synth.tiny_chain(50, 1)
    with Chain(good) as ch:
        with pytest.raises(RLGLError):
            ch.solve("threshold", max_steps=0)
        with pytest.raises(RLGLError):
            ch.step("mask")
        with pytest.raises(RLGLError):
            ch.set_params(top_frac=0.0)
    with pytest.raises(RLGLError) as e:
        Chain(good, c=np.ones(50), h=np.ones(50))
    assert e.value.name == "RLGL_EINVAL"


def test_profile_moves_and_move_log(medium):
    """The gated profiling run makes the same moves as rlgl_step and the
    device-side move log records them."""
    csr, p = medium
    with Chain(csr) as a, Chain(csr) as b:
        for ch in (a, b):
            ch.set_params(theta_scale=0.5)
        a.profile(2)
        kt = a.profile_moves("link_threshold", 0.0, 20)
        for _ in range(20):
            b.step("link_threshold", info=False)
        ca, ha = a.get_state()
        cb, hb = b.get_state()
        # pushes add in a nondeterministic order: equal up to FP64 rounding
        assert np.abs(ha - hb).max() <= 1e-12 * np.abs(hb).max()
        assert np.abs(ca - cb).max() <= 1e-12 * np.abs(cb).max()
        assert kt["select"][1] == 20 and kt["select"][0] > 0
        log = a.move_log(50)
        assert len(log) == 20 and [r["move"] for r in log] == list(range(20))
        deg = np.diff(csr.row_ptr)
        assert all(r["edges_pushed"] <= csr.nnz and r["green"] <= csr.n for r in log)
        assert log[-1]["sum_hist"] > 0
