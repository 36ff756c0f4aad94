"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics
(worked examples, closed forms, invariants, brute force, library routines),
chosen so that a dropped term, a wrong sign or index, or a transposed operand
in the oracle fails at least one of them. No GPU is needed."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2008_02710_gb300 import synth
from tests.golden_io import read_example3, read_example9, read_selection_cases


def csr_from_fractions(P):
    A = np.array([[float(x) for x in row] for row in P])
    return synth.from_dense(A)


# ---------------------------------------------------------------- Example 3

def test_example3_step0_and_degenerate_move():
    ex = read_example3()
    csr = csr_from_fractions(ex["P"])
    p = oracle.transition_probs(csr)
    m0 = np.array([float(x) for x in ex["M0"]])
    C, H = oracle.initial_step(csr, p, m0)
    assert np.array_equal(C, [float(x) for x in ex["C1"]])
    assert np.array_equal(H, [float(x) for x in ex["H1"]])
    green = np.zeros(4, np.uint8)
    green[int(ex["G1"][0]) - 1] = 1
    oracle.move(csr, p, green, C, H)
    assert np.array_equal(C, [0.0] * 4) and np.array_equal(H, [0.0] * 4)


def test_example3_degenerate_status_and_estimate_raises():
    ex = read_example3()
    csr = csr_from_fractions(ex["P"])
    p = oracle.transition_probs(csr)
    C, H = oracle.initial_step(csr, p, np.array([1.0, 0, 0, 0]))
    mask = np.array([[1, 0, 0, 0]], np.uint8)
    info = oracle.solve(csr, p, C, H, sched=oracle.MASK, masks=mask, tol=1e-12, max_steps=10)
    assert info["status"] == "EDEGENERATE"
    with pytest.raises(ArithmeticError):
        oracle.estimate(H)


def test_example3_stationary_law_gth_and_oracle():
    ex = read_example3()
    pi_star = np.array([float(x) for x in ex["pi"]])
    A = np.array([[float(x) for x in row] for row in ex["P"]])
    assert np.allclose(oracle.gth(A), pi_star, atol=1e-15, rtol=0)
    csr = csr_from_fractions(ex["P"])
    pi, C, H, info = oracle.run(csr, sched=oracle.ALL_GREEN, tol=1e-14, max_steps=100000)
    assert info["status"] == "OK"
    assert np.abs(pi - pi_star).sum() < 1e-12


# ---------------------------------------------------------------- Example 9

@pytest.mark.parametrize("M", [(Fraction(1, 8), Fraction(1, 4), Fraction(1, 4), Fraction(3, 8)),
                               (Fraction(1, 2), Fraction(1, 8), Fraction(1, 8), Fraction(1, 4))])
@pytest.mark.parametrize("table", ["example9_table1.txt", "example9_table2.txt"])
def test_example9_tables_exact(table, M):
    """Every row of both printed tables, for dyadic M_0 (exact in FP64)."""
    ex = read_example3()
    csr = csr_from_fractions(ex["P"])
    p = oracle.transition_probs(csr)
    rows = read_example9(table, M)
    C, H = oracle.initial_step(csr, p, np.array([float(x) for x in M]))
    for t, Ht, Ct, g in rows:
        assert np.array_equal(H, [float(x) for x in Ht]), (table, t, H, Ht)
        assert np.array_equal(C, [float(x) for x in Ct]), (table, t, C, Ct)
        green = np.zeros(4, np.uint8)
        green[g - 1] = 1
        oracle.move(csr, p, green, C, H)


def test_example9_table2_periodic_nonconvergence_and_exact_when_balanced():
    ex = read_example3()
    csr = csr_from_fractions(ex["P"])
    p = oracle.transition_probs(csr)
    masks = np.zeros((4, 4), np.uint8)
    for k, g in enumerate([1, 2, 4, 3]):
        masks[k, g - 1] = 1
    C, H = oracle.initial_step(csr, p, np.array([0.125, 0.25, 0.25, 0.375]))
    info = oracle.solve(csr, p, C, H, sched=oracle.MASK, masks=masks, tol=1e-12, max_steps=400)
    assert info["status"] == "ENOCONV" and info["resid"] > 0.1
    # M3 = M4 > 0: exact at t = 3 (two moves).
    C, H = oracle.initial_step(csr, p, np.array([0.25, 0.25, 0.25, 0.25]))
    info = oracle.solve(csr, p, C, H, sched=oracle.MASK, masks=masks, tol=1e-15, max_steps=400)
    assert info["status"] == "OK" and info["moves"] == 2
    assert np.allclose(oracle.estimate(H), [2 / 7, 1 / 7, 2 / 7, 2 / 7], atol=1e-15, rtol=0)


# ------------------------------------------- power iteration equivalence

def test_all_green_is_power_iteration():
    """G_t = [N] gives H_t = M_0 P^(t-1) and H_t 1 = 1 (Sec. 2.3.1)."""
    csr = synth.tiny_chain(60, seed=3)
    p = oracle.transition_probs(csr)
    P = oracle.dense_P(csr, p)
    m0 = synth.weights(60, 5).astype(np.float64)
    m0 /= m0.sum()
    C, H = oracle.initial_step(csr, p, m0)
    allg = np.ones(60, np.uint8)
    for t in range(1, 25):
        ref = m0 @ np.linalg.matrix_power(P, t - 1)
        assert np.abs(H - ref).max() < 1e-14
        assert abs(H.sum() - 1.0) < 1e-13
        oracle.move(csr, p, allg, C, H)


def test_initial_cash_is_m0_times_P_minus_I():
    csr = synth.tiny_chain(50, seed=4)
    p = oracle.transition_probs(csr)
    P = oracle.dense_P(csr, p)
    assert np.allclose(P.sum(1), 1.0, atol=1e-15)
    C, H = oracle.initial_step(csr, p)
    m0 = np.full(50, 1 / 50)
    assert np.abs(C - (m0 @ P - m0)).max() < 1e-16
    assert np.array_equal(H, m0)
    assert abs(C.sum()) < 1e-15


# ------------------------------------------------------------ invariants

@pytest.mark.parametrize("sched", [oracle.ALL_GREEN, oracle.THRESHOLD, oracle.TOPFRAC,
                                   oracle.LINK_THRESHOLD])
def test_invariants_every_step(sched):
    """sum C = 0, ||C||_1 never grows, C = H(P - I) at every step."""
    csr = synth.tiny_chain(300, seed=7)
    pi, C, H, info = oracle.run(csr, sched=sched, top_frac=0.05, tol=1e-13, max_steps=20000,
                                check_every=1)
    assert info["status"] == "OK"
    assert info["sum_cash"] < 1e-15
    assert info["l1_growth"] < 1e-15
    assert info["invariant"] < 1e-13


def test_invariant_residual_detects_a_perturbation():
    csr = synth.tiny_chain(40, seed=2)
    p = oracle.transition_probs(csr)
    C, H = oracle.initial_step(csr, p)
    assert oracle.invariant_residual(csr, p, C, H) < 1e-16
    C[3] += 1e-6
    assert abs(oracle.invariant_residual(csr, p, C, H) - 1e-6) < 1e-12


# ------------------------------------------------- stationary laws

def _random_dense_chain(n, seed, density=0.4):
    rng = np.random.default_rng(seed)
    A = (rng.random((n, n)) < density) * rng.integers(1, 1 << 20, (n, n)) / float(1 << 20)
    A[np.arange(n), (np.arange(n) + 1) % n] = 0.5
    A[np.arange(n), np.arange(n)] += 0.25
    return A


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (7, 2), (30, 3), (120, 4)])
def test_gth_against_brute_force_solve(n, seed):
    A = _random_dense_chain(n, seed)
    P = A / A.sum(1, keepdims=True)
    M = P.T - np.eye(n)
    M[-1, :] = 1.0
    b = np.zeros(n)
    b[-1] = 1.0
    ref = np.linalg.solve(M, b)
    pi = oracle.gth(P)
    assert np.abs(pi - ref).sum() < 1e-13
    assert np.abs(pi @ P - pi).sum() < 1e-14


def test_gth_two_state_closed_form():
    a, b = 0.3, 0.125
    pi = oracle.gth(np.array([[1 - a, a], [b, 1 - b]]))
    assert np.allclose(pi, [b / (a + b), a / (a + b)], atol=1e-16, rtol=0)


@pytest.mark.parametrize("sched", [oracle.ALL_GREEN, oracle.THRESHOLD, oracle.TOPFRAC,
                                   oracle.LINK_THRESHOLD])
def test_tiny_chain_1000_against_gth(sched):
    """The N = 1000 tiny chain: RLGL to ||C||_1/H1 < 1e-12 agrees with GTH."""
    csr = synth.tiny_chain(1000, seed=1)
    p = oracle.transition_probs(csr)
    ref = oracle.gth(oracle.dense_P(csr, p))
    pi, C, H, info = oracle.run(csr, sched=sched, top_frac=0.01, tol=1e-12, max_steps=200000)
    assert info["status"] == "OK"
    assert np.abs(pi - ref).sum() <= 1e-11
    assert abs(pi.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("sched", [oracle.ALL_GREEN, oracle.THRESHOLD])
def test_two_wheels_degree_law(sched):
    """Random walk on an undirected graph: pi_i = d_i / sum d (two-wheels graph)."""
    csr = synth.two_wheels()
    assert csr.nnz == 42
    d = csr.degrees().astype(float)
    pi, C, H, info = oracle.run(csr, sched=sched, tol=1e-14, max_steps=100000)
    assert info["status"] == "OK"
    assert np.abs(pi - d / d.sum()).sum() < 1e-12


def test_doubly_stochastic_uniform():
    csr = synth.doubly_stochastic(500, 5, seed=3)
    p = oracle.transition_probs(csr)
    P = oracle.dense_P(csr, p)
    assert np.abs(P.sum(0) - 1).max() < 1e-14
    pi, C, H, info = oracle.run(csr, sched=oracle.THRESHOLD, tol=1e-13, max_steps=100000)
    assert info["status"] == "OK"
    assert np.abs(pi - 1 / 500).sum() < 1e-11


def test_symmetrised_rmat_degree_law():
    csr = synth.rmat_chain(10, 8, seed=2, undirected=True)
    d = csr.degrees().astype(float)
    p = oracle.transition_probs(csr)
    pi, it, delta = oracle.power_iteration(csr, p, tol=1e-13, maxit=200000)
    assert np.abs(pi - d / d.sum()).sum() < 1e-10
    pi2, C, H, info = oracle.run(csr, sched=oracle.THRESHOLD, tol=1e-13, max_steps=200000)
    assert np.abs(pi2 - d / d.sum()).sum() < 1e-11


def test_power_iteration_threads_bitwise_and_matches_gth():
    csr = synth.tiny_chain(800, seed=9)
    p = oracle.transition_probs(csr)
    a, ia, _ = oracle.power_iteration(csr, p, tol=1e-14, nthreads=1)
    b, ib, _ = oracle.power_iteration(csr, p, tol=1e-14, nthreads=4)
    assert ia == ib and np.array_equal(a, b)
    ref = oracle.gth(oracle.dense_P(csr, p))
    assert np.abs(a - ref).sum() < 1e-12


# ------------------------------------------ mean-field block models

def _sbm(sizes, p, q):
    # P depends on p/q only (rows are normalised), so the weights are scaled
    # to the FP32-exact integers round(p/q) and 1.
    return synth.from_dense(synth.sbm_mean_field(sizes, round(p / q), 1.0))


def _two_block(K, n, p, q):
    return _sbm([K * n, n], p, q)


def test_two_block_lambda2_closed_form():
    K, n, p, q = 4, 25, 0.1, 0.01
    csr = _two_block(K, n, p, q)
    P = oracle.dense_P(csr, oracle.transition_probs(csr))
    ev = np.sort(np.abs(np.linalg.eigvals(P)))[::-1]
    lam2 = (p * p - q * q) * K / ((p * K + q) * (q * K + p))
    assert abs(ev[1] - lam2) < 1e-12


@pytest.mark.parametrize("block,factor", [(0, lambda K, p, q: p * K / (p * K + q)),
                                          (1, lambda K, p, q: p / (q * K + p))])
def test_two_block_one_block_contraction(block, factor):
    """Eqs. CG1 / CG2: ||C_{t+1}||_1 = factor * ||C_t||_1 for G_t = B_1 or B_2."""
    K, n, p, q = 4, 25, 0.1, 0.01
    csr = _two_block(K, n, p, q)
    pr = oracle.transition_probs(csr)
    C, H = oracle.initial_step(csr, pr)
    green = np.zeros(csr.n, np.uint8)
    if block == 0:
        green[:K * n] = 1
    else:
        green[K * n:] = 1
    f = factor(K, p, q)
    # Red nodes keep their rounding errors, so the check has an absolute
    # floor at rounding level of the initial cash.
    floor = 1e-14 * oracle.l1(C)
    for _ in range(12):
        before = oracle.l1(C)
        oracle.move(csr, pr, green, C, H)
        assert abs(oracle.l1(C) - f * before) <= 1e-13 * before + floor


def test_two_block_all_green_rate_is_lambda2():
    K, n, p, q = 4, 25, 0.1, 0.01
    csr = _two_block(K, n, p, q)
    pr = oracle.transition_probs(csr)
    C, H = oracle.initial_step(csr, pr)
    lam2 = (p * p - q * q) * K / ((p * K + q) * (q * K + p))
    allg = np.ones(csr.n, np.uint8)
    for _ in range(10):
        before = oracle.l1(C)
        oracle.move(csr, pr, allg, C, H)
        assert abs(oracle.l1(C) - lam2 * before) <= 1e-12 * before


def test_three_block_single_block_moves_and_divergence():
    """Eqs. c1ii / c1ij (with denominators N_i(p-q)+Nq, Eq. P3) for one block
    move, and Theorem 12: giving the green light to block 1 alone leaves
    liminf ||C_t||_1 > 0 for N = (50, 20, 10), p = 0.1, q = 0.01."""
    sizes, p, q = [50, 20, 10], 0.1, 0.01
    N = sum(sizes)
    csr = _sbm(sizes, p, q)
    pr = oracle.transition_probs(csr)
    C, H = oracle.initial_step(csr, pr)
    starts = np.cumsum([0] + sizes)
    blk = lambda v, b: v[starts[b]:starts[b + 1]]
    green = np.zeros(N, np.uint8)
    green[:50] = 1
    for _ in range(5):
        c = [blk(C, b)[0] for b in range(3)]
        for b in range(3):
            assert np.ptp(blk(C, b)) < 1e-17
        oracle.move(csr, pr, green, C, H)
        den = sizes[0] * (p - q) + N * q
        assert abs(blk(C, 0)[0] - c[0] * sizes[0] * p / den) < 1e-16
        for j in (1, 2):
            assert abs(blk(C, j)[0] - (c[j] + c[0] * sizes[0] * q / den)) < 1e-16
    info = oracle.solve(csr, pr, C, H, sched=oracle.MASK, masks=green[None, :], tol=1e-12,
                        max_steps=3000)
    assert info["status"] == "ENOCONV" and info["resid"] > 1e-4


def test_three_block_initial_cash_closed_form():
    """Sec. 5.2 prints the per-block initial cash after one power-iteration
    step, c_i = (zeta/N) sum_j N_j (N_j - N_i) / ((N_i zeta + N)(N_j zeta + N)),
    with zeta read as (p - q)/q. That expression is M_0 - M_0 P; Alg. 1 gives
    C_1 = M_0 (P - I), the same magnitudes with the opposite sign."""
    sizes, p, q = [50, 20, 10], 0.1, 0.01
    N, zeta = sum(sizes), (p - q) / q
    csr = _sbm(sizes, p, q)
    C, H = oracle.initial_step(csr, oracle.transition_probs(csr))
    starts = np.cumsum([0] + sizes)
    for i, Ni in enumerate(sizes):
        c_paper = zeta / N * sum(Nj * (Nj - Ni) / ((Ni * zeta + N) * (Nj * zeta + N))
                                 for Nj in sizes)
        blk = C[starts[i]:starts[i + 1]]
        assert np.abs(blk - (-c_paper)).max() < 1e-15
    assert C[0] > 0 and C[-1] < 0


def test_dobrushin_bound_all_green():
    """Theorem 7 with m = 1: ||C_t||_1 <= 2 delta(P)^(t-1) (Eq. dobrushin)."""
    A = _random_dense_chain(12, 11, density=0.9)
    P = A / A.sum(1, keepdims=True)
    delta = 1 - min(np.minimum(P[i], P[k]).sum() for i in range(12) for k in range(12))
    assert delta < 1
    csr = synth.from_dense(A)
    pr = oracle.transition_probs(csr)
    C, H = oracle.initial_step(csr, pr)
    allg = np.ones(12, np.uint8)
    for t in range(1, 40):
        assert oracle.l1(C) <= 2 * delta ** (t - 1) * (1 + 1e-12)
        oracle.move(csr, pr, allg, C, H)


# -------------------------------------------------- schedule semantics

def test_selection_hand_worked_cases():
    for case in read_selection_cases():
        if case["sched"] == "threshold_r1":
            g, th = oracle.select(case["cash"], oracle.THRESHOLD, theta_scale=case["param"], r=1)
        elif case["sched"] == "threshold_r2":
            g, th = oracle.select(case["cash"], oracle.THRESHOLD, theta_scale=case["param"], r=2)
        elif case["sched"] == "link_r1":
            g, th = oracle.select(case["cash"], oracle.LINK_THRESHOLD, theta_scale=case["param"],
                                  r=1, row_ptr=np.array([0, 3, 4, 6, 10]))
        else:
            g, th = oracle.select(case["cash"], oracle.TOPFRAC, top_frac=case["param"])
        assert sorted(np.nonzero(g)[0].tolist()) == case["green"], case
        assert abs(th - case["theta"]) < 1e-15, case


def test_topfrac_single_is_max_abs_cash():
    """k = 1 is RLGL_MaxC: the node with maximum |C| (np.argmax)."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        c = rng.standard_normal(37)
        g, th = oracle.select(c, oracle.TOPFRAC, top_frac=1 / 37)
        assert np.nonzero(g)[0].tolist() == [int(np.argmax(np.abs(c)))]


def test_move_synchronous_semantics_brute_force():
    """A move is C <- C - M(I - P) with M taken before any update: checked
    against the dense matrix product on tiny random chains and masks."""
    rng = np.random.default_rng(8)
    for trial in range(40):
        n = int(rng.integers(2, 9))
        A = _random_dense_chain(n, 100 + trial, density=0.5)
        csr = synth.from_dense(A)
        pr = oracle.transition_probs(csr)
        P = oracle.dense_P(csr, pr)
        C = rng.standard_normal(n)
        C -= C.mean()
        H = rng.standard_normal(n)
        g = (rng.random(n) < 0.5).astype(np.uint8)
        M = C * g
        C_ref = C - M @ (np.eye(n) - P)
        H_ref = H + M
        C2, H2 = C.copy(), H.copy()
        oracle.move(csr, pr, g, C2, H2)
        assert np.abs(C2 - C_ref).max() < 1e-14
        assert np.array_equal(H2, H_ref)


def test_duplicate_edges_add():
    # row 0 lists target 1 twice with weight 1 and target 0 once with weight 2:
    # p_01 = 2/4, p_00 = 2/4 either way.
    csr = synth.edges_to_csr(2, np.array([0, 0, 0, 1]), np.array([1, 1, 0, 0]),
                             np.array([1, 1, 2, 1], np.float32))
    P = oracle.dense_P(csr, oracle.transition_probs(csr))
    assert np.allclose(P, [[0.5, 0.5], [1.0, 0.0]], atol=0, rtol=0)


def test_not_stochastic_rejected():
    csr = synth.edges_to_csr(3, np.array([0, 1]), np.array([1, 0]), None)
    with pytest.raises(ValueError):
        oracle.transition_probs(csr)


# ------------------------------------------- block round robin and PC

def test_splitmix64_published_outputs():
    """The PC schedule's generator against the reference outputs of
    SplitMix64 from state 0 (Steele, Lea and Flood 2014; the published
    reference implementation's first three values)."""
    assert oracle.sm64_outputs(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                         0x06C45D188009454F]


def test_pc_uniforms_are_uniform_and_counter_based():
    u = np.array([[oracle.pc_uniform(7, t, i) for i in range(2000)] for t in range(5)])
    assert u.min() >= 0.0 and u.max() < 1.0
    # same counter, same value; different moves differ
    assert oracle.pc_uniform(7, 3, 11) == u[3, 11]
    assert not np.array_equal(u[0], u[1])
    # Kolmogorov-Smirnov against U(0,1) at the 1e-4 level
    from scipy import stats
    assert stats.kstest(u.ravel(), "uniform").pvalue > 1e-4
    # u is a multiple of 2^-53 (53 high bits of the 64-bit output)
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))


@pytest.mark.parametrize("n,K", [(10, 4), (10, 6), (1000, 7), (1000, 1), (5, 9)])
def test_block_rr_partitions_the_nodes(n, K):
    """K' consecutive moves green every node exactly once, in contiguous
    blocks of ceil(N / K) nodes taken in order."""
    b = -(-n // min(K, n))
    kp = -(-n // b)
    C = np.ones(n)
    seen = np.zeros(n, int)
    for t in range(kp):
        g, _ = oracle.select(C, oracle.BLOCK_RR, move=t, rr_blocks=K)
        idx = np.nonzero(g)[0]
        assert idx.min() == t * b and idx.max() == min(n, (t + 1) * b) - 1
        assert len(idx) == idx.max() - idx.min() + 1
        seen += g
    assert np.all(seen == 1)
    g, _ = oracle.select(C, oracle.BLOCK_RR, move=kp, rr_blocks=K)  # the cycle restarts
    assert np.nonzero(g)[0].min() == 0


def test_block_rr_one_block_is_power_iteration():
    csr = synth.tiny_chain(300, seed=4)
    p = oracle.transition_probs(csr)
    C1, H1 = oracle.initial_step(csr, p)
    C2, H2 = C1.copy(), H1.copy()
    oracle.solve(csr, p, C1, H1, sched=oracle.BLOCK_RR, rr_blocks=1, tol=0.0, max_steps=40)
    oracle.solve(csr, p, C2, H2, sched=oracle.ALL_GREEN, tol=0.0, max_steps=40)
    assert np.array_equal(C1, C2) and np.array_equal(H1, H2)


def test_block_rr_equals_the_same_masks_and_converges():
    """BLOCK_RR is the MASK schedule with the block masks (a generalized
    cyclic G, Sec. 3.2); it converges to the stationary law."""
    csr = synth.tiny_chain(500, seed=6)
    p = oracle.transition_probs(csr)
    K = 7
    b = -(-csr.n // K)
    masks = np.zeros((K, csr.n), np.uint8)
    for k in range(K):
        masks[k, k * b:(k + 1) * b] = 1
    C1, H1 = oracle.initial_step(csr, p)
    C2, H2 = C1.copy(), H1.copy()
    i1 = oracle.solve(csr, p, C1, H1, sched=oracle.BLOCK_RR, rr_blocks=K, tol=1e-12,
                      max_steps=100000)
    i2 = oracle.solve(csr, p, C2, H2, sched=oracle.MASK, masks=masks, tol=1e-12, max_steps=100000)
    assert i1["status"] == i2["status"] == "OK" and i1["moves"] == i2["moves"]
    assert np.array_equal(H1, H2)
    ref = oracle.gth(oracle.dense_P(csr, p))
    assert np.abs(oracle.estimate(H1) - ref).sum() < 1e-10


def test_pc_large_k_is_all_nonzero_nodes():
    """With k |C_i| / ||C||_1 >= 1 for every nonzero C_i, every node with cash
    is green: the trajectory is power iteration's."""
    csr = synth.tiny_chain(300, seed=4)
    p = oracle.transition_probs(csr)
    C1, H1 = oracle.initial_step(csr, p)
    C2, H2 = C1.copy(), H1.copy()
    oracle.solve(csr, p, C1, H1, sched=oracle.PC, pc_frac=1e30, tol=0.0, max_steps=30)
    oracle.solve(csr, p, C2, H2, sched=oracle.ALL_GREEN, tol=0.0, max_steps=30)
    assert np.array_equal(C1, C2) and np.array_equal(H1, H2)


def test_pc_inclusion_frequencies():
    """Node i is green with probability min(1, k |C_i| / ||C||_1): over many
    moves (fresh draws each t) the counts match within 5 standard deviations."""
    rng = np.random.default_rng(3)
    n = 200
    C = rng.normal(size=n) * np.where(rng.random(n) < 0.1, 20.0, 1.0)
    C[::17] = 0.0
    k = 0.05 * n
    pi_ = np.minimum(1.0, k * np.abs(C) / np.abs(C).sum())
    T = 4000
    cnt = np.zeros(n)
    for t in range(T):
        g, _ = oracle.select(C, oracle.PC, move=t, pc_frac=0.05, seed=11)
        cnt += g
    sd = np.sqrt(T * pi_ * (1 - pi_)) + 1e-9
    assert np.all(np.abs(cnt - T * pi_) <= 5 * sd + 1e-9)
    assert np.all(cnt[C == 0] == 0)
    assert np.all(cnt[pi_ == 1.0] == T)


def test_pc_converges():
    csr = synth.tiny_chain(500, seed=6)
    pi, C, H, info = oracle.run(csr, sched=oracle.PC, pc_frac=0.2, seed=5, tol=1e-12,
                                max_steps=200000)
    p = oracle.transition_probs(csr)
    assert info["status"] == "OK"
    assert np.abs(pi - oracle.gth(oracle.dense_P(csr, p))).sum() < 1e-10


def test_block_rr_dobrushin_bound():
    """Sec. 3.2: for delta(P) < 1 (Eq. dobrushin) and a deterministic G that
    greens every node within m moves (Eq. cycle), ||C_t||_1 <=
    2 delta^-1 delta^(t/m). BLOCK_RR with K blocks has m = K."""
    rng = np.random.default_rng(12)
    n, K = 40, 5
    W = rng.random((n, n)) ** 3 + 0.01
    W = np.round(W * 2 ** 20) / 2 ** 20
    csr = synth.from_dense(W)
    p = oracle.transition_probs(csr)
    P = oracle.dense_P(csr, p)
    delta = 1.0 - min(np.minimum(P[i], P[k]).sum() for i in range(n) for k in range(n))
    assert 0 < delta < 1
    C, H = oracle.initial_step(csr, p)
    for t in range(1, 121):
        g, _ = oracle.select(C, oracle.BLOCK_RR, move=t - 1, rr_blocks=K)
        oracle.move(csr, p, g, C, H)
        assert np.abs(C).sum() <= 2.0 / delta * delta ** (t / K) + 1e-15


def test_degree_law_is_the_stationary_law_of_an_undirected_walk():
    """d_i / sum d solves pi = pi P for a symmetrised graph (GTH on a small
    symmetrised R-MAT with the cycle both ways and self-loops)."""
    csr = synth.rmat_chain(8, 4, seed=3, undirected=True)
    p = oracle.transition_probs(csr)
    ref = oracle.gth(oracle.dense_P(csr, p))
    assert np.abs(oracle.degree_law(csr) - ref).sum() < 1e-12


# ---------------------------------------- stale threshold (Sec. 6, theta_lag)

@pytest.mark.parametrize("sched,theta", [(oracle.THRESHOLD, 1e-10), (oracle.ALL_GREEN, 0.0)])
def test_stale_threshold_with_fixed_theta_is_one_more_move(sched, theta):
    """With a fixed threshold (or none) the stale-threshold variant differs
    from Alg. 1 only in its stop: the move whose test succeeds is still made.
    So it ends exactly one move of the plain rule later, and reports the
    tested ||C_t||_1 over the H 1 after that move."""
    csr = synth.tiny_chain(300, seed=4)
    p = oracle.transition_probs(csr)
    C0, H0 = oracle.initial_step(csr, p)
    C, H = C0.copy(), H0.copy()
    plain = oracle.solve(csr, p, C, H, sched=sched, abs_theta=theta, tol=1e-6, max_steps=100000)
    assert plain["status"] == "OK" and plain["moves"] >= 3
    l1_tested = np.abs(C).sum()
    g, _ = oracle.select(C, sched, abs_theta=theta)
    oracle.move(csr, p, g, C, H)
    C2, H2 = C0.copy(), H0.copy()
    lag = oracle.solve(csr, p, C2, H2, sched=sched, abs_theta=theta, tol=1e-6, max_steps=100000,
                       theta_lag=1)
    assert lag["status"] == "OK"
    assert lag["moves"] == plain["moves"] + 1
    assert np.array_equal(C2, C) and np.array_equal(H2, H)
    assert lag["resid"] == pytest.approx(l1_tested / abs(H.sum()), rel=1e-13)


@pytest.mark.parametrize("sched", [oracle.THRESHOLD, oracle.LINK_THRESHOLD, oracle.PC])
def test_stale_threshold_moves_use_the_previous_cash(sched):
    """Moves 1 and 2 of the variant both take their statistics from C_1 (the
    cash before move 1), move 3 from C_2: rebuilt from single selections
    whose statistics cash is given explicitly."""
    csr = synth.tiny_chain(400, seed=5)
    p = oracle.transition_probs(csr)
    C0, H0 = oracle.initial_step(csr, p)
    kw = dict(theta_scale=0.5, row_ptr=csr.row_ptr, pc_frac=0.05, seed=7)
    C, H = C0.copy(), H0.copy()
    prev = C.copy()
    g, th1 = oracle.select(C, sched, move=0, **kw)
    oracle.move(csr, p, g, C, H)
    g2, th2 = oracle.select(C, sched, move=1, cstat=prev, **kw)
    assert th2 == th1
    prev = C.copy()
    oracle.move(csr, p, g2, C, H)
    g3, _ = oracle.select(C, sched, move=2, cstat=prev, **kw)
    oracle.move(csr, p, g3, C, H)
    C2, H2 = C0.copy(), H0.copy()
    info = oracle.solve(csr, p, C2, H2, sched=sched, theta_scale=0.5, pc_frac=0.05, seed=7,
                        tol=0.0, max_steps=3, theta_lag=1)
    assert info["status"] == "ENOCONV" and info["moves"] == 3
    assert np.array_equal(C2, C) and np.array_equal(H2, H)


@pytest.mark.parametrize("sched", [oracle.THRESHOLD, oracle.LINK_THRESHOLD, oracle.PC])
def test_stale_threshold_converges_to_gth(sched):
    csr = synth.tiny_chain(1000, seed=1)
    p = oracle.transition_probs(csr)
    ref = oracle.gth(oracle.dense_P(csr, p))
    pi, C, H, info = oracle.run(csr, sched=sched, theta_scale=0.5, tol=1e-12, max_steps=200000,
                                theta_lag=1, check_every=50)
    assert info["status"] == "OK"
    assert np.abs(pi - ref).sum() <= 1e-11
    assert info["invariant"] < 1e-13 and info["l1_growth"] < 1e-15


def test_select_statistics_cash_sets_theta_and_pc_constant():
    """The statistics cash alone sets theta (THRESHOLD: theta scales with it)
    and the PC normaliser (doubling it halves every p_i, so the green set
    can only shrink for the same uniforms)."""
    rng = np.random.default_rng(3)
    C = rng.standard_normal(5000)
    g1, th1 = oracle.select(C, oracle.THRESHOLD, theta_scale=1.0)
    g2, th2 = oracle.select(C, oracle.THRESHOLD, theta_scale=1.0, cstat=3.0 * C)
    assert th2 == pytest.approx(3.0 * th1, rel=1e-14)
    assert np.array_equal(g2, (np.abs(C) >= th2).astype(np.uint8))
    p1, _ = oracle.select(C, oracle.PC, pc_frac=0.2, move=4, seed=11)
    p2, _ = oracle.select(C, oracle.PC, pc_frac=0.2, move=4, seed=11, cstat=2.0 * C)
    assert np.all(p2 <= p1) and p2.sum() < 0.7 * p1.sum()
