/*
 * RLGL oracle -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, obviously-correct FP64 CPU restatement of the Red Light
 * Green Light method (Avrachenkov, Brown, Litvak, "Red Light Green Light
 * Method for Solving Large Markov Chains", J. Sci. Comput. 93:18, 2022).
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load it. It shares no code with the CUDA library.
 *
 * Notation follows Sec. 2.1: cash C_t, history H_t, moved cash M_t, green
 * set G_t, transition matrix P = (p_ij) given by its out-links (CSR).
 *
 * Parity pins (see tests/test_oracle_pins.py): Example 3 and the two tables
 * of Example 9 (Sec. 3.3), power-iteration equivalence (Sec. 2.3.1), the
 * cash-balance invariant (Eq. recursion_H_res), the two-block mean-field
 * contraction factors (Eqs. CG1, CG2), the three-block divergence (Theorem
 * 12), GTH against brute-force solves, closed forms d_i / sum d and 1/N.
 * Every function below is pinned by at least one of them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { SCHED_ALL_GREEN = 0, SCHED_THRESHOLD = 1, SCHED_TOPFRAC = 2, SCHED_MASK = 3,
       SCHED_LINK_THRESHOLD = 4, SCHED_BLOCK_RR = 5, SCHED_PC = 6 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOTSTOCHASTIC = 2, OR_EDEGENERATE = 5, OR_ENOCONV = 6 };

/*
 * Transition probabilities from raw weights (Sec. 2.1: P is row-stochastic).
 * p_e = w_e / sum of w over row i (sum in CSR order), or 1/deg_i when w is
 * NULL, so that a repeated edge i->j carries multiplicity/deg_i in total.
 * Returns OR_ENOTSTOCHASTIC for an empty row or a non-positive weight.
 */
int oracle_transition_probs(int64_t n, const int64_t* row_ptr, const int32_t* col,
                            const float* w, double* p) {
    (void)col;
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = row_ptr[i], e = row_ptr[i + 1];
        if (e <= b) return OR_ENOTSTOCHASTIC;
        if (w) {
            double s = 0.0;
            for (int64_t k = b; k < e; ++k) {
                if (!(w[k] > 0.0f) || !isfinite(w[k])) return OR_ENOTSTOCHASTIC;
                s += (double)w[k];
            }
            for (int64_t k = b; k < e; ++k) p[k] = (double)w[k] / s;
        } else {
            double d = (double)(e - b);
            for (int64_t k = b; k < e; ++k) p[k] = 1.0 / d;
        }
    }
    return OR_OK;
}

/*
 * The update of Eqs. recursion_H and recursion_C for a given moved-cash
 * vector M:  C <- C - M + M P,  H <- H + M.  First every mover's cash M_i
 * leaves it, then it is routed to its out-neighbours in proportion to p_ij
 * (rows in increasing i, each row in CSR order), then the history grows.
 */
static void apply_moved_cash(int64_t n, const int64_t* row_ptr, const int32_t* col,
                             const double* p, const double* M, double* C, double* H) {
    for (int64_t i = 0; i < n; ++i) C[i] -= M[i];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) C[col[k]] += M[i] * p[k];
    for (int64_t i = 0; i < n; ++i) H[i] += M[i];
}

/*
 * One synchronous RLGL move for a given green set (Eq. recursion_M:
 * M_t = C_t I(G_t), i.e. M_i = C_i for i in G and 0 otherwise; then
 * apply_moved_cash). What a green node sends is its cash at the start of
 * the step. stats (nullable) receives {|G|, sum_{i in G} deg_i, sum |M_i|}.
 */
void oracle_move(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* p,
                 const uint8_t* green, double* C, double* H, double* stats) {
    double* M = (double*)calloc((size_t)n, sizeof(double));
    double cnt = 0.0, edges = 0.0, mabs = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (green[i]) {
            M[i] = C[i];
            cnt += 1.0;
            edges += (double)(row_ptr[i + 1] - row_ptr[i]);
            mabs += fabs(M[i]);
        }
    apply_moved_cash(n, row_ptr, col, p, M, C, H);
    free(M);
    if (stats) {
        stats[0] = cnt;
        stats[1] = edges;
        stats[2] = mabs;
    }
}

/*
 * Step 0 (Eq. init; the initial step of Alg. 1): C_0 = 0, H_0 = 0, G_0 = [N] and
 * the moved cash is the given distribution M_0 (uniform 1/N when m0 is
 * NULL), not C_0. Afterwards H = H_1 = M_0 and C = C_1 = -M_0 (I - P).
 */
void oracle_initial_step(int64_t n, const int64_t* row_ptr, const int32_t* col,
                         const double* p, const double* m0, double* C, double* H) {
    double* M = (double*)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        M[i] = m0 ? m0[i] : 1.0 / (double)n;
        C[i] = 0.0;
        H[i] = 0.0;
    }
    apply_moved_cash(n, row_ptr, col, p, M, C, H);
    free(M);
}

static int cmp_desc(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x < y) - (x > y);
}

/*
 * Uniform numbers of the PC schedule: the counter-based form of SplitMix64
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014). Its k-th output for seed s is mix(s + k g), with
 * g = 0x9E3779B97F4A7C15 and mix the generator's output function below.
 * Move t draws for node i the value
 *   u_{t,i} = 2^-53 floor(mix(key_t + (i + 1) g) / 2^11),
 *   key_t = mix(seed + (t + 1) g),
 * a double in [0, 1).
 */
static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The generator in its sequential form: state += g, return mix(state). */
uint64_t oracle_sm64_next(uint64_t* state) {
    *state += 0x9E3779B97F4A7C15ull;
    return sm64_mix(*state);
}

double oracle_pc_uniform(uint64_t seed, int64_t t, int64_t i) {
    const uint64_t g = 0x9E3779B97F4A7C15ull;
    const uint64_t key = sm64_mix(seed + (uint64_t)(t + 1) * g);
    return (double)(sm64_mix(key + (uint64_t)(i + 1) * g) >> 11) * 0x1.0p-53;
}

/*
 * Green-light schedules (Sec. 6, cash-dependent heuristics), in the
 * synchronous data-parallel form:
 *   ALL_GREEN : G = [N]                           (power iteration, Sec. 2.3.1)
 *   THRESHOLD : G = {i : |C_i| >= theta, C_i != 0}, with
 *               theta = scale * (sum_j |C_j|^r / N)^(1/r) from this same C
 *               (the threshold theta_t(r) of RLGL_Theta), or theta = the
 *               given absolute value when abs_theta > 0;
 *   LINK_THRESHOLD : the same test on the cash per out-link, v_i = |C_i| / d_i
 *               (d_i = out-degree counting repeats): G = {i : v_i >= theta,
 *               C_i != 0}, theta = scale * (sum_j v_j^r / N)^(1/r) or the given
 *               value. A move of node i costs d_i links (the cost unit of
 *               Sec. 6 and Sec. 4.2), so v_i is the cash moved per link used;
 *   TOPFRAC   : k = ceil(f N); theta = the k-th largest |C_i|;
 *               G = {i : |C_i| >= theta, C_i != 0} (ties all included;
 *               RLGL_MaxC widened to "large, not necessarily largest");
 *   MASK      : G = {i : mask_i != 0};
 *   BLOCK_RR  : the nodes cut into contiguous blocks of b = ceil(N / K) nodes
 *               (K = rr_blocks, at most N), K' = ceil(N / b) of them; move t
 *               (t = 0, 1, ... counted from step 0) greens block t mod K':
 *               G = {i : floor(i / b) = t mod K'}: RLGL_RR of Sec. 6 taken a
 *               block at a time, a generalized cyclic G (Sec. 3.2, Eq.
 *               cycle) with m = K';
 *   PC        : each node with C_i != 0 is green with probability
 *               p_i = min(1, k |C_i| / ||C||_1), k = pc_frac N, decided by
 *               u_{t,i} < p_i (oracle_pc_uniform): RLGL_PC of Sec. 6 (one
 *               node drawn with probability proportional to |C_i|) with
 *               about k nodes drawn at once, independently.
 * Zero-cash nodes are left out of the cash-dependent sets; moving zero cash
 * changes nothing. row_ptr is read only by LINK_THRESHOLD. `move` is t for
 * BLOCK_RR and PC. Cstat is the cash whose statistics set theta (THRESHOLD,
 * LINK_THRESHOLD, TOPFRAC) and ||C||_1 (PC); NULL means C itself (the
 * stale-threshold variant of oracle_solve passes the previous move's cash).
 * Writes green[] and returns theta (0 for the schedules without a threshold).
 */
static double select_value(int32_t sched, const int64_t* row_ptr, const double* C, int64_t i) {
    if (sched == SCHED_LINK_THRESHOLD) return fabs(C[i]) / (double)(row_ptr[i + 1] - row_ptr[i]);
    return fabs(C[i]);
}

double oracle_select(int64_t n, const int64_t* row_ptr, const double* C, int32_t sched,
                     double theta_scale, int32_t r, double abs_theta, double top_frac,
                     const uint8_t* mask, int64_t move, int64_t rr_blocks, double pc_frac,
                     uint64_t seed, const double* Cstat, uint8_t* green) {
    double theta = 0.0;
    if (!Cstat) Cstat = C;
    if (sched == SCHED_BLOCK_RR) {
        int64_t K = rr_blocks < 1 ? 1 : (rr_blocks > n ? n : rr_blocks);
        int64_t b = (n + K - 1) / K;
        int64_t nblocks = (n + b - 1) / b;
        int64_t cur = move % nblocks;
        for (int64_t i = 0; i < n; ++i) green[i] = (i / b == cur) ? 1 : 0;
        return 0.0;
    }
    if (sched == SCHED_PC) {
        double l1 = 0.0;
        for (int64_t j = 0; j < n; ++j) l1 += fabs(Cstat[j]);
        const double k = pc_frac * (double)n;
        for (int64_t i = 0; i < n; ++i) {
            green[i] = 0;
            if (C[i] == 0.0 || l1 == 0.0) continue;
            double pi_ = k * fabs(C[i]) / l1;
            if (pi_ > 1.0) pi_ = 1.0;
            green[i] = (oracle_pc_uniform(seed, move, i) < pi_) ? 1 : 0;
        }
        return 0.0;
    }
    if (sched == SCHED_ALL_GREEN) {
        for (int64_t i = 0; i < n; ++i) green[i] = 1;
        return 0.0;
    }
    if (sched == SCHED_MASK) {
        for (int64_t i = 0; i < n; ++i) green[i] = mask[i] ? 1 : 0;
        return 0.0;
    }
    if (sched == SCHED_THRESHOLD || sched == SCHED_LINK_THRESHOLD) {
        if (abs_theta > 0.0) {
            theta = abs_theta;
        } else {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                double v = select_value(sched, row_ptr, Cstat, j);
                s += (r == 1) ? v : pow(v, (double)r);
            }
            theta = (r == 1) ? theta_scale * (s / (double)n)
                             : theta_scale * pow(s / (double)n, 1.0 / (double)r);
        }
    } else { /* SCHED_TOPFRAC */
        int64_t k = (int64_t)ceil(top_frac * (double)n);
        if (k < 1) k = 1;
        if (k > n) k = n;
        double* a = (double*)malloc((size_t)n * sizeof(double));
        for (int64_t j = 0; j < n; ++j) a[j] = fabs(Cstat[j]);
        qsort(a, (size_t)n, sizeof(double), cmp_desc);
        theta = a[k - 1];
        free(a);
    }
    for (int64_t i = 0; i < n; ++i)
        green[i] = (C[i] != 0.0 && select_value(sched, row_ptr, C, i) >= theta) ? 1 : 0;
    return theta;
}

double oracle_l1(int64_t n, const double* x) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += fabs(x[i]);
    return s;
}

double oracle_sum(int64_t n, const double* x) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i];
    return s;
}

/*
 * ||C - C_0 - H (P - I)||_1 : the cash-balance identity H_t + C_t =
 * H_t P + C_0 (Eq. recursion_H_res). c0 may be NULL (C_0 = 0).
 */
double oracle_invariant_residual(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                 const double* p, const double* C, const double* H,
                                 const double* c0) {
    double* r = (double*)calloc((size_t)n, sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) r[col[k]] += H[i] * p[k];
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double hp_minus_h = r[j] - H[j];
        s += fabs(C[j] - (c0 ? c0[j] : 0.0) - hp_minus_h);
    }
    free(r);
    return s;
}

/*
 * Algorithm 1. State (C, H) holds C_t, H_t on entry (t >= 1, normally
 * straight after oracle_initial_step, i.e. t = 1) and on exit.
 * Loop, for t = 1, 2, ...:
 *   if |H_t 1| <= 1e-12 sum|H_t|            -> OR_EDEGENERATE (Sec. 2.1: the
 *                                              estimate is undefined);
 *   if t >= 2 and ||C_t||_1 / |H_t 1| < tol -> OR_OK   (the stop test of Alg. 1);
 *   if max_steps moves were made           -> OR_ENOCONV;
 *   choose G_t from C_t; move.
 * safety_every > 0 makes every safety_every-th move all-green.
 * mask (MASK schedule) holds `mask_period` green sets of n bytes, used
 * cyclically. When check != NULL, the per-step invariants are checked and
 * their worst values stored: check[0] = max |sum C| / (1 + sum|M|),
 * check[1] = max growth of ||C||_1 relative to (1 + sum|M|) (it never grows,
 * Theorem 6's proof), check[2] = max invariant residual / sum|H| (every
 * check_every steps when check_every > 0).
 * out[0] = moves made, out[1] = ||C||_1/|H 1| at exit, out[2] = edge pushes
 * (sum over moves of sum_{i in G} deg_i), out[3] = H 1. move0 = moves made
 * since step 0 before this call (the t of BLOCK_RR and PC); rr_blocks,
 * pc_frac and seed: see oracle_select.
 *
 * theta_lag = 1: the stale threshold that Sec. 6 allows for RLGL_Theta (the
 * threshold "updated less frequently"), one move stale. The first move of
 * the call is as above. Every later move t takes its statistics (theta, and
 * ||C||_1 for PC) from C_{t-1}, the cash before the previous move, and its
 * stop test from C_t in the same pass as its selection, so that the move is
 * made whatever the test says: the order of a later move is
 *   degenerate test; max_steps test; choose G_t with C_{t-1}'s statistics;
 *   move; stop with OR_OK if t >= 2 and ||C_t||_1 / |H_t 1| < tol,
 * and out[1] is then ||C_t||_1 / |H_{t+1} 1|.
 */
int oracle_solve(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* p,
                 int32_t sched, double theta_scale, int32_t r, double abs_theta,
                 double top_frac, const uint8_t* mask, int64_t mask_period,
                 int64_t safety_every, double tol, int64_t max_steps, double* C, double* H,
                 int64_t check_every, double* check, double* out, int64_t move0,
                 int64_t rr_blocks, double pc_frac, uint64_t seed, int32_t theta_lag) {
    uint8_t* green = (uint8_t*)malloc((size_t)n);
    double* Cprev = theta_lag ? (double*)malloc((size_t)n * sizeof(double)) : NULL;
    int have_prev = 0;
    int64_t moves = 0;
    double pushes = 0.0;
    int status = OR_ENOCONV;
    if (check) check[0] = check[1] = check[2] = 0.0;
    for (int64_t t = 1;; ++t) {
        double l1 = oracle_l1(n, C), hs = oracle_sum(n, H), habs = oracle_l1(n, H);
        if (out) { out[1] = (hs != 0.0) ? l1 / fabs(hs) : INFINITY; out[3] = hs; }
        if (fabs(hs) <= 1e-12 * habs || habs == 0.0) { status = OR_EDEGENERATE; break; }
        const int lagged = theta_lag && have_prev;
        const int conv = t >= 2 && l1 / fabs(hs) < tol;
        if (conv && !lagged) { status = OR_OK; break; }
        if (moves >= max_steps) { status = OR_ENOCONV; break; }
        int32_t s = sched;
        if (safety_every > 0 && (moves + 1) % safety_every == 0) s = SCHED_ALL_GREEN;
        const uint8_t* mk = (s == SCHED_MASK) ? mask + (size_t)((moves % mask_period) * n) : NULL;
        oracle_select(n, row_ptr, C, s, theta_scale, r, abs_theta, top_frac, mk, move0 + moves,
                      rr_blocks, pc_frac, seed, lagged ? Cprev : NULL, green);
        if (theta_lag) {
            memcpy(Cprev, C, (size_t)n * sizeof(double));
            have_prev = 1;
        }
        double st[3];
        oracle_move(n, row_ptr, col, p, green, C, H, st);
        ++moves;
        pushes += st[1];
        if (check) {
            double scale = 1.0 + st[2];
            double sc = fabs(oracle_sum(n, C)) / scale;
            double growth = (oracle_l1(n, C) - l1) / scale;
            if (sc > check[0]) check[0] = sc;
            if (growth > check[1]) check[1] = growth;
            if (check_every > 0 && moves % check_every == 0) {
                double ir = oracle_invariant_residual(n, row_ptr, col, p, C, H, NULL) /
                            oracle_l1(n, H);
                if (ir > check[2]) check[2] = ir;
            }
        }
        if (lagged && conv) {
            status = OR_OK;
            hs = oracle_sum(n, H);
            if (out) { out[1] = (hs != 0.0) ? l1 / fabs(hs) : INFINITY; out[3] = hs; }
            break;
        }
    }
    if (out) { out[0] = (double)moves; out[2] = pushes; }
    free(Cprev);
    free(green);
    return status;
}

/* Estimate pi_hat = H / (H 1) (Eq. pi_hat). Returns OR_EDEGENERATE when
 * |H 1| <= 1e-12 sum |H|. */
int oracle_estimate(int64_t n, const double* H, double* pi) {
    double hs = oracle_sum(n, H), habs = oracle_l1(n, H);
    if (fabs(hs) <= 1e-12 * habs || habs == 0.0) return OR_EDEGENERATE;
    for (int64_t i = 0; i < n; ++i) pi[i] = H[i] / hs;
    return OR_OK;
}

/*
 * Reference stationary law by power iteration, pi_{t+1} = pi_t P (the PI
 * reference method of Sec. 6), run until ||pi_t - pi_{t+1}||_1 <= tol or
 * maxit iterations; the reference vector used by the paper to measure errors
 * is obtained this way. The product is taken in pull form over the
 * in-links (each output entry is one sum, in a fixed order), so running it
 * on several threads gives the same bits as on one. pi holds the start
 * vector on entry (uniform when pi[0] < 0) and the result on exit.
 * Returns the iterations made; *delta_out = last ||pi_t - pi_{t+1}||_1.
 */
int64_t oracle_power_iteration(int64_t n, const int64_t* row_ptr, const int32_t* col,
                               const double* p, double tol, int64_t maxit, int32_t nthreads,
                               double* pi, double* delta_out) {
    int64_t nnz = row_ptr[n];
    int64_t* t_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* t_src = (int32_t*)malloc((size_t)nnz * sizeof(int32_t));
    double* t_p = (double*)malloc((size_t)nnz * sizeof(double));
    int64_t* cur = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    double* nxt = (double*)malloc((size_t)n * sizeof(double));
    for (int64_t k = 0; k < nnz; ++k) t_ptr[col[k] + 1]++;
    for (int64_t j = 0; j < n; ++j) t_ptr[j + 1] += t_ptr[j];
    memcpy(cur, t_ptr, (size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t q = cur[col[k]]++;
            t_src[q] = (int32_t)i;
            t_p[q] = p[k];
        }
    if (pi[0] < 0.0)
        for (int64_t i = 0; i < n; ++i) pi[i] = 1.0 / (double)n;
    int64_t it = 0;
    double delta = INFINITY;
    while (it < maxit) {
#pragma omp parallel for schedule(static) num_threads(nthreads)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int64_t q = t_ptr[j]; q < t_ptr[j + 1]; ++q) s += pi[t_src[q]] * t_p[q];
            nxt[j] = s;
        }
        delta = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            delta += fabs(nxt[j] - pi[j]);
            pi[j] = nxt[j];
        }
        ++it;
        if (delta <= tol) break;
    }
    if (delta_out) *delta_out = delta;
    free(t_ptr); free(t_src); free(t_p); free(cur); free(nxt);
    return it;
}

/*
 * Grassmann-Taksar-Heyman state reduction (the exact method cited in
 * Sec. 1.1, Grassmann, Taksar, Heyman 1985): Gaussian elimination on the
 * dense row-stochastic matrix A (n x n, row-major, overwritten) that uses
 * no subtractions. For k = n-1 .. 1: s = sum_{j<k} a_kj; a_ik /= s (i<k);
 * a_ij += a_ik a_kj (i,j<k). Back substitution: x_0 = 1,
 * x_j = sum_{i<j} x_i a_ij; pi = x / sum x.
 * Returns OR_OK, or OR_EINVAL when some s is 0 (reducible chain).
 */
int oracle_gth(int64_t n, double* A, double* pi) {
    for (int64_t k = n - 1; k >= 1; --k) {
        double s = 0.0;
        for (int64_t j = 0; j < k; ++j) s += A[k * n + j];
        if (!(s > 0.0)) return OR_EINVAL;
        for (int64_t i = 0; i < k; ++i) A[i * n + k] /= s;
        for (int64_t i = 0; i < k; ++i) {
            double aik = A[i * n + k];
            if (aik == 0.0) continue;
            for (int64_t j = 0; j < k; ++j) A[i * n + j] += aik * A[k * n + j];
        }
    }
    pi[0] = 1.0;
    double tot = 1.0;
    for (int64_t j = 1; j < n; ++j) {
        double x = 0.0;
        for (int64_t i = 0; i < j; ++i) x += pi[i] * A[i * n + j];
        pi[j] = x;
        tot += x;
    }
    for (int64_t j = 0; j < n; ++j) pi[j] /= tot;
    return OR_OK;
}
