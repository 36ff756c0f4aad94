/*
 * rlgl.h -- C ABI of librlgl: the data-parallel green-light cash-push sweep
 * of the Red Light Green Light (RLGL) method on one GPU (sm_103a).
 *
 * Method (Avrachenkov, Brown, Litvak, "Red Light Green Light Method for
 * Solving Large Markov Chains"): for an ergodic chain with row-stochastic
 * P on [N], find pi* = pi* P, sum pi* = 1 (Sec. 2.1). Every node i holds cash
 * C_i (any sign, total zero) and history H_i. At each step a set G_t of
 * nodes gets the green light; each green node adds its cash to its history
 * and routes it along its out-edges in proportion to p_ij, then its cash is
 * zero (Eqs. recursion_M, recursion_H, recursion_C; Alg. 1). The estimate is
 * pi_hat = H / (H 1) (Eq. pi_hat). All-green is power iteration (Sec. 2.3.1).
 *
 * Conventions for every entry point:
 *  - Every call returns an rlgl_status. No exception crosses the ABI, and no
 *    device code traps or asserts; a failing call leaves a message for
 *    rlgl_last_error(ctx).
 *  - Pointers marked (memspace) are host pointers when the accompanying
 *    rlgl_memspace is RLGL_HOST and device pointers (this GPU) when it is
 *    RLGL_DEVICE. Input arrays are copied into buffers owned by the context;
 *    the caller keeps ownership of everything it passes and may free it once
 *    the call returns. Outputs go to caller-allocated buffers.
 *  - A context owns all its device memory and works on one CUDA stream. Calls
 *    on one context are not thread-safe; different contexts are independent.
 *    Device memory comes from a stream-ordered pool shared by the contexts of
 *    a device, so creating and destroying contexts does not synchronise the
 *    device (freed memory up to 4 GiB is kept in the pool).
 *  - Node indices are 0-based; n < 2^27 and nnz < 2^37.
 */
#ifndef RLGL_H
#define RLGL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlgl_ctx rlgl_ctx; /* opaque; owns all its device memory */

typedef enum {
    RLGL_OK = 0,
    RLGL_EINVAL = 1,          /* bad argument or malformed CSR */
    RLGL_ENOTSTOCHASTIC = 2,  /* a row has no out-edge, or a weight is <= 0 or not finite */
    RLGL_ENOMEM = 3,          /* device or pinned host allocation failed */
    RLGL_ECUDA = 4,           /* a CUDA runtime call failed (message in rlgl_last_error) */
    RLGL_EDEGENERATE = 5,     /* |H 1| <= 1e-12 sum|H|: pi_hat undefined (Sec. 2.1, Example 3) */
    RLGL_ENOCONV = 6,         /* max_steps moves made without reaching tol */
    RLGL_ETIMEOUT = 7         /* the solve exceeded its wall-clock limit (params.time_limit_s) */
} rlgl_status;

/* Green-light schedules (Sec. 6 heuristics, synchronous data-parallel form).
 *  ALL_GREEN : G = [N] (power iteration, Sec. 2.3.1).
 *  THRESHOLD : G = {i : |C_i| >= theta, C_i != 0} (RLGL_Theta's test). theta
 *              = the call's theta when > 0, else
 *              params.theta_scale * (sum_j |C_j|^r / N)^(1/r) from the same C.
 *  TOPFRAC   : k = ceil(f N) with f = the call's theta when in (0,1], else
 *              params.top_frac; theta = k-th largest |C_i|, exact;
 *              G = {i : |C_i| >= theta, C_i != 0} (ties included; RLGL_MaxC
 *              widened to a fraction).
 *  MASK      : G = the current set from rlgl_set_masks (cycled).
 *  LINK_THRESHOLD : the THRESHOLD test applied to the cash per out-link,
 *              v_i = |C_i| / d_i (d_i = out-degree counting repeats):
 *              G = {i : v_i >= theta, C_i != 0}, theta = the call's theta when
 *              > 0, else params.theta_scale * (sum_j v_j^r / N)^(1/r). Moving
 *              node i costs d_i links, the paper's unit of work (Sec. 6), so v_i
 *              is the cash moved per link used.
 *  BLOCK_RR  : RLGL_RR (Sec. 6) a block at a time: nodes in contiguous blocks
 *              of b = ceil(N / K) nodes, K = params.rr_blocks clipped to
 *              [1, N]; move t (t - 1 = moves made since step 0) greens block
 *              (t - 1) mod ceil(N / b). A generalized cyclic G (Sec. 3.2).
 *  PC        : RLGL_PC (Sec. 6) drawing about k = params.pc_frac N nodes at
 *              once: node i is green when C_i != 0 and
 *              u ||C||_1 < k |C_i| (in FP64), u the SplitMix64 draw of node i
 *              for this move: key = mix(seed + t g), u = 2^-53 *
 *              floor(mix(key + (i + 1) g) / 2^11), g = 0x9E3779B97F4A7C15,
 *              mix the generator's output function (Steele, Lea and Flood,
 *              OOPSLA 2014).
 *  BLOCK_RR and PC serve single chains only (EINVAL in batch mode). */
typedef enum {
    RLGL_ALL_GREEN = 0,
    RLGL_THRESHOLD = 1,
    RLGL_TOPFRAC = 2,
    RLGL_MASK = 3,
    RLGL_LINK_THRESHOLD = 4,
    RLGL_BLOCK_RR = 5,
    RLGL_PC = 6
} rlgl_schedule;

/* FP64: cash, moved cash and history in FP64.
 * MIXED: cash and per-edge products in FP32, history and every reduction in
 * FP64; the cash is re-derived in FP64 from the history, C = C_0 + H (P - I)
 * (Eq. recursion_H_res), whenever ||C||_1 has fallen by params.refresh_factor
 * since the last re-derivation, when it has stopped falling (params.stall_moves),
 * and always before a solve reports convergence. */
typedef enum { RLGL_FP64 = 0, RLGL_MIXED = 1 } rlgl_precision;

typedef enum { RLGL_HOST = 0, RLGL_DEVICE = 1 } rlgl_memspace;

typedef struct {
    double theta_scale;     /* THRESHOLD auto-theta multiplier (default 1) */
    int32_t r;              /* exponent r of theta_t(r) (default 1) */
    double top_frac;        /* TOPFRAC fraction when the call's theta is not in (0,1] (default 0.01) */
    double pull_crossover;  /* a move whose green edges reach this fraction of nnz pulls over
                               the in-links instead of pushing (default 0.9: on GB300 a pull
                               over all in-links costs about as much as pushing every edge) */
    int32_t safety_every;   /* every K-th move of a solve is all-green (0 = never, default) */
    double refresh_factor;  /* MIXED only: see rlgl_precision (default 1e-4; 0 = only at the end) */
    double time_limit_s;    /* wall-clock limit of one rlgl_solve, checked on the device (default 600) */
    int64_t rr_blocks;      /* BLOCK_RR: number of blocks K (default 8) */
    double pc_frac;         /* PC: expected green fraction k / N before capping (default 0.05) */
    uint64_t seed;          /* PC: seed of the counter-based draws (default 0) */
    int32_t persistent;     /* 1 (default): a single-chain solve with any schedule runs as one
                               persistent cooperative kernel per stretch between FP64
                               re-derivations of the cash, with grid barriers between the phases
                               of a move (TOPFRAC: one more per radix pass of its threshold);
                               0: one kernel per phase. Same moves either way. */
    double barrier_limit_s; /* persistent sweep: longest wait at a grid barrier (default 2,
                               at most 60); a wait that runs out ends the solve with
                               RLGL_ETIMEOUT and leaves the context usable */
    int32_t test_skip_barrier; /* testing only (default 0): 1 makes one block of the sweep
                                  leave before its first barrier, so that the others' wait
                                  runs out (exercises the bounded wait without a fault) */
    int32_t stall_moves;    /* MIXED only: re-derive the cash also when ||C||_1 has not fallen
                               below its value of this many moves ago (FP32 rounding floor, e.g.
                               in a node with a million in-links); 0 = off (default 32) */
    int32_t theta_lag;      /* 1: stale threshold, one move old (Sec. 6 lets RLGL_Theta's
                               threshold be updated less often). The first move of a solve call
                               is as with 0; every later move takes theta (and ||C||_1 for PC)
                               from the cash before the previous move, computes its own cash's
                               statistics while it selects, and is made whatever its stop test
                               says (the call stops after it; solve_info.resid is then
                               ||C_t||_1 / |H_{t+1} 1|). Saves the statistics pass and one grid
                               barrier per move. Persistent sweep only: rlgl_solve returns
                               RLGL_EINVAL for TOPFRAC, batches and persistent = 0; rlgl_step
                               and rlgl_profile_moves ignore it. Default 0 */
    int32_t batch_block;    /* threads per block of the persistent batch solve: 128, 256 (default)
                               or 512 (the merge-path tiles of the chains' pulls hold 1024, 2048
                               and 2048 rows + links) */
} rlgl_params;

typedef struct {
    int64_t green;          /* |G_t| */
    int64_t edges_pushed;   /* sum_{i in G_t} deg_i: links used by the move (Sec. 6) */
    int32_t mode;           /* 0 none, 1 push over out-links, 2 pull over in-links */
    double theta;           /* threshold used (THRESHOLD / TOPFRAC), else 0 */
    double l1_cash;         /* ||C_{t+1}||_1 after the move */
    double sum_cash;        /* sum C_{t+1} (zero up to rounding) */
    double sum_hist;        /* H_{t+1} 1 */
} rlgl_step_info;

typedef struct {
    int64_t moves;          /* moves made by this call */
    int64_t edges_pushed;   /* links used by those moves */
    int64_t green_total;    /* sum of |G_t| */
    int64_t push_moves, pull_moves, refreshes;
    int64_t iterations;     /* device-loop iterations (moves + re-derivation-only passes + the final test) */
    double resid;           /* ||C||_1 / |H 1| at exit (Alg. 1's stopping quantity) */
    double l1_cash, sum_hist;
} rlgl_solve_info;

/* One entry of the per-move log (see rlgl_move_log). */
typedef struct {
    int64_t move;           /* t - 1: moves made since step 0 when this one started */
    int64_t green;          /* |G_t| */
    int64_t edges_pushed;   /* sum_{i in G_t} deg_i */
    int32_t mode;           /* 0 none, 1 push, 2 pull */
    double theta;           /* threshold used (0 when none) */
    double l1_cash;         /* ||C_t||_1 before the move */
    double sum_hist;        /* H_{t+1} 1 after the move */
    float phase_us[6];      /* persistent sweep only (else 0), from block 0's clock: stats work,
                               wait at the barrier after it, select work (with the decisions),
                               wait, push/pull work, wait; microseconds. A move of the stale
                               threshold has no statistics pass: its first two are 0 */
} rlgl_move_record;

/* Fills p with the defaults listed in rlgl_params. */
rlgl_status rlgl_default_params(rlgl_params* p);

/*
 * Creates a context for the chain given by its out-links (CSR), uploads it,
 * builds the in-link (CSC) copy used by pull moves and residuals, and
 * performs step 0 (Eq. init; the initial step of Alg. 1): H = H_1 = M_0 and
 * C = C_1 = -M_0 (I - P), total zero.
 *   n, nnz   : nodes and edges; row i's out-edges are col[row_ptr[i] ..
 *              row_ptr[i+1]-1].
 *   row_ptr  : (src) int64 [n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 *   col      : (src) int32 [nnz], 0 <= col < n. Repeated (i, j) pairs add.
 *   w        : (src) float [nnz] raw positive weights, p_ij = w_ij / sum_k w_ik;
 *              NULL means unit weights, p_ij = multiplicity / out-degree.
 *   m0       : (src) double [n], the step-0 distribution M_0; NULL = uniform 1/N.
 *   prec     : RLGL_FP64 or RLGL_MIXED.
 *   src      : memspace of row_ptr, col, w, m0.
 *   stream   : cudaStream_t to work on (NULL: the context creates its own).
 * Every row needs at least one out-edge (else RLGL_ENOTSTOCHASTIC).
 */
rlgl_status rlgl_create(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                        const float* w, const double* m0, rlgl_precision prec,
                        rlgl_memspace src, void* stream, rlgl_ctx** out);

/*
 * As rlgl_create, but starts from a given state (c, h) (src memspace, double
 * [n] each; checkpoint resume) instead of step 0. C_0 := c - h (P - I) is
 * recorded so that the invariant of Eq. recursion_H_res is checked against
 * it. Returns RLGL_EINVAL when |sum c| > 1e-12 max(1, ||c||_1).
 */
rlgl_status rlgl_create_from_state(int64_t n, int64_t nnz, const int64_t* row_ptr,
                                   const int32_t* col, const float* w, const double* c,
                                   const double* h, rlgl_precision prec, rlgl_memspace src,
                                   void* stream, rlgl_ctx** out);

/*
 * A batch of independent chains in one context (many chains, one launch per
 * kernel): the chains are stacked block-diagonally, chain k owning the nodes
 * node_ptr[k] .. node_ptr[k+1]-1, and no edge may leave its chain
 * (RLGL_EINVAL otherwise). Every chain runs Alg. 1 on its own: its own
 * statistics, threshold (THRESHOLD / LINK_THRESHOLD), stopping test and
 * tolerance, and its own estimate pi_hat = H / (H 1) over its nodes. Step 0
 * uses M_0 uniform within each chain. A chain that stops is frozen while
 * the others continue; rlgl_solve returns when every chain has stopped
 * (RLGL_OK when all converged, else the worst of ETIMEOUT, EDEGENERATE,
 * ENOCONV) and rlgl_batch_chains reports each chain. RLGL_TOPFRAC is not
 * available for a batch. The other arguments are those of rlgl_create,
 * with node ids global (0..n-1); node_ptr is int64 [n_chains+1] in src.
 */
rlgl_status rlgl_batch_create(int64_t n_chains, const int64_t* node_ptr, int64_t n, int64_t nnz,
                              const int64_t* row_ptr, const int32_t* col, const float* w,
                              rlgl_precision prec, rlgl_memspace src, void* stream, rlgl_ctx** out);

/* Per-chain tolerances (host double [n_chains], each >= 0), used by
 * rlgl_solve when its tol argument is negative. */
rlgl_status rlgl_batch_set_tol(rlgl_ctx* ctx, const double* tol);

/* Per chain (host arrays of n_chains, each nullable): the status of its last
 * solve (a rlgl_status value; -1 while running), moves made since step 0,
 * and ||C||_1 / |H 1|. */
rlgl_status rlgl_batch_chains(rlgl_ctx* ctx, int32_t* status, int64_t* moves, double* resid);

/* Step 0 again with a new M_0 (src memspace, double [n]; NULL = uniform,
 * within each chain for a batch),
 * keeping the uploaded chain. Clears the recorded C_0. */
rlgl_status rlgl_reset(rlgl_ctx* ctx, const double* m0, rlgl_memspace src);

/* Green sets for RLGL_MASK: `period` sets of n bytes (nonzero = green),
 * row-major, used cyclically from the first one on. src memspace. */
rlgl_status rlgl_set_masks(rlgl_ctx* ctx, const uint8_t* masks, int64_t period,
                           rlgl_memspace src);

/*
 * One synchronous move (the move of Alg. 1): choose G_t from the
 * current cash by the schedule, then C <- C - M_t (I - P), H <- H + M_t with
 * M_t = C_t I(G_t). theta: see rlgl_schedule. info may be NULL (then the call
 * does not wait for the GPU); when given, the call synchronises and fills it.
 */
rlgl_status rlgl_step(rlgl_ctx* ctx, rlgl_schedule sched, double theta, rlgl_step_info* info);

/*
 * Algorithm 1 until t >= 2 and ||C_t||_1 / |H_t 1| < tol (its stop test), or
 * max_steps moves (RLGL_ENOCONV), or a degenerate history (RLGL_EDEGENERATE).
 * The whole loop runs on the device as one CUDA graph with a conditional
 * while-node: no host round trip per move. tol = 0 with max_steps = T makes
 * exactly T moves. Synchronises before returning; info may be NULL.
 * 1 <= max_steps <= 10^8 (else RLGL_EINVAL).
 */
rlgl_status rlgl_solve(rlgl_ctx* ctx, rlgl_schedule sched, double theta, double tol,
                       int64_t max_steps, rlgl_solve_info* info);
/* (For a batch, tol >= 0 applies to every chain and tol < 0 uses the
 * per-chain tolerances of rlgl_batch_set_tol.) */

/* rlgl_solve split in two, so that the host can do other work (or drive
 * other contexts) while the device loop runs: rlgl_solve_async queues the
 * solve graph on the context's stream and returns; rlgl_query sets
 * *finished to 1 once it has completed (or when nothing is pending);
 * rlgl_wait waits, fills info and returns the solve's status exactly as
 * rlgl_solve would. Between rlgl_solve_async and rlgl_wait every other call
 * on the context returns RLGL_EINVAL. */
rlgl_status rlgl_solve_async(rlgl_ctx* ctx, rlgl_schedule sched, double theta, double tol,
                             int64_t max_steps);
rlgl_status rlgl_query(rlgl_ctx* ctx, int32_t* finished);
rlgl_status rlgl_wait(rlgl_ctx* ctx, rlgl_solve_info* info);

/* pi_hat = H / (H 1) (Eq. pi_hat), FP64, into pi_out (dst memspace, double
 * [n]). RLGL_EDEGENERATE when |H 1| <= 1e-12 sum|H| (pi_out untouched). */
rlgl_status rlgl_estimate(rlgl_ctx* ctx, double* pi_out, rlgl_memspace dst);

/* The estimate restricted to the nodes [lo, hi) and normalised over them:
 * pi_out[i - lo] = H_i / sum_{k in [lo, hi)} H_k (FP64; dst memspace, double
 * [hi - lo]). With the auxiliary-node chain P^(0) of Sec. 2.3.2 (node 0 the
 * auxiliary node) the range [1, N) gives the PageRank vector of the original
 * nodes (Eq. pi_hat over the original nodes). RLGL_EINVAL unless
 * 0 <= lo < hi <= n, and for a batch; RLGL_EDEGENERATE when |sum H| <=
 * 1e-12 sum|H| over the range (pi_out untouched). */
rlgl_status rlgl_estimate_range(rlgl_ctx* ctx, int64_t lo, int64_t hi, double* pi_out,
                                rlgl_memspace dst);

/* Current (C_t, H_t) as FP64 (dst memspace; either pointer may be NULL). */
rlgl_status rlgl_get_state(rlgl_ctx* ctx, double* c, double* h, rlgl_memspace dst);

/* ||C_t - C_0 - H_t (P - I)||_1 in FP64 (Eq. recursion_H_res): zero up to
 * rounding on the FP64 path; the accumulated FP32 drift on the MIXED path. */
rlgl_status rlgl_invariant_residual(rlgl_ctx* ctx, double* l1);

/* Re-derives C = C_0 + H (P - I) in FP64 (rounded to the cash type) and
 * returns the residual it removed in *l1_before (nullable). */
rlgl_status rlgl_refresh(rlgl_ctx* ctx, double* l1_before);

rlgl_status rlgl_set_params(rlgl_ctx* ctx, const rlgl_params* p);
rlgl_status rlgl_get_params(const rlgl_ctx* ctx, rlgl_params* p);

/* Per-kernel-class device time (ms) and launch counts accumulated while
 * profiling is on (rlgl_profile(ctx, 1)): eager moves then record a CUDA
 * event pair around every kernel on the context's stream. Classes, in order:
 * 0 stats, 1 select, 2 push, 3 pull, 4 top-k select, 5 refresh,
 * 6 persistent sweep. ms[7], launches[7]. rlgl_profile(ctx, 0) stops and clears nothing;
 * rlgl_profile(ctx, 2) clears. */
rlgl_status rlgl_profile(rlgl_ctx* ctx, int32_t mode);
rlgl_status rlgl_kernel_times(rlgl_ctx* ctx, double* ms, int64_t* launches);

/* Profiling run: `moves` eager moves (as rlgl_step) whose kernels are all
 * queued before the stream is released, with a CUDA event pair around every
 * kernel, so each pair measures the kernel's own device time. Adds to the
 * totals read by rlgl_kernel_times. Synchronises. */
rlgl_status rlgl_profile_moves(rlgl_ctx* ctx, rlgl_schedule sched, double theta, int64_t moves);

/* Profiling run of the persistent sweep (params.persistent): `moves` moves
 * made as a solve with tol 0 and max_steps = moves, the sweep launched
 * eagerly with a CUDA event pair around each launch (class 6) and around
 * each FP64 re-derivation kernel (class 5). EINVAL when the sweep does not
 * serve the context (batch) or the setting (TOPFRAC with theta_lag).
 * Synchronises; the
 * solve ends with status ENOCONV on the device, which this call does not
 * report. */
rlgl_status rlgl_profile_sweep(rlgl_ctx* ctx, rlgl_schedule sched, double theta, int64_t moves);

/* Copies the log of the last min(count, 65536) moves, oldest first, into
 * out (host, count entries); *written receives the number copied. The log
 * is kept on the device by the select kernel and survives rlgl_reset. */
rlgl_status rlgl_move_log(rlgl_ctx* ctx, rlgl_move_record* out, int64_t count, int64_t* written);

/*
 * ||C - C_0 - H (P - I)||_1 for a state held in the caller's own device
 * buffers, computed without allocating any device memory. The paper has no
 * counterpart: this entry point exists for callers that may not call
 * cudaMalloc or cudaFree, for example a service whose device memory belongs
 * to a framework's pool (cudaFree also synchronises the whole device).
 *   n, nnz, row_ptr, col, w : the chain as for rlgl_create, all DEVICE
 *              pointers (w may be NULL: unit weights).
 *   c, h     : device double [n], the cash C_t and history H_t.
 *   c0       : device double [n] or NULL (C_0 = 0).
 *   l1_out   : device double [1]; receives the residual, or NaN when an
 *              index of the CSR is out of range, a row is empty, or a row's
 *              weights do not sum to a positive number.
 *   stream   : cudaStream_t the work is queued on (NULL: legacy stream).
 * Asynchronous: returns after queueing three kernels; *l1_out is ready when
 * the stream reaches that point. Its scratch is one fixed array in device
 * memory (8 MiB of accumulators plus 8 KiB), held by every GPU that loads
 * the library until the process exits, so n is limited to 2^20 nodes:
 * RLGL_EINVAL beyond that, for NULL pointers, or for n or nnz < 1. RLGL_ECUDA
 * when a launch fails, or, with nothing queued, when an error of earlier
 * work is already pending on the calling thread (that error is left pending
 * for its owner, not cleared). The first call on each device looks up that
 * array's device address (cudaGetSymbolAddress). All calls on a device share
 * the array and each one clears it first, so calls whose work overlaps on
 * the GPU (two streams, or two threads) race and give wrong results;
 * serialise them.
 */
rlgl_status rlgl_invariant_residual_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr,
                                            const int32_t* col, const float* w, const double* c,
                                            const double* h, const double* c0, double* l1_out,
                                            void* stream);

/* Device bytes a context for such a chain (or batch of n_chains) holds once
 * created, for admission control; -1 for n or nnz < 1. Transient memory
 * during creation (the in-link build) adds about (n + 1) 8 bytes. */
int64_t rlgl_footprint(int64_t n, int64_t nnz, int32_t weighted, rlgl_precision prec,
                       int64_t n_chains);

/* The CUDA stream the context works on (cudaStream_t). */
void* rlgl_stream(const rlgl_ctx* ctx);

/* Last error message of ctx (or of the calling thread when ctx is NULL). */
const char* rlgl_last_error(const rlgl_ctx* ctx);
const char* rlgl_status_string(rlgl_status s);

/* Destroys the solve graphs kept from destroyed contexts and returns how
 * many there were. rlgl_destroy does not destroy a context's executable
 * graphs itself, because that can wait for unrelated work still running on
 * the device; call this where no solve is running (it may wait for the
 * device otherwise). */
int64_t rlgl_release_retired(void);

/* Frees the context and all its device memory (NULL is a no-op); its solve
 * graphs are kept until rlgl_release_retired. */
void rlgl_destroy(rlgl_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RLGL_H */
