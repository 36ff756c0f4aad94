// Device kernels of the RLGL green-light sweep (sm_103a).
//
// One move of Alg. 1 (Eqs. recursion_M, recursion_H, recursion_C) runs as
//   stats   : ||C||_1, sum C, sum |C|^r in FP64 (the stop test of Alg. 1;
//             threshold theta_t(r), Sec. 6) + solve control;
//   [top-k] : exact k-th largest |C| by radix select (TOPFRAC);
//   select  : G = {i : |C_i| >= theta, C_i != 0}; for i in G: m_i = C_i,
//             C_i <- 0, H_i += m_i (FP64); frontier compaction with warp
//             ballots and a block scan; chooses push or pull;
//   push    : c_j += m_i p_ij over the frontier's out-links (edge-balanced
//             chunks, red.global adds), or
//   pull    : c_j += sum_{i in in(j)} m_i p_ij over the in-links (merge-path
//             tiles staged in shared memory; no atomics for whole rows).
// The MIXED path re-derives C = C_0 + H (P - I) in FP64 (Eq.
// recursion_H_res) with the same merge-path pull.
//
// p_ij is never materialised: s_i = 1 / sum_k w_ik is kept per row (FP64)
// and a green row sends m~_i = m_i s_i, so edge (i, j) carries m~_i w_ij
// (unit weights: w_ij = 1, s_i = 1 / deg_i).
//
// No kernel spins or waits on another block: cross-block results are
// combined by the last block to finish (an atomic ticket), so nothing here
// can hang.
#pragma once
#include <cstddef>
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace rlgl {

constexpr int kThreads = 256;         // threads per block, every kernel
constexpr int kNodesPerThread = 4;    // node kernels: nodes per thread per block-iteration
constexpr int kNodesPerIter = kThreads * kNodesPerThread;
constexpr int kPushChunk = 1024;      // edges per push chunk
constexpr int kMpIpt = 8;             // merge-path items per thread
constexpr int kMpItems = kThreads * kMpIpt;  // merge-path items (rows + edges) per tile
constexpr int kCountBits = 27;        // frontier reservation: (edges << 27) | count
constexpr int kRadixBits = 11;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kMaxGrid = 4096;
constexpr int kLogCap = 1 << 16;      // per-move log entries (ring)

struct MoveRecord {                   // layout of rlgl_move_record
    long long move, green, edges;
    int mode, pad;
    double theta, l1, hsum;
    float phase_us[6];
};

// Per-chain state of a batch (many independent chains on one block-diagonal
// CSR). acc[] are atomic accumulators, zero at rest: 0 ||C||_1, 1 sum C,
// 2 sum v^r, 3 sum of moved cash, 4 sum |moved cash|, 5 sum H, 6 sum |H|.
struct ChainState {
    double acc[7];
    double l1, sum, sumr, theta, hsum, habs, tol;
    double l1r;              // persistent batch: ||C||_1 after the last re-derivation
    long long n, moves;
    // persistent batch: the last solve's moves, links, green nodes, push and
    // pull moves and re-derivations of this chain
    long long s_moves, s_edges, s_green, s_push, s_pull, s_refr;
    float theta_f;
    int done, status, fresh;  // fresh: the cash is exact (step 0 or re-derived)
};

struct BatchView {
    const int* chain_of;   // node -> chain
    ChainState* cs;
    int nchains;
};

enum Mode : int { MODE_NONE = 0, MODE_PUSH = 1, MODE_PULL = 2 };
enum Sched : int {
    SCHED_ALL_GREEN = 0,
    SCHED_THRESHOLD = 1,
    SCHED_TOPFRAC = 2,
    SCHED_MASK = 3,
    SCHED_LINK = 4,
    SCHED_BLOCK_RR = 5,
    SCHED_PC = 6
};
enum Status : int { ST_OK = 0, ST_DEGENERATE = 5, ST_NOCONV = 6, ST_TIMEOUT = 7 };

// Parameters the host writes before a solve or a step (one memcpy).
struct Control {
    double tol;
    double theta_arg;        // the call's theta
    double theta_scale;
    double top_frac;
    double pull_crossover;
    double refresh_factor;
    double time_limit_ns;
    long long max_steps;
    long long max_iters;
    long long nnz;
    long long rr_blocks;     // BLOCK_RR: K
    double pc_frac;          // PC: k = pc_frac N
    unsigned long long seed; // PC: generator seed
    unsigned long long barrier_limit_ns;  // persistent sweep: longest barrier wait
    int test_skip_barrier;   // persistent sweep: one block leaves before its first barrier
    int stall_moves;         // MIXED: re-derive when ||C||_1 has not fallen in this many moves
    int sched;
    int r;
    int safety_every;
    int solving;             // 1: solve (stop tests active), 0: single step
    int mixed;               // MIXED precision path
    int n_masks;
    int theta_lag;           // persistent sweep: theta from the previous move's cash
    int pad[1];
};

struct DevState {
    Control ctl;
    // statistics of the current cash (written by the stats kernel)
    double l1, sum, sumr, theta;
    float theta_f;           // FP32 threshold of the MIXED path (see set_theta)
    float pad_f;
    double hsum, habs;       // H 1 (kept incrementally) and an upper bound of sum |H|
    double l1_refresh;       // ||C||_1 right after the last re-derivation
    double stall_mark;       // ||C||_1 at the start of the current stall window (MIXED)
    long long stall_count;   // moves in the current stall window
    double resid_l1;         // residual measured by the last refresh pass
    double last_mabs;
    // last move and totals
    long long green, edges;
    long long moves;         // moves since step 0 (t - 1)
    long long solve_moves, iters, mask_cursor;
    long long tot_green, tot_edges, push_moves, pull_moves, refreshes;
    long long base_green, base_edges, base_push, base_pull, base_refreshes;  // at solve start
    unsigned long long t_start;
    unsigned long long reserve;   // packed frontier reservation
    unsigned int ticket;
    int mode, done, status, fresh, want_refresh, skip_move, force_refresh, apply_refresh;
    // top-k radix select
    unsigned long long tk_prefix;
    long long tk_remain;
    int tk_shift, tk_width;
    unsigned int hist[kRadixBins];
};

// ----------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T> struct KeyOf;
template <> struct KeyOf<float> {
    using K = unsigned int;
    static constexpr int bits = 31;
    __device__ static K key(float v) { return __float_as_uint(v) & 0x7fffffffu; }
    __device__ static double value(unsigned long long k) { return (double)__uint_as_float((unsigned)k); }
};
template <> struct KeyOf<double> {
    using K = unsigned long long;
    static constexpr int bits = 63;
    __device__ static K key(double v) { return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull; }
    __device__ static double value(unsigned long long k) { return __longlong_as_double((long long)k); }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block; the result is valid in thread 0. scratch: 32 T.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    T s = 0;
    if (wid == 0) {
        s = (lane < (int)(blockDim.x >> 5)) ? scratch[lane] : T(0);
        s = warp_sum(s);
    }
    return s;
}

// K block sums at once (two barriers in all); thread 0 receives the totals
// in v. scratch holds K * 32 values.
template <typename T, int K>
__device__ __forceinline__ void block_sum_n(T (&v)[K], T* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) scratch[k * 32 + wid] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const T x = (lane < (int)(blockDim.x >> 5)) ? scratch[k * 32 + lane] : T(0);
            v[k] = warp_sum(x);
        }
    }
}

// Block-wide exclusive scan of 64-bit values (blockDim = kBT). Returns
// the exclusive prefix; *total receives the block total (all threads).
template <int kBT = kThreads>
__device__ __forceinline__ unsigned long long block_exscan(unsigned long long v,
                                                           unsigned long long* total) {
    __shared__ unsigned long long wsum[kBT / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long s = (lane < kBT / 32) ? wsum[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kBT / 32) wsum[lane] = s;  // inclusive warp prefixes
    }
    __syncthreads();
    unsigned long long before = (wid > 0) ? wsum[wid - 1] : 0ull;
    *total = wsum[kBT / 32 - 1];
    return before + x - v;
}

// Last-block-done: every block calls this after writing its partials; the
// return value is true in exactly one block (the last), whose threads then
// see every other block's partials. Resets the ticket for the next kernel.
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) *ticket = 0u;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// Reductions into global memory whose old value nobody reads: red.global
// (no value comes back, so the issuing warp tracks nothing).
__device__ __forceinline__ void red_add(float* p, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// Loads of data that other blocks of the same kernel may have written: from
// L2 (ld.global.cg) when kCg, so that no stale L1 line is read.
template <bool kCg, typename T>
__device__ __forceinline__ T ld_shared_data(const T* p) {
    if (kCg) return __ldcg(p);
    return *p;
}


// In the last block: out[k] = sum over blocks b of part[K b + k], with all
// threads of the block, in a fixed order (per-thread strided sums, then a
// fixed tree), so the result does not depend on block scheduling. The
// result is valid in thread 0.
template <int K>
__device__ __forceinline__ void reduce_partials(const double* part, int nb, double* out) {
    __shared__ double scratch[32];
    // Groups of 4 partials per thread, each group's loads issued before its
    // adds: one round trip per group (one in all for up to 1024 blocks).
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int g0 = 0; g0 < nb; g0 += 4 * kThreads) {
        double v[4][K];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = g0 + threadIdx.x + u * kThreads;
#pragma unroll
            for (int k = 0; k < K; ++k) v[u][k] = (b < nb) ? ldcg(part + K * b + k) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] += v[u][k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = block_sum(acc[k], scratch);
}

// The scalar part of the device state (everything before the radix
// histogram), staged in shared memory by the last block of a kernel: one
// parallel load, the bookkeeping on the copy, one parallel store. This keeps
// the serial tail of a kernel from paying one global round trip per field.
constexpr int kStWords = (int)(offsetof(DevState, hist) / sizeof(unsigned int));
struct StStage {
    unsigned int w[kStWords];
};
__device__ __forceinline__ DevState* st_stage_in(const DevState* st, StStage* sh) {
    const unsigned int* src = reinterpret_cast<const unsigned int*>(st);
    for (int k = threadIdx.x; k < kStWords; k += blockDim.x) sh->w[k] = __ldcg(src + k);
    __syncthreads();
    return reinterpret_cast<DevState*>(sh);
}
__device__ __forceinline__ void st_stage_out(DevState* st, const StStage* sh) {
    __syncthreads();
    unsigned int* dst = reinterpret_cast<unsigned int*>(st);
    for (int k = threadIdx.x; k < kStWords; k += blockDim.x) dst[k] = sh->w[k];
}

// ------------------------------------------------------- stats + control

// Stores theta and its FP32 form for the MIXED path. For the |C| tests the
// FP32 threshold is theta rounded up, so that for an FP32 cash value v,
// |v| >= theta_f exactly when |v| >= theta; the per-link test compares an
// FP32 product and uses theta rounded to nearest.
__device__ __forceinline__ void set_theta(DevState* st, double theta, int sched) {
    st->theta = theta;
    st->theta_f = (sched == SCHED_LINK) ? __double2float_rn(theta) : __double2float_ru(theta);
}

// Per-move constants of the cash-independent and sampled schedules.
//   BLOCK_RR: nodes in contiguous blocks of rr_b = ceil(N / K) (K clipped to
//             [1, N]); move t greens block t mod ceil(N / rr_b).
//   PC      : node i is green when C_i != 0 and u_{t,i} ||C||_1 < k |C_i|,
//             i.e. u_{t,i} < min(1, k |C_i| / ||C||_1) (k = pc_frac N), with
//             u_{t,i} the counter-based SplitMix64 draw (Steele, Lea and
//             Flood 2014): key_t = mix(seed + (t + 1) g), u_{t,i} =
//             2^-53 floor(mix(key_t + (i + 1) g) / 2^11).
struct SchedAux {
    long long rr_lo, rr_hi;   // BLOCK_RR: the green block [rr_lo, rr_hi)
    double pc_k, pc_l1;
    unsigned long long pc_key;
};

constexpr unsigned long long kSm64Gamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ SchedAux sched_aux(const Control& c, long long n, long long move, double l1,
                                              int sched) {
    SchedAux a;
    a.rr_lo = a.rr_hi = 0;
    a.pc_k = a.pc_l1 = 0.0;
    a.pc_key = 0ull;
    if (sched == SCHED_BLOCK_RR) {
        long long K = c.rr_blocks < 1 ? 1 : (c.rr_blocks > n ? n : c.rr_blocks);
        const long long b = (n + K - 1) / K;
        const long long nb = (n + b - 1) / b;
        a.rr_lo = (move % nb) * b;
        a.rr_hi = a.rr_lo + b < n ? a.rr_lo + b : n;
    } else if (sched == SCHED_PC) {
        a.pc_k = c.pc_frac * (double)n;
        a.pc_l1 = l1;
        a.pc_key = sm64_mix(c.seed + (unsigned long long)(move + 1) * kSm64Gamma);
    }
    return a;
}

// Whether node i (cash v, 1/out-degree idg) is green under `sched`
// (ALL_GREEN, THRESHOLD, LINK_THRESHOLD, MASK, BLOCK_RR, PC; TOPFRAC uses
// THRESHOLD's test with its radix-selected theta).
template <typename T>
__device__ __forceinline__ bool green_test_v(int sched, T v, T idg, long long i, T th,
                                             const unsigned char* mask, const SchedAux& ax) {
    switch (sched) {
        case SCHED_ALL_GREEN: return true;
        case SCHED_MASK: return mask[i] != 0;
        case SCHED_LINK: return (v != T(0)) && (fabs(v) * idg >= th);
        case SCHED_BLOCK_RR: return i >= ax.rr_lo && i < ax.rr_hi;
        case SCHED_PC: {
            if (v == T(0)) return false;
            const double u = (double)(sm64_mix(ax.pc_key + (unsigned long long)(i + 1) * kSm64Gamma) >> 11) *
                             0x1.0p-53;
            return u * ax.pc_l1 < ax.pc_k * fabs((double)v);
        }
        default: return (v != T(0)) && (fabs(v) >= th);
    }
}

template <typename T>
__device__ __forceinline__ bool green_test(int sched, T v, long long i, T th,
                                           const unsigned char* mask, const T* __restrict__ ideg,
                                           const SchedAux& ax) {
    const T idg = (sched == SCHED_LINK) ? __ldg(ideg + i) : T(0);
    return green_test_v<T>(sched, v, idg, i, th, mask, ax);
}

constexpr double kNoMark = 1e300;

// MIXED path: FP32 rounding of the cash (above all in nodes that receive
// very many additions, like the auxiliary node of a PageRank chain) leaves
// a floor under ||C||_1 that the re-derivation trigger may never reach.
// True when ||C||_1 has not gone below its value of stall_moves moves ago;
// advances the window.
__device__ __forceinline__ bool cash_stalled(double l1, double& mark, long long& count, int stall_moves) {
    if (stall_moves <= 0) return false;
    if (++count < stall_moves) return false;
    const bool stalled = l1 >= mark;
    mark = l1;
    count = 0;
    return stalled;
}

// Decides, after the cash statistics of C_t are known, whether the solve
// stops (the stop test of Alg. 1: t >= 2 and ||C_t||_1 / |H_t 1| < tol) and sets the
// threshold for this move. Runs in one thread.
__device__ void control_after_stats(DevState* st, unsigned long long cond_handle,
                                    unsigned long long cond_refresh, int use_cond, int n) {
    const Control& c = st->ctl;
    st->skip_move = 0;
    if (c.solving) {
        unsigned long long now = globaltimer();
        if (st->iters == 0) st->t_start = now;
        st->iters++;
        double hs = st->hsum;
        bool degenerate = !(fabs(hs) > 1e-12 * st->habs) || st->habs == 0.0;
        bool converged = st->moves >= 1 && st->l1 / fabs(hs) < c.tol;
        int stop = -1;
        if (degenerate) {
            stop = ST_DEGENERATE;
        } else if (converged) {
            if (c.mixed && !st->fresh) {
                // The FP32 cash has drifted from H (P - I): re-derive it and
                // test again before declaring convergence.
                st->want_refresh = 1;
                st->skip_move = 1;
            } else {
                stop = ST_OK;
            }
        } else if (st->solve_moves >= c.max_steps) {
            stop = ST_NOCONV;
        } else if ((double)(now - st->t_start) > c.time_limit_ns || st->iters > c.max_iters) {
            stop = ST_TIMEOUT;
        }
        if (stop >= 0) {
            st->done = 1;
            st->status = stop;
            if (use_cond) {
                cudaGraphSetConditional(cond_handle, 0u);
                if (c.mixed) cudaGraphSetConditional(cond_refresh, 0u);
            }
            return;
        }
        if (c.mixed && ((c.refresh_factor > 0.0 && st->l1 < c.refresh_factor * st->l1_refresh) ||
                        cash_stalled(st->l1, st->stall_mark, st->stall_count, c.stall_moves)))
            st->want_refresh = 1;  // applied at the start of the next iteration
        // the refresh of the next iteration runs only when requested
        if (use_cond && c.mixed) cudaGraphSetConditional(cond_refresh, st->want_refresh ? 1u : 0u);
    }
    // Threshold of this move.
    int sched = c.sched;
    if (c.safety_every > 0 && ((st->solve_moves + 1) % c.safety_every) == 0) sched = SCHED_ALL_GREEN;
    st->mode = MODE_NONE;
    if (sched == SCHED_THRESHOLD || sched == SCHED_LINK) {
        if (c.theta_arg > 0.0) {
            set_theta(st, c.theta_arg, sched);
        } else {
            double mean = st->sumr / (double)n;
            set_theta(st, (c.r == 1) ? c.theta_scale * mean : c.theta_scale * pow(mean, 1.0 / c.r),
                      sched);
        }
    } else if (sched == SCHED_TOPFRAC) {
        double f = (c.theta_arg > 0.0 && c.theta_arg <= 1.0) ? c.theta_arg : c.top_frac;
        long long k = (long long)ceil(f * (double)n);
        if (k < 1) k = 1;
        if (k > n) k = n;
        st->tk_remain = k;
        st->tk_prefix = 0ull;
        set_theta(st, 0.0, sched);
    } else {
        set_theta(st, 0.0, sched);
    }
}

// Chain of the nodes [it0, it0 + kNodesPerIter) when one chain holds them
// all (chain ids grow with node ids), else -1.
__device__ __forceinline__ int iter_chain(const BatchView& bv, long long it0, int n) {
    long long last = it0 + kNodesPerIter - 1;
    if (last >= n) last = n - 1;
    int a = bv.chain_of[it0], b = bv.chain_of[last];
    return a == b ? a : -1;
}

// Adds the block's values to chain ch's accumulators (all threads call it;
// ch is the same in every thread).
template <int K, typename V>
__device__ __forceinline__ void block_chain_add(ChainState* cs, int ch, const int* ks, const V* v,
                                                V* scratch) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        V t = block_sum(v[k], scratch);
        if (threadIdx.x == 0 && t != V(0)) atomicAdd(&cs[ch].acc[ks[k]], (double)t);
    }
}

__device__ __forceinline__ int status_rank(int st) {
    return st == ST_OK ? 0 : st == ST_NOCONV ? 1 : st == ST_DEGENERATE ? 2 : 3;
}
__device__ __forceinline__ int rank_status(int r) {
    return r == 0 ? ST_OK : r == 1 ? ST_NOCONV : r == 2 ? ST_DEGENERATE : ST_TIMEOUT;
}

// The batch form of control_after_stats, run by every thread of the last
// block: each chain takes its statistics from its accumulators, is tested
// for its own stop (the stop test of Alg. 1 with its own tolerance) and gets its own
// threshold; the loop ends when no chain is left running.
__device__ void batch_control(DevState* st, const BatchView& bv, unsigned long long cond_handle,
                              unsigned long long cond_refresh, int use_cond) {
    __shared__ int s_active, s_need, s_worst, s_timeout;
    __shared__ double scratch[32];
    const Control& c = st->ctl;
    if (threadIdx.x == 0) {
        s_active = 0;
        s_need = 0;
        s_worst = 0;
        st->skip_move = 0;
        int to = 0;
        if (c.solving) {
            unsigned long long now = globaltimer();
            if (st->iters == 0) st->t_start = now;
            st->iters++;
            to = ((double)(now - st->t_start) > c.time_limit_ns || st->iters > c.max_iters) ? 1 : 0;
        }
        s_timeout = to;
    }
    __syncthreads();
    int sched = c.sched;
    if (c.safety_every > 0 && ((st->solve_moves + 1) % c.safety_every) == 0) sched = SCHED_ALL_GREEN;
    const bool link = c.sched == SCHED_LINK;
    const int r = c.r;
    double l1sum = 0.0, ssum = 0.0;
    for (int k = threadIdx.x; k < bv.nchains; k += blockDim.x) {
        ChainState* ch = bv.cs + k;
        const double a = __ldcg(&ch->acc[0]), sm = __ldcg(&ch->acc[1]), sr = __ldcg(&ch->acc[2]);
        ch->acc[0] = 0.0;
        ch->acc[1] = 0.0;
        ch->acc[2] = 0.0;
        ch->l1 = a;
        ch->sum = sm;
        ch->sumr = (r == 1 && !link) ? a : sr;
        l1sum += a;
        ssum += sm;
        if (ch->done) continue;
        if (c.solving) {
            const double hs = ch->hsum;
            const bool degenerate = !(fabs(hs) > 1e-12 * ch->habs) || ch->habs == 0.0;
            const bool converged = ch->moves >= 1 && a / fabs(hs) < ch->tol;
            int stop = -1;
            if (degenerate) stop = ST_DEGENERATE;
            else if (converged) {
                if (c.mixed && !st->fresh) atomicOr(&s_need, 1);
                else stop = ST_OK;
            } else if (st->solve_moves >= c.max_steps) stop = ST_NOCONV;
            else if (s_timeout) stop = ST_TIMEOUT;
            if (stop >= 0) {
                ch->done = 1;
                ch->status = stop;
                atomicMax(&s_worst, status_rank(stop));
                continue;
            }
        }
        double th = 0.0;
        if (sched == SCHED_THRESHOLD || sched == SCHED_LINK) {
            const double mean = ch->sumr / (double)ch->n;
            th = c.theta_arg > 0.0 ? c.theta_arg
                                   : (r == 1 ? c.theta_scale * mean : c.theta_scale * pow(mean, 1.0 / r));
        }
        ch->theta = th;
        ch->theta_f = (sched == SCHED_LINK) ? __double2float_rn(th) : __double2float_ru(th);
        atomicAdd(&s_active, 1);
    }
    l1sum = block_sum(l1sum, scratch);
    ssum = block_sum(ssum, scratch);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->l1 = l1sum;
        st->sum = ssum;
        st->sumr = 0.0;
        st->theta = 0.0;
        st->mode = MODE_NONE;
        if (c.solving) {
            if (s_active == 0) {
                st->done = 1;
                st->status = rank_status(s_worst);
                if (use_cond) {
                    cudaGraphSetConditional(cond_handle, 0u);
                    if (c.mixed) cudaGraphSetConditional(cond_refresh, 0u);
                }
                return;
            }
            if (s_need) {
                st->want_refresh = 1;
                st->skip_move = 1;
            } else if (c.mixed && c.refresh_factor > 0.0 && st->l1 < c.refresh_factor * st->l1_refresh) {
                st->want_refresh = 1;
            }
            if (use_cond && c.mixed) cudaGraphSetConditional(cond_refresh, st->want_refresh ? 1u : 0u);
        }
    }
}

// Batch statistics: per chain ||C||_1, sum C, sum v^r, accumulated per
// block-iteration (one atomic per statistic when the iteration lies inside
// one chain), then batch_control.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bstats(const T* __restrict__ c,
                                                     const T* __restrict__ ideg, int n,
                                                     DevState* st, BatchView bv,
                                                     unsigned long long cond_handle,
                                                     unsigned long long cond_refresh, int use_cond) {
    if (st->done) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond_handle, 0u);
        return;
    }
    __shared__ T tscratch[32];
    const int r = st->ctl.r;
    const bool link = st->ctl.sched == SCHED_LINK;
    const int ks[3] = {0, 1, 2};
    for (long long it0 = (long long)blockIdx.x * kNodesPerIter; it0 < n;
         it0 += (long long)gridDim.x * kNodesPerIter) {
        const int uni = iter_chain(bv, it0, n);
        T a = T(0), sm = T(0), pr = T(0);
#pragma unroll
        for (int q = 0; q < kNodesPerThread; ++q) {
            const long long i = it0 + q * kThreads + threadIdx.x;
            if (i >= n) continue;
            const T v = c[i];
            const T av = fabs(v);
            const T tv = link ? av * ideg[i] : av;
            const T pv = (link && r == 1) ? tv : (r == 2 ? tv * tv : (r > 2 ? pow(tv, (T)r) : T(0)));
            if (uni >= 0) {
                a += av;
                sm += v;
                pr += pv;
            } else {
                const int ch = bv.chain_of[i];
                atomicAdd(&bv.cs[ch].acc[0], (double)av);
                atomicAdd(&bv.cs[ch].acc[1], (double)v);
                if (pv != T(0)) atomicAdd(&bv.cs[ch].acc[2], (double)pv);
            }
        }
        if (uni >= 0) {
            const T vals[3] = {a, sm, pr};
            block_chain_add<3>(bv.cs, uni, ks, vals, tscratch);
        }
    }
    if (!last_block(&st->ticket)) return;
    batch_control(st, bv, cond_handle, cond_refresh, use_cond);
}

// Per-thread sums over the nodes first, first + stride, ... of ||C||_1,
// sum C and sum v^r (v = |C_i|, or |C_i| / d_i for the per-link test), in
// the cash type (FP32 on the MIXED path: GB300's FP64 rate is low).
template <typename T, bool kCg>
__device__ __forceinline__ void stats_slice(const T* __restrict__ c, const T* __restrict__ ideg,
                                            long long n, bool link, int r, int vec_ok,
                                            long long first, long long stride, T& a, T& s, T& pr) {
    auto add = [&](T v, T idg) {
        const T av = fabs(v);
        a += av;
        s += v;
        const T tv = link ? av * idg : av;
        if (link && r == 1) pr += tv;
        else if (r == 2) pr += tv * tv;
        else if (r > 2) pr += pow(tv, (T)r);
    };
    // 16-byte vector loads (4 FP32 / 2 FP64 values), two vectors in flight
    // per thread, then the scalar tail.
    using V = typename std::conditional<std::is_same<T, float>::value, float4, double2>::type;
    constexpr int kW = sizeof(V) / sizeof(T);
    const long long nv = vec_ok ? n / kW : 0;
    const V* cv = reinterpret_cast<const V*>(c);
    const V* iv = reinterpret_cast<const V*>(ideg);
    long long k = first;
    for (; k + stride < nv; k += 2 * stride) {
        const V x0 = ld_shared_data<kCg>(cv + k), x1 = ld_shared_data<kCg>(cv + k + stride);
        V d0, d1;
        if (link) { d0 = iv[k]; d1 = iv[k + stride]; } else { d0 = x0; d1 = x1; }
        const T* p0 = reinterpret_cast<const T*>(&x0);
        const T* p1 = reinterpret_cast<const T*>(&x1);
        const T* q0 = reinterpret_cast<const T*>(&d0);
        const T* q1 = reinterpret_cast<const T*>(&d1);
#pragma unroll
        for (int u = 0; u < kW; ++u) add(p0[u], q0[u]);
#pragma unroll
        for (int u = 0; u < kW; ++u) add(p1[u], q1[u]);
    }
    for (; k < nv; k += stride) {
        const V x0 = ld_shared_data<kCg>(cv + k);
        V d0 = link ? iv[k] : x0;
        const T* p0 = reinterpret_cast<const T*>(&x0);
        const T* q0 = reinterpret_cast<const T*>(&d0);
#pragma unroll
        for (int u = 0; u < kW; ++u) add(p0[u], q0[u]);
    }
    for (long long i = nv * kW + first; i < n; i += stride)
        add(ld_shared_data<kCg>(c + i), link ? ideg[i] : T(0));
}

// ||C||_1, sum C and sum v^r (v = |C_i|, or |C_i| / d_i for the per-link
// test) of the current cash, then control. Each thread sums its nodes in the
// cash type (FP32 on the MIXED path: GB300's FP64 rate is low) and the
// per-thread sums are combined in FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_stats(const T* __restrict__ c,
                                                    const T* __restrict__ ideg, int n,
                                                    DevState* st, double* part,
                                                    unsigned long long cond_handle,
                                                    unsigned long long cond_refresh, int use_cond,
                                                    int vec_ok) {
    if (st->done) {
        // Never leave the device loop running once the solve is over.
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond_handle, 0u);
        return;
    }
    T a = T(0), s = T(0), pr = T(0);
    const int r = st->ctl.r;
    const bool link = st->ctl.sched == SCHED_LINK;
    stats_slice<T, false>(c, ideg, n, link, r, vec_ok, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                          (long long)gridDim.x * blockDim.x, a, s, pr);
    // block sums in the cash type too; the partials of the blocks are
    // combined in FP64
    __shared__ T tscratch[32];
    const T ba = block_sum(a, tscratch);
    const T bs = block_sum(s, tscratch);
    const T bp = block_sum(pr, tscratch);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = (double)ba;
        part[3 * blockIdx.x + 1] = (double)bs;
        part[3 * blockIdx.x + 2] = (double)bp;
    }
    if (!last_block(&st->ticket)) return;
    double tot[3];
    reduce_partials<3>(part, gridDim.x, tot);
    __shared__ StStage stage;
    DevState* ss = st_stage_in(st, &stage);
    if (threadIdx.x == 0) {
        ss->l1 = tot[0];
        ss->sum = tot[1];
        ss->sumr = (r == 1 && !link) ? tot[0] : tot[2];
        control_after_stats(ss, cond_handle, cond_refresh, use_cond, n);
    }
    st_stage_out(st, &stage);
}

// ------------------------------------------------------ top-k radix select

// One radix pass of the exact k-th largest |C| (keys = IEEE bit patterns of
// |C|, whose unsigned order is the order of the values). pass_shift is the
// bit position of this digit; the digits above it are fixed in tk_prefix.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_radix_pass(const T* __restrict__ c, int n,
                                                         DevState* st, int shift, int width) {
    if (st->done || st->skip_move) return;
    if (st->ctl.sched != SCHED_TOPFRAC) return;
    if (st->ctl.safety_every > 0 && ((st->solve_moves + 1) % st->ctl.safety_every) == 0) return;
    __shared__ unsigned int h[kRadixBins];
    const int nbins = 1 << width;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const int hi_shift = shift + width;
    const unsigned long long prefix = st->tk_prefix;
    const unsigned long long mask = (unsigned long long)(nbins - 1);
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // Whole warps iterate together so equal digits can be merged with
    // __match_any_sync (one shared-memory atomic per distinct digit per warp).
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const long long i = base + lane;
        int digit = -1;
        if (i < n) {
            unsigned long long k = (unsigned long long)KeyOf<T>::key(c[i]);
            bool match = (hi_shift >= KeyOf<T>::bits) || ((k >> hi_shift) == (prefix >> hi_shift));
            if (match) digit = (int)((k >> shift) & mask);
        }
        unsigned int peers = __match_any_sync(0xffffffffu, digit);
        if (digit >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[digit], (unsigned)__popc(peers));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (h[b]) atomicAdd(&st->hist[b], h[b]);
    if (!last_block(&st->ticket)) return;
    // Bucket of the remaining k-th largest key: thread t owns 8 bins counted
    // from the top; a block scan gives the count above its bins.
    __shared__ int found;
    __shared__ long long above_found;
    if (threadIdx.x == 0) found = -1;
    const int per = kRadixBins / kThreads;  // 8
    const int top = nbins - 1 - threadIdx.x * per;
    unsigned long long mine = 0;
    unsigned int hb[kRadixBins / kThreads];
#pragma unroll
    for (int q = 0; q < per; ++q) {
        int b = top - q;
        hb[q] = (b >= 0) ? __ldcg(&st->hist[b]) : 0u;
        mine += hb[q];
    }
    unsigned long long total;
    unsigned long long above = block_exscan(mine, &total);
    const long long remain = st->tk_remain;
    if ((long long)above < remain && (long long)(above + mine) >= remain) {
        long long cum = (long long)above;
#pragma unroll
        for (int q = 0; q < per; ++q) {
            int b = top - q;
            if (b >= 0 && cum + (long long)hb[q] >= remain) {
                found = b;
                above_found = cum;
                break;
            }
            cum += hb[q];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int digit = found >= 0 ? found : 0;
        long long cum = found >= 0 ? above_found : 0;
        st->tk_prefix = prefix | ((unsigned long long)digit << shift);
        st->tk_remain = remain - cum;
        if (shift == 0) set_theta(st, KeyOf<T>::value(st->tk_prefix), SCHED_TOPFRAC);
    }
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) st->hist[b] = 0u;
}

// ------------------------------------------------------------------ select

// m~_i = m_i s_i, the cash a green row sends per unit of edge weight: in
// FP64 on the FP64 path, in FP32 (with s_i rounded to FP32) on the MIXED path.
__device__ __forceinline__ double moved_per_weight(double v, const double* s, const float*, long long i) {
    return v * s[i];
}
__device__ __forceinline__ float moved_per_weight(float v, const double*, const float* sf, long long i) {
    return v * sf[i];
}

// Green-light selection, snapshot and frontier compaction (Eq. recursion_M
// and Eq. recursion_H): for every green node, m_i = C_i, C_i <- 0,
// H_i += m_i, and the frontier entry (edge offset, CSR base, m~_i = m_i s_i)
// is written. Dense mt[i] = m~_i (0 for red nodes) feeds the pull.
template <typename T, bool kBatch>
__global__ void __launch_bounds__(kThreads) k_select(
    T* __restrict__ c, double* __restrict__ H, const double* __restrict__ s,
    const float* __restrict__ sf, const long long* __restrict__ row_ptr,
    const T* __restrict__ ideg, const unsigned char* __restrict__ masks, int n,
    T* __restrict__ mt, long long* __restrict__ f_eoff, long long* __restrict__ f_base,
    T* __restrict__ f_m, int* __restrict__ chunk_row, DevState* st, double* part,
    MoveRecord* __restrict__ log, unsigned long long cond_mode, int use_cond, BatchView bv) {
    if (st->done || st->skip_move) return;
    const Control& ctl = st->ctl;
    int sched = ctl.sched;
    if (ctl.safety_every > 0 && ((st->solve_moves + 1) % ctl.safety_every) == 0) sched = SCHED_ALL_GREEN;
    // The MIXED path compares in FP32 against theta_f (see set_theta); the
    // FP64 path compares in FP64.
    const T theta = std::is_same<T, float>::value ? (T)st->theta_f : (T)st->theta;
    const unsigned char* mask = nullptr;
    if (sched == SCHED_MASK) mask = masks + (size_t)(st->mask_cursor % ctl.n_masks) * (size_t)n;
    const SchedAux ax = sched_aux(ctl, n, st->moves, st->l1, sched);

    __shared__ double scratch[32];
    __shared__ T tscratch[32];
    __shared__ unsigned long long base_sh;
    T msum = T(0), mabs = T(0);  // per-thread sums in the cash type

    // Batch: all-green goes through the frontier path, since nodes of chains
    // that have stopped are red.
    const bool dense_all = (sched == SCHED_ALL_GREEN) && !kBatch;
    for (long long it0 = (long long)blockIdx.x * kNodesPerIter; it0 < n;
         it0 += (long long)gridDim.x * kNodesPerIter) {
        int idx[kNodesPerThread];
        T val[kNodesPerThread], scv[kNodesPerThread];
        long long rb[kNodesPerThread];
        int rdeg[kNodesPerThread];
        bool g[kNodesPerThread];
        unsigned long long mine = 0ull;
        int uni = -1;
        if (kBatch) {
            uni = iter_chain(bv, it0, n);
            msum = T(0);
            mabs = T(0);
        }
        // Row offsets are read for every node (not only green ones) so that
        // these loads overlap the cash loads instead of waiting for the test.
        if (!dense_all) {
#pragma unroll
            for (int q = 0; q < kNodesPerThread; ++q) {
                const long long i = it0 + q * kThreads + threadIdx.x;
                rb[q] = (i < n) ? row_ptr[i] : 0;
                rdeg[q] = (i < n) ? (int)(row_ptr[i + 1] - rb[q]) : 0;
            }
        }
#pragma unroll
        for (int q = 0; q < kNodesPerThread; ++q) {
            long long i = it0 + q * kThreads + threadIdx.x;
            idx[q] = (int)i;
            g[q] = false;
            val[q] = T(0);
            // s_i now: red_add below orders every later load after it
            scv[q] = (i < n) ? moved_per_weight(T(1), s, sf, i) : T(0);
            if (i < n) {
                T v = c[i];
                val[q] = v;
                T th = theta;
                bool active = true;
                if (kBatch) {
                    const ChainState& ch = bv.cs[uni >= 0 ? uni : bv.chain_of[i]];
                    active = !ch.done;
                    th = std::is_same<T, float>::value ? (T)ch.theta_f : (T)ch.theta;
                }
                g[q] = active && green_test<T>(sched, v, i, th, mask, ideg, ax);
            }
            if (g[q] && !dense_all) mine += ((unsigned long long)rdeg[q] << kCountBits) + 1ull;
        }
        if (dense_all) {
            // All-green always pulls: no frontier, no degrees.
#pragma unroll
            for (int q = 0; q < kNodesPerThread; ++q) {
                long long i = idx[q];
                if (i >= n) continue;
                const T v = val[q];
                c[i] = T(0);
                red_add(H + i, (double)v);  // no load: the L2 adds
                msum += v;
                mabs += fabs(v);
                mt[i] = v * scv[q];
            }
            continue;
        }
        unsigned long long total;
        unsigned long long pre = block_exscan(mine, &total);
        if (threadIdx.x == 0) base_sh = total ? atomicAdd(&st->reserve, total) : 0ull;
        __syncthreads();
        unsigned long long base = base_sh + pre;
        long long k = (long long)(base & ((1ull << kCountBits) - 1ull));
        long long e = (long long)(base >> kCountBits);
#pragma unroll
        for (int q = 0; q < kNodesPerThread; ++q) {
            long long i = idx[q];
            if (i >= n) continue;
            if (g[q]) {
                const T v = val[q];
                const T mtil = v * scv[q];
                c[i] = T(0);
                red_add(H + i, (double)v);  // no load: the L2 adds
                if (kBatch && uni < 0) {
                    const int ch = bv.chain_of[i];
                    atomicAdd(&bv.cs[ch].acc[3], (double)v);
                    atomicAdd(&bv.cs[ch].acc[4], (double)fabs(v));
                } else {
                    msum += v;
                    mabs += fabs(v);
                }
                mt[i] = mtil;
                f_eoff[k] = e;
                f_base[k] = rb[q] - e;
                f_m[k] = mtil;
                // chunk b starts inside this row when e <= b*CH < e + deg
                long long b0 = (e + kPushChunk - 1) / kPushChunk;
                long long b1 = (e + rdeg[q] + kPushChunk - 1) / kPushChunk;
                for (long long b = b0; b < b1; ++b) chunk_row[b] = (int)k;
                ++k;
                e += rdeg[q];
            } else {
                mt[i] = T(0);
            }
        }
        if (kBatch && uni >= 0) {
            const int ks[2] = {3, 4};
            const T vals[2] = {msum, mabs};
            block_chain_add<2>(bv.cs, uni, ks, vals, tscratch);
        }
        __syncthreads();
    }
    if (kBatch) {
        msum = T(0);
        mabs = T(0);
    }
    const double bmsum = (double)block_sum(msum, tscratch);
    const double bmabs = (double)block_sum(mabs, tscratch);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = bmsum;
        part[2 * blockIdx.x + 1] = bmabs;
    }
    if (!last_block(&st->ticket)) return;
    double tot[2];
    reduce_partials<2>(part, gridDim.x, tot);
    double bsum = 0.0, babs = 0.0;
    if (kBatch) {
        // per chain: history totals and the move count of running chains
        for (int k = threadIdx.x; k < bv.nchains; k += blockDim.x) {
            ChainState* ch = bv.cs + k;
            const double m = __ldcg(&ch->acc[3]), ma = __ldcg(&ch->acc[4]);
            ch->acc[3] = 0.0;
            ch->acc[4] = 0.0;
            ch->hsum += m;
            ch->habs += ma;
            bsum += m;
            babs += ma;
            if (!ch->done) {
                ch->moves++;
                ch->fresh = 0;
            }
        }
        bsum = block_sum(bsum, scratch);
        babs = block_sum(babs, scratch);
    }
    __shared__ StStage stage;
    DevState* ss = st_stage_in(st, &stage);
    if (threadIdx.x == 0) {
        const double ms = kBatch ? bsum : tot[0], ma = kBatch ? babs : tot[1];
        unsigned long long rsv = ss->reserve;
        long long green = (long long)(rsv & ((1ull << kCountBits) - 1ull));
        long long edges = (long long)(rsv >> kCountBits);
        if (dense_all) {  // every node, every edge (no frontier built)
            green = n;
            edges = ss->ctl.nnz;
        }
        ss->reserve = 0ull;
        ss->green = green;
        ss->edges = edges;
        ss->hsum += ms;
        ss->habs += ma;
        ss->last_mabs = ma;
        ss->moves++;
        ss->solve_moves++;
        ss->tot_green += green;
        ss->tot_edges += edges;
        ss->fresh = 0;
        if (sched == SCHED_MASK) ss->mask_cursor++;
        int mode;
        if (green == 0) mode = MODE_NONE;
        else if (sched == SCHED_ALL_GREEN || (double)edges >= ss->ctl.pull_crossover * (double)ss->ctl.nnz)
            mode = MODE_PULL;
        else
            mode = MODE_PUSH;
        ss->mode = mode;
        if (mode == MODE_PUSH) ss->push_moves++;
        if (mode == MODE_PULL) ss->pull_moves++;
        // in the solve graph, only the chosen one of pull / push is launched
        if (use_cond) cudaGraphSetConditional(cond_mode, mode == MODE_PULL ? 1u : 0u);
        MoveRecord rec;
        rec.move = ss->moves - 1;
        rec.green = green;
        rec.edges = edges;
        rec.mode = mode;
        rec.pad = 0;
        rec.theta = theta;
        rec.l1 = ss->l1;
        rec.hsum = ss->hsum;
        for (int k = 0; k < 6; ++k) rec.phase_us[k] = 0.f;
        log[rec.move % kLogCap] = rec;
    }
    st_stage_out(st, &stage);
}

// -------------------------------------------------------------------- push

// c_j += m~_i w_ij for every out-edge of every frontier row (Eq.
// grl_update_C). Work is split into chunks of kPushChunk consecutive
// frontier edges, whatever the row degrees; chunk_row[b] is the frontier row
// holding the chunk's first edge (written by k_select). Within a chunk each
// edge slot is labelled with its row by marking the row starts and taking a
// block-wide running maximum, so every edge costs one shared-memory read;
// edges are then handled in a coalesced order (slot = thread + q * threads).

// Hub targets of the push: up to kHubSlots nodes of the largest in-degree,
// each in the slot hub_slot(id) of a direct-mapped table (-1: empty). The
// push sums the additions a block makes to each hub in shared memory and
// adds them to the cash once per block and move: one address takes its
// additions one after another, so a hub's thousands of in-links a move
// would otherwise queue on one L2 line.
constexpr int kHubSlots = 64;
__host__ __device__ __forceinline__ int hub_slot(int j) { return (int)(((unsigned int)j * 0x9E3779B1u) >> 26); }

// Shared memory of the push chunk loop.
template <typename T, int kBT = kThreads>
struct PushSmem {
    int row[kPushChunk];
    long long base[kPushChunk + 1];
    T m[kPushChunk + 1];
    int wmax[kBT / 32];
    int hub[kHubSlots];
    double hot[kHubSlots];
};

// The chunks of a push over E frontier edges of K frontier rows (see
// k_push): b = first, first + step, ..., or, when `next` is given, chunks
// handed out one at a time by that counter (thread 0 asks for the next one
// while the block works on the current one), so that blocks that meet slow
// atomics take fewer chunks.
// Targets in the hub table `hubs` (kHubSlots ids, -1 empty; nullptr: none),
// like the auxiliary node of a PageRank chain, which every node feeds, are
// summed per block in FP64 in shared memory and added to the cash once per
// block: one global addition per block instead of one per in-link, all of
// which would queue on one L2 address.
template <typename T, bool kHasW, bool kCg, int kBT = kThreads>
__device__ __forceinline__ void push_chunks(T* __restrict__ c, const int* __restrict__ col,
                                            const float* __restrict__ w,
                                            const long long* __restrict__ f_eoff,
                                            const long long* __restrict__ f_base,
                                            const T* __restrict__ f_m,
                                            const int* __restrict__ chunk_row, long long E,
                                            long long K, long long first, long long step,
                                            PushSmem<T, kBT>& sm, const int* __restrict__ hubs,
                                            unsigned long long* next = nullptr) {
    constexpr int kPer = kPushChunk / kBT;  // edge slots per thread
    const long long nchunks = (E + kPushChunk - 1) / kPushChunk;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ long long s_next;
    long long b = first;
    if (hubs) {
        for (int t = threadIdx.x; t < kHubSlots; t += kBT) {
            sm.hub[t] = __ldg(hubs + t);
            sm.hot[t] = 0.0;
        }
        __syncthreads();
    }
    if (next) {
        if (threadIdx.x == 0) s_next = (long long)atomicAdd(next, 1ull);
        __syncthreads();
        b = s_next;
        __syncthreads();
    }
    while (b < nchunks) {
        if (next && threadIdx.x == 0) s_next = (long long)atomicAdd(next, 1ull);  // read below
        const long long e0 = b * kPushChunk;
        const int ne = (int)min((long long)kPushChunk, E - e0);
        const long long k0 = ld_shared_data<kCg>(chunk_row + b);
        const long long k1 = (b + 1 < nchunks) ? (long long)ld_shared_data<kCg>(chunk_row + b + 1) : K - 1;
        const int nr = (int)(k1 - k0 + 1);
#pragma unroll
        for (int q = 0; q < kPer; ++q) sm.row[threadIdx.x * kPer + q] = 0;
        __syncthreads();
        for (int r = threadIdx.x; r < nr; r += blockDim.x) {
            const long long eo = ld_shared_data<kCg>(f_eoff + k0 + r);
            sm.base[r] = ld_shared_data<kCg>(f_base + k0 + r);
            sm.m[r] = ld_shared_data<kCg>(f_m + k0 + r);
            const long long off = eo - e0;  // row 0 starts at or before the chunk
            if (r > 0 && off < ne) sm.row[(int)off] = r;
        }
        __syncthreads();
        // running maximum over the slots: slot -> row
        int v[kPer];
        int run = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            run = max(run, sm.row[threadIdx.x * kPer + q]);
            v[q] = run;
        }
        int incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl = max(incl, y);
        }
        if (lane == 31) sm.wmax[wid] = incl;
        __syncthreads();
        int before = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) before = 0;
        for (int k = 0; k < wid; ++k) before = max(before, sm.wmax[k]);
#pragma unroll
        for (int q = 0; q < kPer; ++q) sm.row[threadIdx.x * kPer + q] = max(v[q], before);
        __syncthreads();
        // every slot's target and amount first, then the additions: red_add
        // is ordered with the thread's other memory accesses, so a load
        // placed after one would wait for it, one round trip per slot
        int slot_j[kPer];
        T slot_v[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int le = threadIdx.x + q * kBT;
            slot_j[q] = -1;
            slot_v[q] = T(0);
            if (le < ne) {
                const int r = sm.row[le];
                const long long pos = sm.base[r] + e0 + le;
                slot_j[q] = __ldg(col + pos);
                T val = sm.m[r];
                if (kHasW) val = val * (T)__ldg(w + pos);
                slot_v[q] = val;
            }
        }
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int j = slot_j[q];
            if (j < 0) continue;
            const int hs = hub_slot(j);
            if (hubs && sm.hub[hs] == j) {
                slot_j[q] = hs;  // summed below
            } else {
                red_add(c + j, slot_v[q]);
                slot_j[q] = -1;
            }
        }
        if (hubs) {
            // hub targets: one shared-memory addition per warp and hub
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const bool hot = slot_j[q] >= 0;
                unsigned int m = __ballot_sync(0xffffffffu, hot);
                while (m) {
                    const int t = __shfl_sync(0xffffffffu, slot_j[q], __ffs(m) - 1);
                    const bool mine = hot && slot_j[q] == t;
                    double v = warp_sum(mine ? (double)slot_v[q] : 0.0);
                    if (lane == 0) atomicAdd(&sm.hot[t], v);
                    m &= ~__ballot_sync(0xffffffffu, mine);
                }
            }
        }
        __syncthreads();
        if (next) {
            b = s_next;
            __syncthreads();  // everyone has read s_next before thread 0 rewrites it
        } else {
            b += step;
        }
    }
    if (hubs) {
        __syncthreads();
        for (int t = threadIdx.x; t < kHubSlots; t += kBT)
            if (sm.hot[t] != 0.0) red_add(c + sm.hub[t], (T)sm.hot[t]);
    }
}

template <typename T, bool kHasW>
__global__ void __launch_bounds__(kThreads) k_push(
    T* __restrict__ c, const int* __restrict__ col, const float* __restrict__ w,
    const long long* __restrict__ f_eoff, const long long* __restrict__ f_base,
    const T* __restrict__ f_m, const int* __restrict__ chunk_row, const DevState* st, const int* hubs) {
    if (st->done || st->skip_move || st->mode != MODE_PUSH) return;
    __shared__ PushSmem<T> sm;
    push_chunks<T, kHasW, false>(c, col, w, f_eoff, f_base, f_m, chunk_row, st->edges, st->green,
                                 blockIdx.x, gridDim.x, sm, hubs);
}

// ------------------------------------------------------ merge-path pull

// Segmented inclusive scan over the threads of a block: the running sum of
// val restarts wherever key changes. Keys with a value >= 0 must form
// contiguous runs (equal keys are never separated by a different key).
// Returns this thread's scan value; s_key/s_val then hold every thread's
// key and scan value.
template <typename TV, int kBT = kThreads>
__device__ __forceinline__ TV block_segscan(long long key, TV val, long long* s_key, TV* s_val) {
    constexpr int kW = kBT / 32;
    constexpr unsigned kWMask = kW >= 32 ? 0xffffffffu : ((1u << kW) - 1u);
    __shared__ long long w_key[kW];
    __shared__ TV w_val[kW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    TV x = val;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        TV y = __shfl_up_sync(0xffffffffu, x, o);
        long long ky = __shfl_up_sync(0xffffffffu, key, o);
        if (lane >= o && ky == key) x += y;
    }
    if (lane == 31) {
        w_key[wid] = key;
        w_val[wid] = x;
    }
    __syncthreads();
    if (wid == 0 && lane < kW) {
        // the same scan over the warp tails
        long long k = w_key[lane];
        TV v = w_val[lane];
#pragma unroll
        for (int o = 1; o < kW; o <<= 1) {
            TV y = __shfl_up_sync(kWMask, v, o);
            long long ky = __shfl_up_sync(kWMask, k, o);
            if (lane >= o && ky == k) v += y;
        }
        w_val[lane] = v;
    }
    __syncthreads();
    if (wid > 0 && w_key[wid - 1] == key) x += w_val[wid - 1];
    s_key[threadIdx.x] = key;
    s_val[threadIdx.x] = x;
    __syncthreads();
    return x;
}

// Sums over in-links (the CSC of P): out_j += sum_{e in in(j)} src[t_src[e]]
// * t_w[e], balanced over rows + edges by merge-path tiles (Merrill and
// Garland, SC'16). Each tile's edge values are gathered into shared memory
// with coalesced loads of t_src/t_w (all of a thread's loads issued before
// any is used), then every thread consumes kMpIpt merge items. Rows that a
// thread ends are written once; the pieces of a row split between threads
// are joined by a segmented scan over the block, so only rows that cross a
// tile boundary use atomic adds.

// Shared memory of the merge-path tile loop.
// Merge-path items per thread for a block of kBT threads: a tile is
// kBT * mp_ipt(kBT) items (2048 for 256 threads).
__host__ __device__ constexpr int mp_ipt(int kBT) { return kBT >= 512 ? 4 : kMpIpt; }

template <typename TV, int kBT = kThreads>
struct PullSmem {
    TV val[kBT * mp_ipt(kBT)];
    int end[kBT * mp_ipt(kBT) + 1];
    int start0;
    long long ckey[kBT];
    TV cval[kBT];
};

// The tiles b = first, first + step, ... of a merge-path pull (see k_pull),
// or, when `next` is given, tiles handed out one at a time by that counter
// (thread 0 asks for the next one while the block works on the current one),
// so that blocks end within about one tile of one another.
// A row's sum goes into out with one reduction (red.global.add, nothing
// comes back): a load-then-store per row end would put one dependent L2
// round trip per row end on the thread, serialised over the rows a warp's
// threads end at different steps of the merge.
template <typename TV, typename TO, bool kHasW, bool kCg, int kBT = kThreads>
__device__ __forceinline__ void pull_tiles(TO* __restrict__ out, const TV* __restrict__ src,
                                           const long long* __restrict__ t_ptr,
                                           const int* __restrict__ t_src,
                                           const float* __restrict__ t_w,
                                           const long long* __restrict__ tile_r,
                                           const long long* __restrict__ tile_e, long long ntiles,
                                           long long first, long long step, PullSmem<TV, kBT>& sm,
                                           unsigned long long* next = nullptr) {
    constexpr int kIpt = mp_ipt(kBT);  // merge items per thread: a tile is kBT * kIpt items
    __shared__ long long s_tnext;
    long long b = first;
    if (next) {
        if (threadIdx.x == 0) s_tnext = (long long)atomicAdd(next, 1ull);
        __syncthreads();
        b = s_tnext;
        __syncthreads();
    }
    while (b < ntiles) {
        if (next && threadIdx.x == 0) s_tnext = (long long)atomicAdd(next, 1ull);  // read below
        const long long r0 = tile_r[b], e0 = tile_e[b];
        const int nrows = (int)(tile_r[b + 1] - r0);
        const int nedges = (int)(tile_e[b + 1] - e0);
        {
            int sidx[kIpt];
            float wv[kIpt];
            long long re[kIpt];
#pragma unroll
            for (int q = 0; q < kIpt; ++q) {
                const int k = threadIdx.x + q * kBT;
                sidx[q] = (k < nedges) ? __ldg(t_src + e0 + k) : -1;
                if (kHasW) wv[q] = (k < nedges) ? __ldg(t_w + e0 + k) : 0.0f;
                re[q] = (k < nrows) ? __ldg(t_ptr + r0 + 1 + k) : 0;
            }
            TV v[kIpt];
#pragma unroll
            for (int q = 0; q < kIpt; ++q) v[q] = (sidx[q] >= 0) ? ld_shared_data<kCg>(src + sidx[q]) : TV(0);
#pragma unroll
            for (int q = 0; q < kIpt; ++q) {
                const int k = threadIdx.x + q * kBT;
                if (k < nedges) sm.val[k] = kHasW ? v[q] * (TV)wv[q] : v[q];
                if (k < nrows) sm.end[k] = (int)(re[q] - e0);
            }
        }
        if (threadIdx.x == 0) {
            sm.end[nrows] = 0x7fffffff;
            sm.start0 = (int)(t_ptr[r0] - e0);
        }
        __syncthreads();
        const int total = nrows + nedges;
        int d = threadIdx.x * kIpt;
        const bool active = d < total;
        // head piece: the end of a row begun by earlier threads (rowA);
        // tail piece: a row that continues past this thread (carry).
        long long rowA = -1, rowB = -1;
        TV accA = TV(0), accB = TV(0);
        if (active) {
            const int dend = min(d + kIpt, total);
            int lo = max(0, d - nedges), hi = min(d, nrows);
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (sm.end[mid] >= d - mid) hi = mid; else lo = mid + 1;
            }
            int i = lo, j = d - lo;
            const int row_start = (i == 0) ? sm.start0 : sm.end[i - 1];
            bool whole = (j == row_start);  // no edge of row i before this thread
            TV acc = TV(0);
            int cnt = 0;
            for (; d < dend; ++d) {
                if (j < sm.end[i]) {
                    acc += sm.val[j];
                    ++j;
                    ++cnt;
                } else {
                    if (!whole) {
                        rowA = r0 + i;
                        accA = acc;
                    } else if (cnt > 0) {
                        red_add(out + (r0 + i), (TO)acc);
                    }
                    acc = TV(0);
                    cnt = 0;
                    ++i;
                    whole = true;
                }
            }
            if (cnt > 0 || !whole) {
                // the row continues past this thread (or began before it and
                // has not ended here)
                rowB = r0 + i;
                accB = acc;
            }
        }
        // Join the pieces: carry of thread t plus the carries of the threads
        // before it on the same row.
        const TV run = block_segscan<TV, kBT>(rowB, accB, sm.ckey, sm.cval);
        if (rowA >= 0) {
            TV sum = accA;
            if (threadIdx.x > 0 && sm.ckey[threadIdx.x - 1] == rowA) sum += sm.cval[threadIdx.x - 1];
            red_add(out + rowA, (TO)sum);
        }
        // last active thread: its carry leaves the tile
        const int last = (total - 1) / kIpt;
        if ((int)threadIdx.x == last && rowB >= 0) red_add(out + rowB, (TO)run);
        __syncthreads();
        if (next) {
            b = s_tnext;
            __syncthreads();  // everyone has read s_tnext before thread 0 rewrites it
        } else {
            b += step;
        }
    }
}

// kind 0: cash pull (guarded by mode == PULL); kind 1: FP64 residual pull
// into y (guarded by want_refresh / force_refresh). The library launches
// kind 0 only: the residual pull runs over warp tiles (k_rederive_pull).
template <typename TV, typename TO, bool kHasW, int kKind>
__global__ void __launch_bounds__(kThreads) k_pull(
    TO* __restrict__ out, const TV* __restrict__ src, const long long* __restrict__ t_ptr,
    const int* __restrict__ t_src, const float* __restrict__ t_w,
    const long long* __restrict__ tile_r, const long long* __restrict__ tile_e, long long ntiles,
    const DevState* st) {
    if (kKind == 0) {
        if (st->done || st->skip_move || st->mode != MODE_PULL) return;
    } else {
        if (!(st->force_refresh || (st->want_refresh && !st->done))) return;
    }
    __shared__ PullSmem<TV> sm;
    pull_tiles<TV, TO, kHasW, false>(out, src, t_ptr, t_src, t_w, tile_r, tile_e, ntiles, blockIdx.x,
                                     gridDim.x, sm);
}

// ------------------------------------------------------------ refresh

// hsrc_i = H_i s_i (FP64), the source vector of the residual pull.
__global__ void k_refresh_src(const double* __restrict__ H, const double* __restrict__ s, int n,
                              double* __restrict__ hsrc, const DevState* st) {
    if (!(st->force_refresh || (st->want_refresh && !st->done))) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        hsrc[i] = H[i] * s[i];
}

// exact_j = C0_j + (H P)_j - H_j (Eq. recursion_H_res); residual
// sum |C_j - exact_j|; when applying, C_j <- exact_j. Leaves y = 0.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_refresh_apply(
    T* __restrict__ c, const double* __restrict__ H, double* __restrict__ y,
    const double* __restrict__ c0, int n, DevState* st, double* part) {
    if (!(st->force_refresh || (st->want_refresh && !st->done))) return;
    const bool apply = st->apply_refresh || !st->force_refresh;
    __shared__ double scratch[32];
    double rs = 0.0, l1 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double ex = y[i] - H[i];
        if (c0) ex += c0[i];
        double cur = (double)c[i];
        rs += fabs(cur - ex);
        y[i] = 0.0;
        if (apply) {
            T nv = (T)ex;
            c[i] = nv;
            l1 += fabs((double)nv);
        }
    }
    rs = block_sum(rs, scratch);
    l1 = block_sum(l1, scratch);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = rs;
        part[2 * blockIdx.x + 1] = l1;
    }
    if (!last_block(&st->ticket)) return;
    double tot[2];
    reduce_partials<2>(part, gridDim.x, tot);
    if (threadIdx.x == 0) {
        const double R = tot[0], L = tot[1];
        st->resid_l1 = R;
        if (apply) {
            st->fresh = 1;
            st->l1_refresh = L;
            st->refreshes++;
            st->stall_mark = kNoMark;
            st->stall_count = 0;
        }
        st->want_refresh = 0;
        st->force_refresh = 0;
        st->apply_refresh = 0;
    }
}

// ----------------------------------------------------- setup / estimate

// sum H and sum |H| (FP64, deterministic order of partials).
__global__ void __launch_bounds__(kThreads) k_hist_sums(const double* __restrict__ H, int n,
                                                        DevState* st, double* part, int set_state) {
    __shared__ double scratch[32];
    double s = 0.0, a = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = H[i];
        s += v;
        a += fabs(v);
    }
    s = block_sum(s, scratch);
    a = block_sum(a, scratch);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s;
        part[2 * blockIdx.x + 1] = a;
    }
    if (!last_block(&st->ticket)) return;
    double tot[2];
    reduce_partials<2>(part, gridDim.x, tot);
    if (threadIdx.x == 0) {
        const double S = tot[0], A = tot[1];
        if (set_state) { st->hsum = S; st->habs = A; }
        part[2 * kMaxGrid] = S;
        part[2 * kMaxGrid + 1] = A;
    }
}

// Step 0 from the uniform M_0 (Eq. init): H = M_0 = 1/N (1/N_k within chain
// k of a batch) and C_1 = M_0 (P - I), i.e. C_j = (colsum_j - 1) / N, in FP64
// and then rounded to the cash type; ||C_1||_1 of the stored cash goes to
// l1_refresh (the cash is exact: a fresh state), and sum H and sum |H| to
// the state, so that no separate pass over H follows.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_step0_uniform(T* __restrict__ c, double* __restrict__ H,
                                                            const double* __restrict__ colsum, int n,
                                                            const int* __restrict__ chain_of,
                                                            const long long* __restrict__ node_ptr,
                                                            DevState* st, double* part) {
    __shared__ double scratch[32];
    double a = 0.0, hs = 0.0, ha = 0.0;
    const double inv_n = 1.0 / (double)n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double inv = inv_n;
        if (chain_of) {
            const int k = chain_of[i];
            inv = 1.0 / (double)(node_ptr[k + 1] - node_ptr[k]);
        }
        H[i] = inv;
        const T v = (T)(colsum[i] * inv - inv);
        c[i] = v;
        a += fabs((double)v);
        hs += inv;
        ha += fabs(inv);
    }
    a = block_sum(a, scratch);
    hs = block_sum(hs, scratch);
    ha = block_sum(ha, scratch);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = a;
        part[3 * blockIdx.x + 1] = hs;
        part[3 * blockIdx.x + 2] = ha;
    }
    if (!last_block(&st->ticket)) return;
    double tot[3];
    reduce_partials<3>(part, gridDim.x, tot);
    if (threadIdx.x == 0) {
        // sum H and sum |H| as k_hist_sums would find them (the same grid,
        // loop and reduction order per sum)
        st->hsum = tot[1];
        st->habs = tot[2];
        part[2 * kMaxGrid] = tot[1];
        part[2 * kMaxGrid + 1] = tot[2];
        st->l1_refresh = tot[0];
        st->resid_l1 = 0.0;
        st->fresh = 1;
        st->stall_mark = kNoMark;
        st->stall_count = 0;
    }
}

// Batch: per chain sum H and sum |H| into acc[5], acc[6] (zero at rest).
__global__ void __launch_bounds__(kThreads) k_bhist_sums(const double* __restrict__ H, int n,
                                                         BatchView bv) {
    __shared__ double scratch[32];
    const int ks[2] = {5, 6};
    for (long long it0 = (long long)blockIdx.x * kNodesPerIter; it0 < n;
         it0 += (long long)gridDim.x * kNodesPerIter) {
        const int uni = iter_chain(bv, it0, n);
        double hs = 0.0, ha = 0.0;
#pragma unroll
        for (int q = 0; q < kNodesPerThread; ++q) {
            const long long i = it0 + q * kThreads + threadIdx.x;
            if (i >= n) continue;
            const double v = H[i];
            if (uni >= 0) {
                hs += v;
                ha += fabs(v);
            } else {
                const int ch = bv.chain_of[i];
                atomicAdd(&bv.cs[ch].acc[5], v);
                atomicAdd(&bv.cs[ch].acc[6], fabs(v));
            }
        }
        if (uni >= 0) {
            const double vals[2] = {hs, ha};
            block_chain_add<2, double>(bv.cs, uni, ks, vals, scratch);
        }
    }
}

// Batch: moves the per-chain sums from the accumulators into hsum / habs
// (set_state) and leaves them, one chain per thread.
__global__ void k_bhist_finish(BatchView bv, int set_state, double* sums_out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < bv.nchains; k += gridDim.x * blockDim.x) {
        ChainState* ch = bv.cs + k;
        const double S = ch->acc[5], A = ch->acc[6];
        ch->acc[5] = 0.0;
        ch->acc[6] = 0.0;
        if (set_state) {
            ch->hsum = S;
            ch->habs = A;
        }
        if (sums_out) {
            sums_out[2 * k] = S;
            sums_out[2 * k + 1] = A;
        }
    }
}

// Batch estimate: pi_i = H_i / (sum of H over i's chain).
__global__ void k_bscale(const double* __restrict__ H, int n, const int* __restrict__ chain_of,
                         const double* __restrict__ sums, double* __restrict__ pi) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        pi[i] = H[i] / sums[2 * chain_of[i]];
}

// Node -> chain map from the chain offsets (binary search per node).
__global__ void k_chain_of(const long long* __restrict__ node_ptr, int nchains, long long n,
                           int* __restrict__ chain_of) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = nchains - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (node_ptr[mid] <= i) lo = mid; else hi = mid - 1;
        }
        chain_of[i] = lo;
    }
}

// Every edge must stay inside its chain (block-diagonal CSR); err |= 16.
__global__ void k_check_blocks(const long long* __restrict__ row_ptr, const int* __restrict__ col,
                               const int* __restrict__ chain_of, long long n, unsigned int* err) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned int e = 0;
    for (long long i = warp; i < n; i += nwarps) {
        const int ci = chain_of[i];
        for (long long k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 32)
            if (chain_of[col[k]] != ci) e = 16u;
    }
    if (e) atomicOr(err, e);
}

__global__ void k_scale(const double* __restrict__ H, int n, const double* __restrict__ sums,
                        double* __restrict__ pi) {
    double S = sums[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        pi[i] = H[i] / S;
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ x, int n, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (double)x[i];
}

template <typename T>
__global__ void k_from_double(const double* __restrict__ x, int n, T* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (T)x[i];
}

// Checks a CSR: row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz, every row
// non-empty, 0 <= col < n, weights positive and finite. err bits: 1 bad
// row_ptr, 2 empty row, 4 col out of range, 8 bad weight.
__global__ void k_validate(const long long* __restrict__ row_ptr, const int* __restrict__ col,
                           const float* __restrict__ w, long long n, long long nnz,
                           unsigned int* err) {
    unsigned int e = 0;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        long long a = row_ptr[i], b = row_ptr[i + 1];
        if (b < a || a < 0 || b > nnz) e |= 1u;
        else if (b == a) e |= 2u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (row_ptr[0] != 0 || row_ptr[n] != nnz)) e |= 1u;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += stride) {
        int j = col[k];
        if (j < 0 || j >= n) e |= 4u;
        if (w) {
            float x = w[k];
            if (!(x > 0.0f) || !isfinite(x)) e |= 8u;
        }
    }
    if (e) atomicOr(err, e);
}

// s_i = 1 / sum_k w_ik (FP64 sum in CSR order) or 1 / deg_i.
// Rows with more weights than this have their weight sum taken by a whole
// block (k_row_scale_long): one thread summing a million weights in a row
// (the auxiliary node of a PageRank chain) took tens of milliseconds.
constexpr long long kLongRowW = 65536;

__global__ void k_row_scale(const long long* __restrict__ row_ptr, const float* __restrict__ w,
                            long long n, double* __restrict__ s, float* __restrict__ sf,
                            float* __restrict__ idegf, double* __restrict__ idegd,
                            int* __restrict__ long_rows, unsigned int* __restrict__ n_long) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        long long a = row_ptr[i], b = row_ptr[i + 1];
        const double id = 1.0 / (double)(b - a);
        if (idegf) idegf[i] = (float)id;
        if (idegd) idegd[i] = id;
        double sum;
        if (w) {
            if (b - a > kLongRowW) {
                long_rows[atomicAdd(n_long, 1u)] = (int)i;  // summed by k_row_scale_long
                continue;
            }
            sum = 0.0;
            for (long long k = a; k < b; ++k) sum += (double)w[k];
        } else {
            sum = (double)(b - a);
        }
        s[i] = 1.0 / sum;
        if (sf) sf[i] = (float)(1.0 / sum);
    }
}

// s_i = 1 / sum_k w_ik for the long rows k_row_scale listed: block b sums
// row long_rows[b] (FP64, a fixed order for a given block size).
__global__ void __launch_bounds__(kThreads) k_row_scale_long(
    const long long* __restrict__ row_ptr, const float* __restrict__ w, double* __restrict__ s,
    float* __restrict__ sf, const int* __restrict__ long_rows, const unsigned int* __restrict__ n_long) {
    __shared__ double scratch[32];
    if (blockIdx.x >= *n_long) return;
    const long long i = long_rows[blockIdx.x];
    const long long a = row_ptr[i], b = row_ptr[i + 1];
    double acc = 0.0;
    for (long long k = a + threadIdx.x; k < b; k += blockDim.x) acc += (double)w[k];
    const double sum = block_sum(acc, scratch);
    if (threadIdx.x == 0) {
        s[i] = 1.0 / sum;
        if (sf) sf[i] = (float)(1.0 / sum);
    }
}

// In-degree counts into cnt[j + 1].
__global__ void k_count_in(const int* __restrict__ col, long long nnz, long long* cnt) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz;
         k += (long long)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long*)(cnt + col[k] + 1), 1ull);
}

// Row of the first edge of every kPushChunk-edge chunk of the CSR (binary
// search; every row has at least one edge), and out[nchunks] = n - 1.
__global__ void k_chunk_rows(const long long* __restrict__ row_ptr, long long n, long long nnz,
                             int* __restrict__ out) {
    const long long nch = (nnz + kPushChunk - 1) / kPushChunk;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b <= nch;
         b += (long long)gridDim.x * blockDim.x) {
        if (b == nch) {
            out[b] = (int)(n - 1);
            continue;
        }
        const long long e = b * kPushChunk;
        long long lo = 0, hi = n - 1;  // largest i with row_ptr[i] <= e
        while (lo < hi) {
            const long long mid = (lo + hi + 1) >> 1;
            if (row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
        }
        out[b] = (int)lo;
    }
}

// Scatter of the CSR into the CSC with per-column cursors, edge-balanced:
// chunks of kPushChunk consecutive edges whatever the row lengths (a row
// with 10^5 edges spreads over many blocks), each edge labelled with its row
// by marking the row starts in the chunk and a block-wide running maximum
// (as in the push). Order within a CSC row is arbitrary.
__global__ void __launch_bounds__(kThreads) k_csc_scatter(
    const long long* __restrict__ row_ptr, const int* __restrict__ col, const float* __restrict__ w,
    long long nnz, const int* __restrict__ chunk_first_row, long long* cursor, int* __restrict__ t_src,
    float* __restrict__ t_w) {
    constexpr int kPer = kPushChunk / kThreads;
    __shared__ int s_row[kPushChunk];
    __shared__ int s_wmax[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long nch = (nnz + kPushChunk - 1) / kPushChunk;
    for (long long b = blockIdx.x; b < nch; b += gridDim.x) {
        const long long e0 = b * kPushChunk;
        const int ne = (int)min((long long)kPushChunk, nnz - e0);
        const int k0 = chunk_first_row[b];
        const int k1 = (b + 1 < nch) ? chunk_first_row[b + 1] : chunk_first_row[nch];
#pragma unroll
        for (int q = 0; q < kPer; ++q) s_row[threadIdx.x * kPer + q] = 0;
        __syncthreads();
        // rows k0+1..k1 start inside this chunk (offsets relative to k0)
        for (long long r = k0 + 1 + threadIdx.x; r <= k1; r += blockDim.x) {
            const long long off = row_ptr[r] - e0;
            if (off < ne) s_row[(int)off] = (int)(r - k0);
        }
        __syncthreads();
        int v[kPer];
        int run = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            run = max(run, s_row[threadIdx.x * kPer + q]);
            v[q] = run;
        }
        int incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl = max(incl, y);
        }
        if (lane == 31) s_wmax[wid] = incl;
        __syncthreads();
        int before = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) before = 0;
        for (int k = 0; k < wid; ++k) before = max(before, s_wmax[k]);
#pragma unroll
        for (int q = 0; q < kPer; ++q) s_row[threadIdx.x * kPer + q] = max(v[q], before);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int le = threadIdx.x + q * kThreads;
            if (le < ne) {
                const long long e = e0 + le;
                const int j = col[e];
                const long long pos = (long long)atomicAdd((unsigned long long*)(cursor + j), 1ull);
                t_src[pos] = k0 + s_row[le];
                if (w) t_w[pos] = w[e];
            }
        }
        __syncthreads();
    }
}

// colsum_j = sum over in-links (i, j) of s_i w_ij = (1 P)_j in FP64, over the
// CSC with merge-path tiles (balanced whatever the in-degrees); colsum must be
// zero on entry. Computed once per chain: step 0 from the uniform M_0 then
// needs no pass over the edges.
template <bool kHasW>
__global__ void __launch_bounds__(kThreads) k_colsum_tiles(double* __restrict__ colsum,
                                                           const double* __restrict__ s,
                                                           const long long* __restrict__ t_ptr,
                                                           const int* __restrict__ t_src,
                                                           const float* __restrict__ t_w,
                                                           const long long* __restrict__ tile_r,
                                                           const long long* __restrict__ tile_e,
                                                           long long ntiles) {
    __shared__ PullSmem<double> sm;
    pull_tiles<double, double, kHasW, false>(colsum, s, t_ptr, t_src, t_w, tile_r, tile_e, ntiles,
                                             blockIdx.x, gridDim.x, sm);
}

// Hub candidates: nodes whose in-degree is at least thr, appended to
// ids/deg (at most cap; *cnt counts every candidate).
__global__ void k_hub_candidates(const long long* __restrict__ t_ptr, long long n, long long thr, int cap,
                                 int* __restrict__ ids, long long* __restrict__ deg, unsigned int* cnt) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const long long d = t_ptr[j + 1] - t_ptr[j];
        if (d >= thr) {
            const unsigned int k = atomicAdd(cnt, 1u);
            if ((int)k < cap) {
                ids[k] = (int)j;
                deg[k] = d;
            }
        }
    }
}

// Histogram of floor(log2(in-degree)) over the nodes (64 bins).
__global__ void k_indeg_log2_hist(const long long* __restrict__ t_ptr, long long n, unsigned int* hist) {
    __shared__ unsigned int h[64];
    for (int b = threadIdx.x; b < 64; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const long long d = t_ptr[j + 1] - t_ptr[j];
        if (d > 0) atomicAdd(&h[63 - __clzll(d)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 64; b += blockDim.x)
        if (h[b]) atomicAdd(hist + b, h[b]);
}

// Batch: every chain running again (and its tolerance, when tol >= 0).
__global__ void k_bbegin(ChainState* cs, int nchains, double tol, int reset_moves) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nchains; k += gridDim.x * blockDim.x) {
        cs[k].done = 0;
        cs[k].status = 0;
        if (tol >= 0.0) cs[k].tol = tol;
        if (reset_moves) {
            // step 0: exact cash, ||C||_1 taken at the first statistics
            cs[k].moves = 0;
            cs[k].fresh = 1;
            cs[k].l1r = 0.0;
        }
    }
}

// Flags of an out-of-loop refresh (step 0, rlgl_refresh, residual).
__global__ void k_set_refresh_flags(DevState* st, int force, int apply) {
    st->force_refresh = force;
    st->apply_refresh = apply;
}

// Resume from a given state: y holds (H P) from a residual pull; records
// C_0 = c - (H P - H) (Eq. recursion_H_res) in place of the given c (held in
// c0 on entry), sets the cash to c, and leaves y = 0.
template <typename T>
__global__ void k_record_c0(double* __restrict__ c0, const double* __restrict__ H,
                            double* __restrict__ y, T* __restrict__ c, int n, DevState* st) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double cg = c0[i];
        c[i] = (T)cg;
        c0[i] = cg - (y[i] - H[i]);
        y[i] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->force_refresh = 0;
        st->apply_refresh = 0;
    }
}

// Inclusive scan, pass 1: per-block scan of kNodesPerIter elements and the
// block totals.
__global__ void __launch_bounds__(kThreads) k_scan_blocks(long long* x, long long m,
                                                          long long* block_tot) {
    long long base = (long long)blockIdx.x * kNodesPerIter + (long long)threadIdx.x * kNodesPerThread;
    unsigned long long v[kNodesPerThread];
    unsigned long long mine = 0;
#pragma unroll
    for (int q = 0; q < kNodesPerThread; ++q) {
        v[q] = (base + q < m) ? (unsigned long long)x[base + q] : 0ull;
        mine += v[q];
    }
    unsigned long long total;
    unsigned long long pre = block_exscan(mine, &total);
#pragma unroll
    for (int q = 0; q < kNodesPerThread; ++q) {
        pre += v[q];
        if (base + q < m) x[base + q] = (long long)pre;
    }
    if (threadIdx.x == 0) block_tot[blockIdx.x] = (long long)total;
}

// Pass 2: one block scans the block totals in place (exclusive).
__global__ void __launch_bounds__(kThreads) k_scan_tot(long long* tot, long long nb) {
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b0 = 0; b0 < nb; b0 += kThreads) {
        long long b = b0 + threadIdx.x;
        unsigned long long v = (b < nb) ? (unsigned long long)tot[b] : 0ull;
        unsigned long long total;
        unsigned long long pre = block_exscan(v, &total);
        if (b < nb) tot[b] = (long long)(carry + pre);
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

// Pass 3: add the block offsets.
__global__ void k_scan_add(long long* x, long long m, const long long* tot) {
    long long base = (long long)blockIdx.x * kNodesPerIter;
    long long off = tot[blockIdx.x];
    for (int q = threadIdx.x; q < kNodesPerIter; q += blockDim.x)
        if (base + q < m) x[base + q] += off;
}

// Merge-path split of each tile boundary: for diagonal d = b * items, the
// number of rows ended before it (smallest i with t_ptr[i+1] >= d - i).
__global__ void k_mp_partition(const long long* __restrict__ t_ptr, long long n, long long nnz,
                               long long ntiles, int items, long long* tile_r, long long* tile_e) {
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b <= ntiles;
         b += (long long)gridDim.x * blockDim.x) {
        long long d = min(b * (long long)items, n + nnz);
        long long lo = max(0ll, d - nnz), hi = min(d, n);
        while (lo < hi) {
            long long mid = (lo + hi) >> 1;
            if (t_ptr[mid + 1] >= d - mid) hi = mid; else lo = mid + 1;
        }
        tile_r[b] = lo;
        tile_e[b] = d - lo;
    }
}

}  // namespace rlgl
