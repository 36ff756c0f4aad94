// Device kernels of the RLGL green-light sweep (sm_103a).
//
// One move of Alg. 1 (Eqs. recursion_M, recursion_H, recursion_C) runs as
//   stats   : ||C||_1, sum C, sum |C|^r in FP64 (stopping rule, Alg. 1 line
//             (7); threshold theta_t(r), Sec. 6) + solve control;
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
#include <cstdint>
#include <cuda_runtime.h>

namespace rlgl {

constexpr int kThreads = 256;         // threads per block, every kernel
constexpr int kNodesPerThread = 4;    // node kernels: nodes per thread per block-iteration
constexpr int kNodesPerIter = kThreads * kNodesPerThread;
constexpr int kPushChunk = 2048;      // edges per push chunk
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
};

enum Mode : int { MODE_NONE = 0, MODE_PUSH = 1, MODE_PULL = 2 };
enum Sched : int {
    SCHED_ALL_GREEN = 0,
    SCHED_THRESHOLD = 1,
    SCHED_TOPFRAC = 2,
    SCHED_MASK = 3,
    SCHED_LINK = 4
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
    int sched;
    int r;
    int safety_every;
    int solving;             // 1: solve (stop tests active), 0: single step
    int mixed;               // MIXED precision path
    int n_masks;
    int pad[2];
};

struct DevState {
    Control ctl;
    // statistics of the current cash (written by the stats kernel)
    double l1, sum, sumr, theta;
    double hsum, habs;       // H 1 (kept incrementally) and an upper bound of sum |H|
    double l1_refresh;       // ||C||_1 right after the last re-derivation
    double resid_l1;         // residual measured by the last refresh pass
    double last_mabs;
    // last move and totals
    long long green, edges;
    long long moves;         // moves since step 0 (t - 1)
    long long solve_moves, iters, mask_cursor;
    long long tot_green, tot_edges, push_moves, pull_moves, refreshes;
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

// Block-wide exclusive scan of 64-bit values (blockDim = kThreads). Returns
// the exclusive prefix; *total receives the block total (all threads).
__device__ __forceinline__ unsigned long long block_exscan(unsigned long long v,
                                                           unsigned long long* total) {
    __shared__ unsigned long long wsum[kThreads / 32];
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
        unsigned long long s = (lane < kThreads / 32) ? wsum[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) wsum[lane] = s;  // inclusive warp prefixes
    }
    __syncthreads();
    unsigned long long before = (wid > 0) ? wsum[wid - 1] : 0ull;
    *total = wsum[kThreads / 32 - 1];
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

// In the last block: out[k] = sum over blocks b of part[K b + k], with all
// threads of the block, in a fixed order (per-thread strided sums, then a
// fixed tree), so the result does not depend on block scheduling. The
// result is valid in thread 0.
template <int K>
__device__ __forceinline__ void reduce_partials(const double* part, int nb, double* out) {
    __shared__ double scratch[32];
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += ldcg(part + K * b + k);
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = block_sum(acc[k], scratch);
}

// ------------------------------------------------------- stats + control

// Decides, after the cash statistics of C_t are known, whether the solve
// stops (Alg. 1 line (7): t >= 2 and ||C_t||_1 / |H_t 1| < tol) and sets the
// threshold for this move. Runs in one thread.
__device__ void control_after_stats(DevState* st, unsigned long long cond_handle, int use_cond,
                                    int n) {
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
            if (use_cond) cudaGraphSetConditional(cond_handle, 0u);
            return;
        }
        if (c.mixed && c.refresh_factor > 0.0 && st->l1 < c.refresh_factor * st->l1_refresh)
            st->want_refresh = 1;  // applied at the start of the next iteration
    }
    // Threshold of this move.
    int sched = c.sched;
    if (c.safety_every > 0 && ((st->solve_moves + 1) % c.safety_every) == 0) sched = SCHED_ALL_GREEN;
    st->mode = MODE_NONE;
    if (sched == SCHED_THRESHOLD || sched == SCHED_LINK) {
        if (c.theta_arg > 0.0) {
            st->theta = c.theta_arg;
        } else {
            double mean = st->sumr / (double)n;
            st->theta = (c.r == 1) ? c.theta_scale * mean : c.theta_scale * pow(mean, 1.0 / c.r);
        }
    } else if (sched == SCHED_TOPFRAC) {
        double f = (c.theta_arg > 0.0 && c.theta_arg <= 1.0) ? c.theta_arg : c.top_frac;
        long long k = (long long)ceil(f * (double)n);
        if (k < 1) k = 1;
        if (k > n) k = n;
        st->tk_remain = k;
        st->tk_prefix = 0ull;
        st->theta = 0.0;
    } else {
        st->theta = 0.0;
    }
}

// ||C||_1, sum C, sum |C|^r (FP64) of the current cash, then control.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_stats(const T* __restrict__ c,
                                                    const int* __restrict__ deg, int n,
                                                    DevState* st, double* part,
                                                    unsigned long long cond_handle, int use_cond) {
    if (st->done) {
        // Never leave the device loop running once the solve is over.
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond_handle, 0u);
        return;
    }
    __shared__ double scratch[32];
    double a = 0.0, s = 0.0, pr = 0.0;
    const int r = st->ctl.r;
    const bool link = st->ctl.sched == SCHED_LINK;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = (double)c[i];
        double av = fabs(v);
        a += av;
        s += v;
        // threshold statistic: |C_i| (THRESHOLD) or |C_i| / d_i (LINK)
        double tv = link ? av / (double)deg[i] : av;
        if (link && r == 1) pr += tv;
        else if (r == 2) pr += tv * tv;
        else if (r > 2) pr += pow(tv, (double)r);
    }
    a = block_sum(a, scratch);
    s = block_sum(s, scratch);
    pr = block_sum(pr, scratch);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = a;
        part[3 * blockIdx.x + 1] = s;
        part[3 * blockIdx.x + 2] = pr;
    }
    if (!last_block(&st->ticket)) return;
    double tot[3];
    reduce_partials<3>(part, gridDim.x, tot);
    if (threadIdx.x == 0) {
        st->l1 = tot[0];
        st->sum = tot[1];
        st->sumr = (r == 1 && !link) ? tot[0] : tot[2];
        control_after_stats(st, cond_handle, use_cond, n);
    }
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
        if (shift == 0) st->theta = KeyOf<T>::value(st->tk_prefix);
    }
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) st->hist[b] = 0u;
}

// ------------------------------------------------------------------ select

// Green-light selection, snapshot and frontier compaction (Eq. recursion_M
// and Eq. recursion_H): for every green node, m_i = C_i, C_i <- 0,
// H_i += m_i, and the frontier entry (edge offset, CSR base, m~_i = m_i s_i)
// is written. Dense mt[i] = m~_i (0 for red nodes) feeds the pull.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_select(
    T* __restrict__ c, double* __restrict__ H, const double* __restrict__ s,
    const long long* __restrict__ row_ptr, const int* __restrict__ deg,
    const unsigned char* __restrict__ masks, int n,
    T* __restrict__ mt, long long* __restrict__ f_eoff, long long* __restrict__ f_base,
    T* __restrict__ f_m, int* __restrict__ chunk_row, DevState* st, double* part,
    MoveRecord* __restrict__ log) {
    if (st->done || st->skip_move) return;
    const Control& ctl = st->ctl;
    int sched = ctl.sched;
    if (ctl.safety_every > 0 && ((st->solve_moves + 1) % ctl.safety_every) == 0) sched = SCHED_ALL_GREEN;
    const double theta = st->theta;
    const unsigned char* mask = nullptr;
    if (sched == SCHED_MASK) mask = masks + (size_t)(st->mask_cursor % ctl.n_masks) * (size_t)n;

    __shared__ double scratch[32];
    __shared__ unsigned long long base_sh;
    double msum = 0.0, mabs = 0.0;

    for (long long it0 = (long long)blockIdx.x * kNodesPerIter; it0 < n;
         it0 += (long long)gridDim.x * kNodesPerIter) {
        int idx[kNodesPerThread];
        T val[kNodesPerThread];
        long long rdeg[kNodesPerThread], rb[kNodesPerThread];
        bool g[kNodesPerThread];
        unsigned long long mine = 0ull;
#pragma unroll
        for (int q = 0; q < kNodesPerThread; ++q) {
            long long i = it0 + q * kThreads + threadIdx.x;
            idx[q] = (int)i;
            g[q] = false;
            val[q] = T(0);
            if (i < n) {
                T v = c[i];
                val[q] = v;
                if (sched == SCHED_ALL_GREEN) g[q] = true;
                else if (sched == SCHED_MASK) g[q] = mask[i] != 0;
                else if (sched == SCHED_LINK) g[q] = (v != T(0)) && (fabs((double)v) / (double)deg[i] >= theta);
                else g[q] = (v != T(0)) && (fabs((double)v) >= theta);
            }
            if (g[q] && sched != SCHED_ALL_GREEN) {
                rb[q] = row_ptr[idx[q]];
                rdeg[q] = row_ptr[idx[q] + 1] - rb[q];
                mine += ((unsigned long long)rdeg[q] << kCountBits) + 1ull;
            }
        }
        if (sched == SCHED_ALL_GREEN) {
            // All-green always pulls: no frontier, no degrees.
#pragma unroll
            for (int q = 0; q < kNodesPerThread; ++q) {
                long long i = idx[q];
                if (i >= n) continue;
                double mv = (double)val[q];
                c[i] = T(0);
                H[i] += mv;
                msum += mv;
                mabs += fabs(mv);
                mt[i] = (T)(mv * s[i]);
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
                T v = val[q];
                double mv = (double)v;
                T mtil = (T)(mv * s[i]);
                c[i] = T(0);
                H[i] += mv;
                msum += mv;
                mabs += fabs(mv);
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
        __syncthreads();
    }
    msum = block_sum(msum, scratch);
    mabs = block_sum(mabs, scratch);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = msum;
        part[2 * blockIdx.x + 1] = mabs;
    }
    if (!last_block(&st->ticket)) return;
    double tot[2];
    reduce_partials<2>(part, gridDim.x, tot);
    if (threadIdx.x == 0) {
        const double ms = tot[0], ma = tot[1];
        unsigned long long rsv = *(volatile unsigned long long*)&st->reserve;
        long long green = (long long)(rsv & ((1ull << kCountBits) - 1ull));
        long long edges = (long long)(rsv >> kCountBits);
        if (sched == SCHED_ALL_GREEN) {  // every node, every edge (no frontier built)
            green = n;
            edges = ctl.nnz;
        }
        st->reserve = 0ull;
        st->green = green;
        st->edges = edges;
        st->hsum += ms;
        st->habs += ma;
        st->last_mabs = ma;
        st->moves++;
        st->solve_moves++;
        st->tot_green += green;
        st->tot_edges += edges;
        st->fresh = 0;
        if (sched == SCHED_MASK) st->mask_cursor++;
        int mode;
        if (green == 0) mode = MODE_NONE;
        else if (sched == SCHED_ALL_GREEN || (double)edges >= ctl.pull_crossover * (double)ctl.nnz)
            mode = MODE_PULL;
        else
            mode = MODE_PUSH;
        st->mode = mode;
        if (mode == MODE_PUSH) st->push_moves++;
        if (mode == MODE_PULL) st->pull_moves++;
        MoveRecord rec;
        rec.move = st->moves - 1;
        rec.green = green;
        rec.edges = edges;
        rec.mode = mode;
        rec.pad = 0;
        rec.theta = theta;
        rec.l1 = st->l1;
        rec.hsum = st->hsum;
        log[rec.move % kLogCap] = rec;
    }
}

// -------------------------------------------------------------------- push

// c_j += m~_i w_ij for every out-edge of every frontier row (Eq.
// grl_update_C). Work is split into chunks of kPushChunk consecutive
// frontier edges, whatever the row degrees; chunk_row[b] is the frontier row
// holding the chunk's first edge (written by k_select).
template <typename T, bool kHasW>
__global__ void __launch_bounds__(kThreads) k_push(
    T* __restrict__ c, const int* __restrict__ col, const float* __restrict__ w,
    const long long* __restrict__ f_eoff, const long long* __restrict__ f_base,
    const T* __restrict__ f_m, const int* __restrict__ chunk_row, const DevState* st) {
    if (st->done || st->skip_move || st->mode != MODE_PUSH) return;
    const long long E = st->edges;
    const long long K = st->green;
    const long long nchunks = (E + kPushChunk - 1) / kPushChunk;
    __shared__ int s_off[kPushChunk + 1];
    __shared__ long long s_base[kPushChunk + 1];
    __shared__ T s_m[kPushChunk + 1];
    for (long long b = blockIdx.x; b < nchunks; b += gridDim.x) {
        const long long e0 = b * kPushChunk;
        const int ne = (int)min((long long)kPushChunk, E - e0);
        const long long k0 = chunk_row[b];
        const long long k1 = (b + 1 < nchunks) ? (long long)chunk_row[b + 1] : K - 1;
        const int nr = (int)(k1 - k0 + 1);
        for (int r = threadIdx.x; r < nr; r += blockDim.x) {
            long long eo = f_eoff[k0 + r];
            s_off[r] = (int)(eo - e0);
            s_base[r] = f_base[k0 + r];
            s_m[r] = f_m[k0 + r];
        }
        __syncthreads();
        for (int le = threadIdx.x; le < ne; le += blockDim.x) {
            // last row whose local offset is <= le
            int lo = 0, hi = nr - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= le) lo = mid; else hi = mid - 1;
            }
            long long pos = s_base[lo] + e0 + le;
            int j = __ldg(col + pos);
            T v = s_m[lo];
            if (kHasW) v = v * (T)__ldg(w + pos);
            atomicAdd(c + j, v);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------ merge-path pull

// Segmented inclusive scan over the threads of a block: the running sum of
// val restarts wherever key changes. Keys with a value >= 0 must form
// contiguous runs (equal keys are never separated by a different key).
// Returns this thread's scan value; s_key/s_val then hold every thread's
// key and scan value.
template <typename TV>
__device__ __forceinline__ TV block_segscan(long long key, TV val, long long* s_key, TV* s_val) {
    __shared__ long long w_key[kThreads / 32];
    __shared__ TV w_val[kThreads / 32];
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
    if (wid == 0 && lane < kThreads / 32) {
        // the same scan over the warp tails
        long long k = w_key[lane];
        TV v = w_val[lane];
#pragma unroll
        for (int o = 1; o < kThreads / 32; o <<= 1) {
            TV y = __shfl_up_sync(0x000000ffu, v, o);
            long long ky = __shfl_up_sync(0x000000ffu, k, o);
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
// kind 0: cash pull (guarded by mode == PULL); kind 1: FP64 residual pull
// into y (guarded by want_refresh / force_refresh).
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
    __shared__ TV s_val[kMpItems];
    __shared__ int s_end[kMpItems + 1];
    __shared__ int s_start0;
    __shared__ long long s_ckey[kThreads];
    __shared__ TV s_cval[kThreads];
    for (long long b = blockIdx.x; b < ntiles; b += gridDim.x) {
        const long long r0 = tile_r[b], e0 = tile_e[b];
        const int nrows = (int)(tile_r[b + 1] - r0);
        const int nedges = (int)(tile_e[b + 1] - e0);
        {
            int sidx[kMpIpt];
            float wv[kMpIpt];
            long long re[kMpIpt];
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) {
                const int k = threadIdx.x + q * kThreads;
                sidx[q] = (k < nedges) ? __ldg(t_src + e0 + k) : -1;
                if (kHasW) wv[q] = (k < nedges) ? __ldg(t_w + e0 + k) : 0.0f;
                re[q] = (k < nrows) ? __ldg(t_ptr + r0 + 1 + k) : 0;
            }
            TV v[kMpIpt];
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) v[q] = (sidx[q] >= 0) ? src[sidx[q]] : TV(0);
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) {
                const int k = threadIdx.x + q * kThreads;
                if (k < nedges) s_val[k] = kHasW ? v[q] * (TV)wv[q] : v[q];
                if (k < nrows) s_end[k] = (int)(re[q] - e0);
            }
        }
        if (threadIdx.x == 0) {
            s_end[nrows] = 0x7fffffff;
            s_start0 = (int)(t_ptr[r0] - e0);
        }
        __syncthreads();
        const int total = nrows + nedges;
        int d = threadIdx.x * kMpIpt;
        const bool active = d < total;
        // head piece: the end of a row begun by earlier threads (rowA);
        // tail piece: a row that continues past this thread (carry).
        long long rowA = -1, rowB = -1;
        TV accA = TV(0), accB = TV(0);
        if (active) {
            const int dend = min(d + kMpIpt, total);
            int lo = max(0, d - nedges), hi = min(d, nrows);
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (s_end[mid] >= d - mid) hi = mid; else lo = mid + 1;
            }
            int i = lo, j = d - lo;
            const int row_start = (i == 0) ? s_start0 : s_end[i - 1];
            bool whole = (j == row_start);  // no edge of row i before this thread
            TV acc = TV(0);
            int cnt = 0;
            for (; d < dend; ++d) {
                if (j < s_end[i]) {
                    acc += s_val[j];
                    ++j;
                    ++cnt;
                } else {
                    if (!whole) {
                        rowA = r0 + i;
                        accA = acc;
                    } else if (cnt > 0) {
                        TO* o = out + (r0 + i);
                        *o = (TO)(*o + (TO)acc);
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
        const TV run = block_segscan<TV>(rowB, accB, s_ckey, s_cval);
        if (rowA >= 0) {
            TV sum = accA;
            if (threadIdx.x > 0 && s_ckey[threadIdx.x - 1] == rowA) sum += s_cval[threadIdx.x - 1];
            TO* o = out + rowA;
            // the tile's first row may have begun in the previous tile
            if (rowA == r0 && s_start0 < 0) atomicAdd(o, (TO)sum);
            else *o = (TO)(*o + (TO)sum);
        }
        // last active thread: its carry leaves the tile
        const int last = (total - 1) / kMpIpt;
        if ((int)threadIdx.x == last && rowB >= 0) atomicAdd(out + rowB, (TO)run);
        __syncthreads();
    }
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
__global__ void k_row_scale(const long long* __restrict__ row_ptr, const float* __restrict__ w,
                            long long n, double* __restrict__ s, int* __restrict__ deg) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        long long a = row_ptr[i], b = row_ptr[i + 1];
        double sum;
        if (w) {
            sum = 0.0;
            for (long long k = a; k < b; ++k) sum += (double)w[k];
        } else {
            sum = (double)(b - a);
        }
        s[i] = 1.0 / sum;
        deg[i] = (int)(b - a);
    }
}

// In-degree counts into cnt[j + 1].
__global__ void k_count_in(const int* __restrict__ col, long long nnz, long long* cnt) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz;
         k += (long long)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long*)(cnt + col[k] + 1), 1ull);
}

// Scatter of the CSR into the CSC with per-row cursors, one warp per row
// (order within a CSC row is arbitrary).
__global__ void k_scatter_in(const long long* __restrict__ row_ptr, const int* __restrict__ col,
                             const float* __restrict__ w, long long n, long long* cursor,
                             int* __restrict__ t_src, float* __restrict__ t_w) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < n; i += nwarps) {
        for (long long k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 32) {
            int j = col[k];
            long long q = (long long)atomicAdd((unsigned long long*)(cursor + j), 1ull);
            t_src[q] = (int)i;
            if (w) t_w[q] = w[k];
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

// Merge-path split of each tile boundary: for diagonal d = b * kMpItems,
// the number of rows ended before it (smallest i with t_ptr[i+1] >= d - i).
__global__ void k_mp_partition(const long long* __restrict__ t_ptr, long long n, long long nnz,
                               long long ntiles, long long* tile_r, long long* tile_e) {
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b <= ntiles;
         b += (long long)gridDim.x * blockDim.x) {
        long long d = min(b * (long long)kMpItems, n + nnz);
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
