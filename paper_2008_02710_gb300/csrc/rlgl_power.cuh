// The persistent all-green sweep (power iteration, Sec. 2.3.1): the moves
// of a single-chain all-green solve in one cooperative kernel, one pass over
// the in-links and two grid barriers a move.
//
// With G_t = [N] a move is M_t = C_t, H <- H + C_t, C_{t+1} = M_t P (Eqs.
// recursion_M, recursion_H, recursion_C; every node's cash leaves it). The
// general sweep makes it in three phases (statistics, select, pull) with
// three barriers. Here the select's work is folded into the pull's row
// epilogue: once the in-link sum of row j is complete, one thread reads
// C_t,j, adds it to H_j, stores C_{t+1},j = the sum and the next move's
// moved cash per weight m~_j = C_{t+1},j s_j, and sums the statistics of
// C_{t+1} and of M_t. A move is
//   pull    : merge-path tiles over the in-links, one warp per tile (the
//             warp's lanes meet only at __syncwarp, never at a block-wide
//             barrier), gathering m~ of the current move; the next tile's
//             bounds and in-link sources are loaded while the warp works on
//             the current one. A row that ends in the tile where it began
//             goes through the epilogue with the tile. A row whose in-links
//             cross tile boundaries adds one piece per tile it spans into a
//             zero-at-rest accumulator.
//   barrier
//   split   : each row that crossed a tile boundary (one per tile whose
//             first row ends in it but began in an earlier tile) takes its
//             sum from the accumulator and goes through the epilogue.
//   barrier ; every block takes the same decisions (stop test of Alg. 1,
//             re-derivation triggers) from the same totals.
// Measured on R-MAT 20 and symmetrised R-MAT 22 (all-green to a fixed move
// count; 8.60 ms and 91.9 ms with the pieces counted as they arrived and the
// row finished by its last piece, within the pull, one fence per piece):
// finishing the split rows after a barrier instead, 7.40 / 79.6 ms; loading
// the next tile's bounds and sources ahead, at three blocks an SM (the
// registers it needs), 7.03 / 77.5 ms; warp tiles of 384 rather than 256
// items (FP32), 6.99 / 72.7 ms. Gathering m~ into shared memory with
// cp.async (two tiles ahead, the warp's operands staged in dynamic shared
// memory) was slower than loading it: 10.9 ms on R-MAT 20.
// The moved cash alternates between two buffers (mt and the residual
// source hsrc, free while no re-derivation runs). The per-move totals
// rotate over three slots: the decision of move t reads slot q, move t adds
// into slot q + 1, and slot q + 2 (read one decision ago) is cleared by
// block 0 at the decision; no block can reach slot q + 2 again before
// block 0 has arrived at the next barrier.
// The moves and their floating-point sums are those of the general sweep's
// all-green moves up to the order of the in-link sums: m~ = C s rounded to
// the cash type, in-link sums in the cash type in merge-path order over warp
// tiles (a split row's pieces added in arrival order), H accumulated in
// FP64.
#pragma once

#include "rlgl_sweep.cuh"

namespace rlgl {

constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kPowerMinBlocks = 3;  // blocks per SM (launch bounds: up to 85 registers a thread)

// Merge-path items per lane of a warp tile: 12 for FP32 cash (384-item
// tiles), 8 for FP64 (256-item tiles, so that a block's static shared
// memory stays within 48 KB).
__host__ __device__ constexpr int power_ipt(int cash_bytes) { return cash_bytes == 4 ? 12 : 8; }

// Shared memory of one warp of the power sweep: its merge-path tile (the
// gathered in-link values, the row ends) and each row's in-link sum (local
// row index).
template <typename T>
struct PowWarp {
    static constexpr int kItems = 32 * power_ipt((int)sizeof(T));
    T val[kItems];
    int end[kItems + 1];
    T rsum[kItems];
};

// Per-thread sums of a move: ||C_{t+1}||_1, sum C_{t+1}, sum M_t, sum |M_t|
// (in the cash type, combined per block and then in FP64).
template <typename T>
struct PowAcc {
    T a, s, m, ma;
};

// Row epilogue of an all-green move: row r's in-link sum v is C_{t+1},r;
// old = C_t,r and sc = s_r.
template <typename T>
__device__ __forceinline__ void power_row_with(const SweepArgs<T>& A, T* __restrict__ mt_next, long long r, T v,
                                               T old, T sc, PowAcc<T>& acc) {
    A.c[r] = v;
    mt_next[r] = v * sc;
    red_add(A.H + r, (double)old);  // M_t,r joins the history (no load: the L2 adds)
    acc.a += fabs(v);
    acc.s += v;
    acc.m += old;
    acc.ma += fabs(old);
}

template <typename T>
__device__ __forceinline__ void power_row(const SweepArgs<T>& A, T* __restrict__ mt_next, long long r, T v,
                                          PowAcc<T>& acc) {
    const T old = __ldcg(A.c + r);  // C_t,r (this kernel stored it one move ago)
    const T sc = __ldg(row_scale(A.sf, A.s, T(0)) + r);
    power_row_with<T>(A, mt_next, r, v, old, sc, acc);
}

// Bounds of tile b: first row, first in-link, rows ending in it, in-links.
struct TileB {
    long long r0, e0;
    int nr, ne;
};

__device__ __forceinline__ TileB tile_bounds(const long long* __restrict__ tile_r,
                                             const long long* __restrict__ tile_e, long long b) {
    TileB t;
    t.r0 = __ldg(tile_r + b);
    t.e0 = __ldg(tile_e + b);
    t.nr = (int)(__ldg(tile_r + b + 1) - t.r0);
    t.ne = (int)(__ldg(tile_e + b + 1) - t.e0);
    return t;
}

// Segmented inclusive scan over the lanes of a warp: the running sum of val
// restarts wherever key changes (keys >= 0 form contiguous runs).
template <typename T>
__device__ __forceinline__ T warp_segscan(long long key, T val) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, val, o);
        const long long ky = __shfl_up_sync(0xffffffffu, key, o);
        if (lane >= o && ky == key) val += y;
    }
    return val;
}

// One move's pull with the row epilogue, a warp per merge-path tile: the
// warps of the grid take the tiles w, w + W, w + 2W, ... for all but the
// last two rounds, and the rest one at a time from the counter `next` (lane
// 0 asks one turn ahead), so that warps end within about one tile of one
// another. While a warp sums a tile, the next tile's bounds and in-link
// sources are in flight. No block-wide barrier: a warp's lanes meet only at
// __syncwarp. The pieces of rows that cross tile boundaries go into facc.
template <typename T, bool kHasW>
__device__ __forceinline__ void power_tiles(const SweepArgs<T>& A, const T* __restrict__ mt_cur,
                                            T* __restrict__ mt_next, PowWarp<T>& ws,
                                            unsigned long long* next, PowAcc<T>& acc) {
    constexpr int kPowIpt = power_ipt((int)sizeof(T));
    const int lane = threadIdx.x & 31;
    const long long ntiles = A.nwtiles;
    const long long nw = (long long)gridDim.x * kWarpsPerBlock;
    const long long w = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const long long rounds = ntiles / nw > 2 ? ntiles / nw - 2 : 0;  // tiles taken in turn
    const long long dyn0 = rounds * nw;                              // the first handed-out tile
    const T* __restrict__ scale = row_scale(A.sf, A.s, T(0));
    unsigned long long grab = 0, g0 = 0;
    if (lane == 0) {
        if (rounds < 1) g0 = atomicAdd(next, 1ull);
        if (rounds < 2) grab = atomicAdd(next, 1ull);  // turn 1
    }
    long long b = rounds > 0 ? w : dyn0 + (long long)__shfl_sync(0xffffffffu, g0, 0);
    TileB t{0, 0, 0, 0};
    int sidx[kPowIpt];
    if (b < ntiles) t = tile_bounds(A.wtile_r, A.wtile_e, b);
#pragma unroll
    for (int q = 0; q < kPowIpt; ++q) {
        const int k = lane + q * 32;
        sidx[q] = (b < ntiles && k < t.ne) ? __ldg(A.t_src + t.e0 + k) : -1;
    }
    for (long long s = 0; b < ntiles; ++s) {
        T oldv = T(0), scv = T(0);
        int start0;
        TileB tn{0, 0, 0, 0};
        long long bn;
        {
            // m~ of this move was written by other warps one move ago: L2
            T v[kPowIpt];
#pragma unroll
            for (int q = 0; q < kPowIpt; ++q) v[q] = (sidx[q] >= 0) ? __ldcg(mt_cur + sidx[q]) : T(0);
#pragma unroll
            for (int q = 0; q < kPowIpt; ++q) {
                const int k = lane + q * 32;
                if (kHasW && k < t.ne) asm volatile("prefetch.global.L1 [%0];" ::"l"(A.t_w + t.e0 + k));
            }
            // the next tile's bounds and sources, in flight over this tile
            bn = s + 1 < rounds ? w + (s + 1) * nw : dyn0 + (long long)__shfl_sync(0xffffffffu, grab, 0);
            if (bn < ntiles && s + 2 >= rounds && lane == 0) grab = atomicAdd(next, 1ull);
            if (bn < ntiles) tn = tile_bounds(A.wtile_r, A.wtile_e, bn);
#pragma unroll
            for (int q = 0; q < kPowIpt; ++q) {
                const int k = lane + q * 32;
                sidx[q] = (bn < ntiles && k < tn.ne) ? __ldg(A.t_src + tn.e0 + k) : -1;
            }
            int re[kPowIpt];
#pragma unroll
            for (int q = 0; q < kPowIpt; ++q) {
                const int k = lane + q * 32;
                re[q] = (k < t.nr) ? (int)(__ldg(A.t_ptr + t.r0 + 1 + k) - t.e0) : 0;
            }
            start0 = (int)(__ldg(A.t_ptr + t.r0) - t.e0);
            // the epilogue's first row of this lane, read with the gathers
            if (lane < t.nr) {
                oldv = __ldcg(A.c + t.r0 + lane);
                scv = __ldg(scale + t.r0 + lane);
            }
#pragma unroll
            for (int q = 0; q < kPowIpt; ++q) {
                const int k = lane + q * 32;
                if (k < t.ne) ws.val[k] = kHasW ? v[q] * (T)__ldg(A.t_w + t.e0 + k) : v[q];
                if (k < t.nr) ws.end[k] = re[q];
            }
        }
        if (lane == 0) ws.end[t.nr] = 0x7fffffff;
        __syncwarp();
        const int total = t.nr + t.ne;
        int d = lane * kPowIpt;
        long long rowA = -1, rowB = -1;
        T accA = T(0), accB = T(0);
        if (d < total) {
            const int dend = min(d + kPowIpt, total);
            int lo = max(0, d - t.ne), hi = min(d, t.nr);
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (ws.end[mid] >= d - mid) hi = mid; else lo = mid + 1;
            }
            int i = lo, j = d - lo;
            const int row_start = (i == 0) ? start0 : ws.end[i - 1];
            bool whole = (j == row_start);  // no in-link of row i before this lane
            T sum = T(0);
            int cnt = 0;
            for (; d < dend; ++d) {
                if (j < ws.end[i]) {
                    sum += ws.val[j];
                    ++j;
                    ++cnt;
                } else {
                    if (!whole) {
                        rowA = t.r0 + i;
                        accA = sum;
                    } else {
                        ws.rsum[i] = sum;  // a row with no in-link sums to zero
                    }
                    sum = T(0);
                    cnt = 0;
                    ++i;
                    whole = true;
                }
            }
            if (cnt > 0 || !whole) {
                rowB = t.r0 + i;
                accB = sum;
            }
        }
        const T run = warp_segscan<T>(rowB, accB);
        const long long pkey = __shfl_up_sync(0xffffffffu, rowB, 1);
        const T pval = __shfl_up_sync(0xffffffffu, run, 1);
        const bool first_split = start0 < 0;  // the tile's first row began in an earlier tile
        if (rowA >= 0) {
            T sum = accA;
            if (lane > 0 && pkey == rowA) sum += pval;
            if (rowA == t.r0 && first_split)
                atomicAdd(A.facc + rowA, sum);  // counted at the next tile
            else
                ws.rsum[rowA - t.r0] = sum;
        }
        const int last = (total - 1) / kPowIpt;
        if (lane == last && rowB >= 0) atomicAdd(A.facc + rowB, run);
        __syncwarp();
        // the rows that end in this tile and began in it
        for (int k = lane; k < t.nr; k += 32) {
            if (k == 0 && first_split) continue;
            if (k == lane)
                power_row_with<T>(A, mt_next, t.r0 + k, ws.rsum[k], oldv, scv, acc);
            else
                power_row<T>(A, mt_next, t.r0 + k, ws.rsum[k], acc);
        }
        __syncwarp();  // the warp's shared memory is rewritten next
        b = bn;
        t = tn;
    }
}

// The rows whose in-links cross warp tiles, once every piece is in facc
// (after the move's first grid barrier): the row that ends in tile b began
// in an earlier tile when t_ptr[r0] < e0. Each such row ends in one tile.
template <typename T>
__device__ __forceinline__ void power_split_rows(const SweepArgs<T>& A, T* __restrict__ mt_next, PowAcc<T>& acc) {
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < A.nwtiles;
         b += (long long)gridDim.x * blockDim.x) {
        const long long r0 = __ldg(A.wtile_r + b);
        if (__ldg(A.wtile_r + b + 1) == r0 || __ldg(A.t_ptr + r0) >= __ldg(A.wtile_e + b)) continue;
        const T v = __ldcg(A.facc + r0);
        A.facc[r0] = T(0);
        power_row<T>(A, mt_next, r0, v, acc);
    }
}

// The FP64 residual pull of a re-derivation (Eq. recursion_H_res), y_j +=
// sum over the in-links e of row j of hsrc[t_src[e]] (* t_w[e]), over the
// same warp tiles as the all-green sweep (kIpt items a lane: the tiles'
// size for the context's cash type) and with the same load order: the next
// tile's bounds and sources are in flight while a warp sums the current
// one. A row's sum goes into y with one reduction where it ends in the tile
// and began in it; a row that crosses a lane or tile boundary adds a piece
// per tile (lanes joined by a segmented scan), so y (zero at rest) holds
// every row's sum once the kernel has ended. Same guard as the block-tile
// pull of kind 1.
template <bool kHasW, int kIpt>
struct RederiveWarp {
    double val[32 * kIpt];
    int end[32 * kIpt + 1];
};

template <bool kHasW, int kIpt>
__global__ void __launch_bounds__(kThreads, kPowerMinBlocks)
    k_rederive_pull(double* __restrict__ y, const double* __restrict__ hsrc, const long long* __restrict__ t_ptr,
                    const int* __restrict__ t_src, const float* __restrict__ t_w,
                    const long long* __restrict__ wtile_r, const long long* __restrict__ wtile_e, long long ntiles,
                    const DevState* st) {
    if (!(st->force_refresh || (st->want_refresh && !st->done))) return;
    __shared__ RederiveWarp<kHasW, kIpt> sm[kWarpsPerBlock];
    RederiveWarp<kHasW, kIpt>& ws = sm[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * kWarpsPerBlock;
    long long b = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    TileB t{0, 0, 0, 0};
    int sidx[kIpt];
    if (b < ntiles) t = tile_bounds(wtile_r, wtile_e, b);
#pragma unroll
    for (int q = 0; q < kIpt; ++q) {
        const int k = lane + q * 32;
        sidx[q] = (b < ntiles && k < t.ne) ? __ldg(t_src + t.e0 + k) : -1;
    }
    while (b < ntiles) {
        const long long bn = b + nw;
        TileB tn{0, 0, 0, 0};
        int start0;
        {
            double v[kIpt];
#pragma unroll
            for (int q = 0; q < kIpt; ++q) v[q] = (sidx[q] >= 0) ? __ldcg(hsrc + sidx[q]) : 0.0;
            // the next tile's bounds and sources, in flight over this tile
            if (bn < ntiles) tn = tile_bounds(wtile_r, wtile_e, bn);
#pragma unroll
            for (int q = 0; q < kIpt; ++q) {
                const int k = lane + q * 32;
                sidx[q] = (bn < ntiles && k < tn.ne) ? __ldg(t_src + tn.e0 + k) : -1;
            }
            int re[kIpt];
#pragma unroll
            for (int q = 0; q < kIpt; ++q) {
                const int k = lane + q * 32;
                re[q] = (k < t.nr) ? (int)(__ldg(t_ptr + t.r0 + 1 + k) - t.e0) : 0;
            }
            start0 = (int)(__ldg(t_ptr + t.r0) - t.e0);
#pragma unroll
            for (int q = 0; q < kIpt; ++q) {
                const int k = lane + q * 32;
                if (k < t.ne) ws.val[k] = kHasW ? v[q] * (double)__ldg(t_w + t.e0 + k) : v[q];
                if (k < t.nr) ws.end[k] = re[q];
            }
        }
        if (lane == 0) ws.end[t.nr] = 0x7fffffff;
        __syncwarp();
        const int total = t.nr + t.ne;
        int d = lane * kIpt;
        long long rowA = -1, rowB = -1;
        double accA = 0.0, accB = 0.0;
        if (d < total) {
            const int dend = min(d + kIpt, total);
            int lo = max(0, d - t.ne), hi = min(d, t.nr);
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (ws.end[mid] >= d - mid) hi = mid; else lo = mid + 1;
            }
            int i = lo, j = d - lo;
            const int row_start = (i == 0) ? start0 : ws.end[i - 1];
            bool whole = (j == row_start);  // no in-link of row i before this lane
            double sum = 0.0;
            int cnt = 0;
            for (; d < dend; ++d) {
                if (j < ws.end[i]) {
                    sum += ws.val[j];
                    ++j;
                    ++cnt;
                } else {
                    if (!whole) {
                        rowA = t.r0 + i;
                        accA = sum;
                    } else if (cnt > 0) {
                        red_add(y + (t.r0 + i), sum);
                    }
                    sum = 0.0;
                    cnt = 0;
                    ++i;
                    whole = true;
                }
            }
            if (cnt > 0 || !whole) {
                rowB = t.r0 + i;
                accB = sum;
            }
        }
        const double run = warp_segscan<double>(rowB, accB);
        const long long pkey = __shfl_up_sync(0xffffffffu, rowB, 1);
        const double pval = __shfl_up_sync(0xffffffffu, run, 1);
        if (rowA >= 0) red_add(y + rowA, accA + ((lane > 0 && pkey == rowA) ? pval : 0.0));
        const int last = (total - 1) / kIpt;
        if (lane == last && rowB >= 0) red_add(y + rowB, run);
        __syncwarp();  // the warp's shared memory is rewritten next
        b = bn;
        t = tn;
    }
}

// Block sums of the per-thread move sums into the slot (thread 0; FP64).
template <typename T>
__device__ __forceinline__ void power_publish(PowAcc<T>& acc, SweepSlot* sl, T* scratch) {
    T v4[4] = {acc.a, acc.s, acc.m, acc.ma};
    block_sum_n<T, 4>(v4, scratch);
    if (threadIdx.x == 0) {
        if (v4[0] != T(0)) atomicAdd(&sl->a, (double)v4[0]);
        if (v4[1] != T(0)) atomicAdd(&sl->s, (double)v4[1]);
        if (v4[2] != T(0)) atomicAdd(&sl->msum, (double)v4[2]);
        if (v4[3] != T(0)) atomicAdd(&sl->mabs, (double)v4[3]);
        if (blockIdx.x == 0) sl->tstamp = globaltimer();
    }
    acc.a = acc.s = acc.m = acc.ma = T(0);
}

__device__ __forceinline__ int rot3(int q) { return q == 2 ? 0 : q + 1; }

template <typename T, bool kHasW>
__global__ void __launch_bounds__(kThreads, kPowerMinBlocks) k_power(SweepArgs<T> A) {
    DevState* st = A.st;
    SweepState* sw = A.sw;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (st->done) {
        if (A.use_cond && lead) cudaGraphSetConditional(A.cond_loop, 0u);
        return;
    }
    __shared__ PowWarp<T> sm[kWarpsPerBlock];
    __shared__ T tscratch[4 * 32];
    __shared__ SweepCtl sc;
    __shared__ Control ctl;
    __shared__ double s_l1_refresh;
    {
        const unsigned int* src = reinterpret_cast<const unsigned int*>(&st->ctl);
        unsigned int* dst = reinterpret_cast<unsigned int*>(&ctl);
        for (int k = threadIdx.x; k < (int)(sizeof(Control) / 4); k += blockDim.x) dst[k] = src[k];
        if (threadIdx.x == 0) s_l1_refresh = st->l1_refresh;
    }
    const int n = A.n;
    if (threadIdx.x == 0) {
        sc.moves = st->moves;
        sc.solve_moves = st->solve_moves;
        sc.iters = st->iters;
        sc.tot_green = st->tot_green;
        sc.tot_edges = st->tot_edges;
        sc.push_moves = st->push_moves;
        sc.pull_moves = st->pull_moves;
        sc.hsum = st->hsum;
        sc.habs = st->habs;
        sc.t_start = st->t_start;
        sc.fresh = st->fresh;
        sc.stall_mark = st->stall_mark;
        sc.stall_count = st->stall_count;
        const unsigned long long arr = ld_acquire_u64(&sw->bar.arrived);
        sc.target = arr - arr % gridDim.x;
        sc.p = (int)(sw->bar.parity % 3u);  // the slot the first decision reads (clear)
        sc.want_refresh = 0;
        sc.have_lag = 0;
    }
    __syncthreads();
    if (ctl.test_skip_barrier && blockIdx.x == gridDim.x - 1 && gridDim.x > 1) return;
    // the moved cash of the current move (mt_cur) and of the next (mt_nxt)
    T* mt_cur = A.mt;
    T* mt_nxt = A.mt2;
    PowAcc<T> acc{T(0), T(0), T(0), T(0)};

    // ------------------------------------------------------- prologue
    // m~ = C s for the first move, the split rows' accumulators cleared, and
    // the statistics of the cash for the first stop test.
    {
        const T* scale = row_scale(A.sf, A.s, T(0));
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const T v = A.c[i];
            A.mt[i] = v * __ldg(scale + i);
            A.facc[i] = T(0);
            acc.a += fabs(v);
            acc.s += v;
        }
        power_publish<T>(acc, &sw->slot[sc.p], tscratch);
    }
    if (!grid_barrier(&sw->bar, sc.target, ctl.barrier_limit_ns)) goto aborted;

    for (;;) {
        // ------------------------------------------------------ decide
        // (thread 0 of every block, from the same totals)
        if (threadIdx.x == 0) {
            SweepSlot* sl = &sw->slot[sc.p];
            if (blockIdx.x == 0) clear_slot(&sw->slot[rot3(rot3(sc.p))]);  // read one decision ago
            const double2 as = ldcg_pair(&sl->a);         // ||C||_1 (and pr, unused)
            const double2 mm = ldcg_pair(&sl->msum);      // the last move's sum M and sum |M|
            const double2 rts = ldcg_pair(&sl->reserve);  // block 0's timer in .y
            const double sum = __ldcg(&sl->s);
            const double l1 = as.x;
            const unsigned long long now = (unsigned long long)__double_as_longlong(rts.y);
            sc.hsum += mm.x;
            sc.habs += mm.y;
            sc.l1 = l1;
            int stop = -1;
            bool skip = false, want_refresh = false;
            if (sc.want_refresh) {
                // the last move was to be followed by a re-derivation
                skip = true;
                want_refresh = true;
            } else {
                if (sc.iters == 0) sc.t_start = now;
                sc.iters++;
                const bool degenerate = !(fabs(sc.hsum) > 1e-12 * sc.habs) || sc.habs == 0.0;
                const bool converged = sc.moves >= 1 && l1 / fabs(sc.hsum) < ctl.tol;
                if (degenerate) {
                    stop = ST_DEGENERATE;
                } else if (converged) {
                    if (ctl.mixed && !sc.fresh) {
                        want_refresh = true;
                        skip = true;
                    } else {
                        stop = ST_OK;
                    }
                } else if (sc.solve_moves >= ctl.max_steps) {
                    stop = ST_NOCONV;
                } else if ((double)(now - sc.t_start) > ctl.time_limit_ns || sc.iters > ctl.max_iters) {
                    stop = ST_TIMEOUT;
                }
                if (stop < 0 && !skip && ctl.mixed &&
                    ((ctl.refresh_factor > 0.0 && l1 < ctl.refresh_factor * s_l1_refresh) ||
                     cash_stalled(l1, sc.stall_mark, sc.stall_count, ctl.stall_moves)))
                    want_refresh = true;  // after this move
            }
            sc.leave = (stop >= 0 || skip) ? 1 : 0;
            sc.want_refresh = want_refresh ? 1 : 0;
            if (blockIdx.x == 0) {
                st->l1 = l1;
                st->sum = sum;
                st->sumr = l1;
                st->theta = 0.0;
                st->theta_f = 0.0f;
                st->hsum = sc.hsum;
                st->habs = sc.habs;
                st->iters = sc.iters;
                st->t_start = sc.t_start;
                st->stall_mark = sc.stall_mark;
                st->stall_count = sc.stall_count;
                if (sc.have_lag) {
                    // the last move's record: H 1 after it
                    MoveRecord* rec = A.log + ((sc.moves - 1) % kLogCap);
                    rec->hsum = sc.hsum;
                }
                if (sc.leave) {
                    st->mode = MODE_NONE;
                    sw->bar.parity = (unsigned int)rot3(sc.p);  // clear (cleared one decision ago)
                    if (stop >= 0) {
                        st->done = 1;
                        st->status = stop;
                    } else {
                        st->want_refresh = 1;
                        st->skip_move = 1;
                    }
                    if (A.use_cond) {
                        if (stop >= 0) cudaGraphSetConditional(A.cond_loop, 0u);
                        if (ctl.mixed) cudaGraphSetConditional(A.cond_refresh, stop >= 0 ? 0u : 1u);
                    }
                } else {
                    // the move is made: green = every node, every in-link pulled
                    st->green = n;
                    st->edges = ctl.nnz;
                    st->mode = MODE_PULL;
                    st->moves = sc.moves + 1;
                    st->solve_moves = sc.solve_moves + 1;
                    st->tot_green = sc.tot_green + n;
                    st->tot_edges = sc.tot_edges + ctl.nnz;
                    st->pull_moves = sc.pull_moves + 1;
                    st->fresh = 0;
                    st->skip_move = 0;
                    MoveRecord rec;
                    rec.move = sc.moves;
                    rec.green = n;
                    rec.edges = ctl.nnz;
                    rec.mode = MODE_PULL;
                    rec.pad = 0;
                    rec.theta = 0.0;
                    rec.l1 = l1;
                    rec.hsum = sc.hsum;  // completed at the next decision
                    for (int q = 0; q < 6; ++q) rec.phase_us[q] = 0.f;
                    A.log[sc.moves % kLogCap] = rec;
                }
            }
            if (!sc.leave) {
                sc.have_lag = 1;  // (here: a move of this launch has a record to complete)
                sc.moves++;
                sc.solve_moves++;
                sc.tot_green += n;
                sc.tot_edges += ctl.nnz;
                sc.pull_moves++;
                sc.fresh = 0;
            }
        }
        __syncthreads();
        if (sc.leave) return;

        // ----------------------------------------------------------- move
        SweepSlot* nsl = &sw->slot[rot3(sc.p)];  // this move's sums and tile counter
        if (lead) sc.ts[0] = globaltimer();
        power_tiles<T, kHasW>(A, mt_cur, mt_nxt, sm[threadIdx.x >> 5], &nsl->chunk_next, acc);
        if (!grid_barrier(&sw->bar, sc.target, ctl.barrier_limit_ns, blockIdx.x == 0 ? sc.ts + 1 : nullptr))
            break;
        power_split_rows<T>(A, mt_nxt, acc);
        power_publish<T>(acc, nsl, tscratch);
        if (!grid_barrier(&sw->bar, sc.target, ctl.barrier_limit_ns, blockIdx.x == 0 ? sc.ts + 3 : nullptr))
            break;
        if (lead) {
            MoveRecord* rec = A.log + ((sc.moves - 1) % kLogCap);
            // the move's work (pull, then the split rows) and the waits at its
            // two barriers (slots 4 and 5)
            rec->phase_us[4] = (float)((sc.ts[1] - sc.ts[0]) + (sc.ts[3] - sc.ts[2])) * 1e-3f;
            rec->phase_us[5] = (float)((sc.ts[2] - sc.ts[1]) + (sc.ts[4] - sc.ts[3])) * 1e-3f;
        }
        {
            T* t = mt_cur;
            mt_cur = mt_nxt;
            mt_nxt = t;
        }
        if (threadIdx.x == 0) sc.p = rot3(sc.p);
        __syncthreads();
    }
aborted:
    // A barrier wait gave up: end the solve with an error status.
    if (threadIdx.x == 0) {
        st->done = 1;
        st->status = ST_BARRIER;
        if (A.use_cond) {
            cudaGraphSetConditional(A.cond_loop, 0u);
            if (ctl.mixed) cudaGraphSetConditional(A.cond_refresh, 0u);
        }
    }
}

}  // namespace rlgl
