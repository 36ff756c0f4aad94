// The persistent all-green sweep (power iteration, Sec. 2.3.1): the moves
// of a single-chain all-green solve in one cooperative kernel, two grid
// barriers a move and one pass over the in-links.
//
// With G_t = [N] a move is M_t = C_t, H <- H + C_t, C_{t+1} = M_t P (Eqs.
// recursion_M, recursion_H, recursion_C; every node's cash leaves it). The
// general sweep makes it in three phases (statistics, select, pull) with
// three barriers. Here the select's work is folded into the pull's row
// epilogue: when the in-link sum of row j is complete, the same thread
// reads C_t,j, adds it to H_j, stores C_{t+1},j = the sum and the next
// move's moved cash per weight m~_j = C_{t+1},j s_j, and sums the
// statistics of C_{t+1} and of M_t. A move is then
//   pull      : merge-path tiles over the in-links (handed out by a
//               counter), gathering m~ of the current move; rows that end
//               in the tile where they began go through the epilogue, the
//               pieces of rows that cross a tile boundary are added into a
//               zero-at-rest accumulator;
//   barrier   ;
//   fix-up    : the rows that crossed a tile boundary (found from the tile
//               table: a tile's first row began before the tile and ends in
//               it) go through the epilogue; block sums of the statistics;
//   barrier   ; every block takes the same decisions (stop test of Alg. 1,
//               re-derivation triggers) from the same totals.
// The moved cash alternates between two buffers (mt and the residual
// source hsrc, free while no re-derivation runs), so that a move gathers
// m~_t while it writes m~_{t+1}.
// The moves and their floating-point sums are those of the general sweep's
// all-green moves: m~ = C s rounded to the cash type, in-link sums in the
// cash type in merge-path order, H accumulated in FP64.
#pragma once

#include "rlgl_sweep.cuh"

namespace rlgl {

// Shared memory of the power sweep: the merge-path tile and each row's
// in-link sum (local row index).
template <typename T>
struct PowSmem {
    PullSmem<T> pull;
    T rsum[kMpItems];
};

// Per-thread sums of a move: ||C_{t+1}||_1, sum C_{t+1}, sum M_t, sum |M_t|
// (in the cash type, combined per block and then in FP64).
template <typename T>
struct PowAcc {
    T a, s, m, ma;
};

// Row epilogue of an all-green move: row r's in-link sum v is C_{t+1},r.
template <typename T>
__device__ __forceinline__ void power_row(const SweepArgs<T>& A, T* __restrict__ mt_next, long long r, T v,
                                          PowAcc<T>& acc) {
    const T old = __ldcg(A.c + r);  // C_t,r (this kernel stored it one move ago)
    const T sc = __ldg(row_scale(A.sf, A.s, T(0)) + r);
    A.c[r] = v;
    mt_next[r] = v * sc;
    red_add(A.H + r, (double)old);  // M_t,r joins the history (no load: the L2 adds)
    acc.a += fabs(v);
    acc.s += v;
    acc.m += old;
    acc.ma += fabs(old);
}

// One move's pull: the merge-path tiles (as pull_tiles) with the row
// epilogue; tiles handed out by the counter `next`.
template <typename T, bool kHasW>
__device__ __forceinline__ void power_tiles(const SweepArgs<T>& A, const T* __restrict__ mt_cur,
                                            T* __restrict__ mt_next, T* __restrict__ facc, PowSmem<T>& sm,
                                            unsigned long long* next, PowAcc<T>& acc) {
    PullSmem<T>& ps = sm.pull;
    __shared__ long long s_tnext;
    if (threadIdx.x == 0) s_tnext = (long long)atomicAdd(next, 1ull);
    __syncthreads();
    long long b = s_tnext;
    __syncthreads();
    const long long ntiles = A.ntiles;
    while (b < ntiles) {
        if (threadIdx.x == 0) s_tnext = (long long)atomicAdd(next, 1ull);  // read at the end
        const long long r0 = __ldg(A.tile_r + b), e0 = __ldg(A.tile_e + b);
        const int nrows = (int)(__ldg(A.tile_r + b + 1) - r0);
        const int nedges = (int)(__ldg(A.tile_e + b + 1) - e0);
        {
            int sidx[kMpIpt];
            float wv[kMpIpt];
            long long re[kMpIpt];
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) {
                const int k = threadIdx.x + q * kThreads;
                sidx[q] = (k < nedges) ? __ldg(A.t_src + e0 + k) : -1;
                if (kHasW) wv[q] = (k < nedges) ? __ldg(A.t_w + e0 + k) : 0.0f;
                re[q] = (k < nrows) ? __ldg(A.t_ptr + r0 + 1 + k) : 0;
            }
            T v[kMpIpt];
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) v[q] = (sidx[q] >= 0) ? __ldcg(mt_cur + sidx[q]) : T(0);
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) {
                const int k = threadIdx.x + q * kThreads;
                if (k < nedges) ps.val[k] = kHasW ? v[q] * (T)wv[q] : v[q];
                if (k < nrows) ps.end[k] = (int)(re[q] - e0);
            }
        }
        if (threadIdx.x == 0) {
            ps.end[nrows] = 0x7fffffff;
            ps.start0 = (int)(__ldg(A.t_ptr + r0) - e0);
        }
        __syncthreads();
        const int total = nrows + nedges;
        int d = threadIdx.x * kMpIpt;
        const bool active = d < total;
        long long rowA = -1, rowB = -1;
        T accA = T(0), accB = T(0);
        if (active) {
            const int dend = min(d + kMpIpt, total);
            int lo = max(0, d - nedges), hi = min(d, nrows);
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (ps.end[mid] >= d - mid) hi = mid; else lo = mid + 1;
            }
            int i = lo, j = d - lo;
            const int row_start = (i == 0) ? ps.start0 : ps.end[i - 1];
            bool whole = (j == row_start);  // no in-link of row i before this thread
            T s = T(0);
            int cnt = 0;
            for (; d < dend; ++d) {
                if (j < ps.end[i]) {
                    s += ps.val[j];
                    ++j;
                    ++cnt;
                } else {
                    if (!whole) {
                        rowA = r0 + i;
                        accA = s;
                    } else {
                        sm.rsum[i] = s;  // a row with no in-link sums to zero
                    }
                    s = T(0);
                    cnt = 0;
                    ++i;
                    whole = true;
                }
            }
            if (cnt > 0 || !whole) {
                rowB = r0 + i;
                accB = s;
            }
        }
        const T run = block_segscan<T>(rowB, accB, ps.ckey, ps.cval);
        if (rowA >= 0) {
            T sum = accA;
            if (threadIdx.x > 0 && ps.ckey[threadIdx.x - 1] == rowA) sum += ps.cval[threadIdx.x - 1];
            // the tile's first row may have begun in an earlier tile
            if (rowA == r0 && ps.start0 < 0) red_add(facc + rowA, sum);
            else sm.rsum[rowA - r0] = sum;
        }
        const int last = (total - 1) / kMpIpt;
        if ((int)threadIdx.x == last && rowB >= 0) red_add(facc + rowB, run);
        __syncthreads();
        // the rows that end in this tile and began in it
        for (int k = (ps.start0 < 0 ? 1 : 0) + (int)threadIdx.x; k < nrows; k += blockDim.x)
            power_row<T>(A, mt_next, r0 + k, sm.rsum[k], acc);
        b = s_tnext;
        __syncthreads();  // the tile's shared memory and s_tnext are rewritten next
    }
}

// The rows that crossed a tile boundary: tile b's first row r0 began before
// the tile (t_ptr[r0] < tile_e[b]) and ends in it (tile_r[b+1] > r0). Their
// pieces are complete in facc once every block has passed the barrier.
template <typename T>
__device__ __forceinline__ void power_fixup(const SweepArgs<T>& A, T* __restrict__ mt_next, T* __restrict__ facc,
                                            PowAcc<T>& acc) {
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < A.ntiles;
         b += (long long)gridDim.x * blockDim.x) {
        const long long r0 = __ldg(A.tile_r + b);
        if (__ldg(A.tile_r + b + 1) > r0 && __ldg(A.t_ptr + r0) < __ldg(A.tile_e + b)) {
            const T v = __ldcg(facc + r0);
            facc[r0] = T(0);
            power_row<T>(A, mt_next, r0, v, acc);
        }
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

template <typename T, bool kHasW>
__global__ void __launch_bounds__(kThreads, kSweepMinBlocks) k_power(SweepArgs<T> A) {
    DevState* st = A.st;
    SweepState* sw = A.sw;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (st->done) {
        if (A.use_cond && lead) cudaGraphSetConditional(A.cond_loop, 0u);
        return;
    }
    __shared__ PowSmem<T> sm;
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
        sc.p = (int)(sw->bar.parity & 1u);
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
    // m~ = C s for the first move, the accumulator of split rows cleared,
    // and the statistics of the cash for the first stop test.
    {
        if (lead) clear_slot(&sw->slot[sc.p ^ 1]);  // the first move's slot
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
            const double2 as = ldcg_pair(&sl->a);        // ||C||_1 (and pr, unused)
            const double2 mm = ldcg_pair(&sl->msum);     // the last move's sum M and sum |M|
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
                    // the last move's record: H 1 after it and its phase times
                    MoveRecord* rec = A.log + ((sc.moves - 1) % kLogCap);
                    rec->hsum = sc.hsum;
                }
                if (sc.leave) {
                    st->mode = MODE_NONE;
                    sw->bar.parity = (unsigned int)(sc.p ^ 1);
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
        SweepSlot* nsl = &sw->slot[sc.p ^ 1];  // this move's sums and tile counter
        if (lead) sc.ts[0] = globaltimer();
        power_tiles<T, kHasW>(A, mt_cur, mt_nxt, A.facc, sm, &nsl->chunk_next, acc);
        if (!grid_barrier(&sw->bar, sc.target, ctl.barrier_limit_ns, blockIdx.x == 0 ? sc.ts + 1 : nullptr))
            break;
        // every block has read this move's decision slot: clear it for the
        // move after next
        if (lead) clear_slot(&sw->slot[sc.p]);
        power_fixup<T>(A, mt_nxt, A.facc, acc);
        power_publish<T>(acc, nsl, tscratch);
        if (!grid_barrier(&sw->bar, sc.target, ctl.barrier_limit_ns, blockIdx.x == 0 ? sc.ts + 3 : nullptr))
            break;
        if (lead) {
            MoveRecord* rec = A.log + ((sc.moves - 1) % kLogCap);
            // pull work, wait at its barrier, fix-up work, wait (slots 4, 5, 2, 3)
            rec->phase_us[4] = (float)(sc.ts[1] - sc.ts[0]) * 1e-3f;
            rec->phase_us[5] = (float)(sc.ts[2] - sc.ts[1]) * 1e-3f;
            rec->phase_us[2] = (float)(sc.ts[3] - sc.ts[2]) * 1e-3f;
            rec->phase_us[3] = (float)(sc.ts[4] - sc.ts[3]) * 1e-3f;
        }
        {
            T* t = mt_cur;
            mt_cur = mt_nxt;
            mt_nxt = t;
        }
        if (threadIdx.x == 0) sc.p ^= 1;
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
