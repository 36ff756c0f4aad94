// The persistent batch solve: many independent chains stacked
// block-diagonally, every chain solved by Alg. 1 on its own (its own
// statistics, threshold, frontier, stop test and tolerance), all in one
// cooperative launch.
//
// Work is handed out by chain: the host sorts the chains by size (largest
// first) and gives chain k a group of g_k blocks (1 for most chains, more
// for the largest, so that no chain takes much longer than an even share of
// the batch). The queue holds one entry per (chain, member); a block takes
// the next entry from a counter, runs that chain's whole solve as member m
// of its group, then takes the next entry. The members of a group meet at
// per-chain barriers (a counter in the chain's own line, bounded waits; a
// group of one block meets at __syncthreads), so chains never wait for one
// another. A move of chain k is, as in the one-chain sweep,
//   stats  : its members' node shares; sums into the chain's slot;
//   barrier; every member takes the same decisions from the same totals;
//   select : the green nodes of each share compacted into the chain's own
//            frontier region (slots node_ptr[k].., edge offsets counted
//            from the chain's first frontier edge, push chunks in the
//            chain's own part of the chunk index);
//   barrier; push over the chain's frontier chunks, or pull over the
//            chain's own merge-path tiles;
//   barrier.
// The MIXED path re-derives a chain's cash in FP64 inside the launch, over
// the chain's tiles, whenever that chain's triggers ask for it.
#pragma once

#include "rlgl_sweep.cuh"

namespace rlgl {

// Accumulators of one move of one chain (zero at rest).
struct BSlot {
    double a, s, pr;        // ||C||_1, sum C, sum v^r
    double msum, mabs;      // sum m_i, sum |m_i| of the moved cash
    double l1r;             // ||C||_1 after a re-derivation
    unsigned long long reserve;     // packed frontier reservation
    unsigned long long chunk_next;  // next push chunk / pull tile (groups of > 1 block)
    unsigned long long tstamp;      // member 0's timer at the end of its stats
    unsigned long long pad[7];
};

// Per chain: the group barrier and two slots (alternating moves).
struct alignas(128) BGroup {
    unsigned long long arrived;  // arrivals of this chain's members
    unsigned int abort;          // a wait of this group gave up
    unsigned int pad[29];
    BSlot slot[2];
};

template <typename T>
struct BatchArgs {
    T* c;
    double* H;
    const double* s;
    const float* sf;
    const long long* row_ptr;
    const T* ideg;
    const unsigned char* masks;
    T* mt;
    long long* f_eoff;
    long long* f_base;
    T* f_m;
    int* chunk_row;
    const int* col;
    const float* w;
    const long long* t_ptr;
    const int* t_src;
    const float* t_w;
    const long long* ct_r;    // per-chain merge-path tiles (global row / edge
    const long long* ct_e;    // coordinates); chain k's entries start at
    const long long* ct_off;  // ct_off[k] and end at ct_off[k+1] - 1
    const long long* node_ptr;
    ChainState* cs;
    BGroup* grp;
    const int* q_chain;   // queue entry -> chain
    const int* q_member;  // queue entry -> member index in the chain's group
    const int* g_of;      // chain -> group size
    long long q_len;
    unsigned long long* q_next;
    double* y;     // FP64 re-derivation accumulator (zero at rest)
    double* hsrc;  // FP64 re-derivation source H s
    DevState* st;
    int nchains;
};

// The decisions of one chain's solve, one copy per block (thread 0 keeps
// it); every member of the group applies the same updates to the same
// totals.
struct BCtl {
    long long moves, solve_moves, edges, green, s_edges, s_green, s_push, s_pull, s_refr;
    double hsum, habs, l1, sum, sumr, theta, tol, l1r, stall_mark;
    long long stall_count;
    unsigned long long target;
    float theta_f;
    int fresh, sched, mode, p, stop, act;  // act: 0 move, 1 re-derive then test again, 2 leave
    int want_refresh;
    SchedAux ax;
    long long mask_off;
};

template <typename T, int kBT>
union BatchSmem {
    PushSmem<T, kBT> push;
    PullSmem<T, kBT> pull;
    PullSmem<double, kBT> pull64;
};

// Group barrier of chain k's g members: __syncthreads for a group of one
// block; else every member's thread 0 fences, adds one to the chain's
// arrival count and waits (bounded) until it reaches the members' common
// target. Returns false in every thread of the block when the group must
// give up (a wait ran out here or in another member).
template <int kBT>
__device__ __forceinline__ bool group_barrier(BGroup* gp, int g, unsigned long long& target,
                                              unsigned long long limit_ns) {
    __shared__ int s_gok;
    __syncthreads();
    if (g == 1) return true;
    if (threadIdx.x == 0) {
        target += (unsigned long long)g;
        __threadfence();
        asm volatile("red.relaxed.gpu.global.add.u64 [%0], 1;" ::"l"(&gp->arrived) : "memory");
        int ok = 1;
        const unsigned long long t0 = globaltimer();
        unsigned int spins = 0;
        while (ld_acquire_u64(&gp->arrived) < target) {
            if ((++spins & 15u) == 0u) {
                if (ld_acquire_u32(&gp->abort)) {
                    ok = 0;
                    break;
                }
                if (globaltimer() - t0 > limit_ns) {
                    atomicExch(&gp->abort, 1u);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
        s_gok = ok;
    }
    __syncthreads();
    return s_gok != 0;
}

// Member m's share of the chain's nodes [a, b): contiguous, in whole
// block-iterations (kBT * kNodesPerThread nodes) where the chain is large.
template <int kBT>
__device__ __forceinline__ void member_share(long long a, long long b, int m, int g, long long& lo,
                                             long long& hi) {
    const long long unit = (long long)kBT * kNodesPerThread;
    const long long iters = (b - a + unit - 1) / unit;
    const long long per = (iters + g - 1) / g;
    lo = a + (long long)m * per * unit;
    hi = lo + per * unit;
    if (lo > b) lo = b;
    if (hi > b) hi = b;
}

// One chain's FP64 re-derivation of its cash, C = H (P - I) (Eq.
// recursion_H_res; a batch starts from step 0, C_0 = 0), by the group:
// H s over the shares, the in-link pull over the chain's tiles into y, then
// C = fl(y - H), y = 0. Returns ||C||_1 of the stored cash in thread 0 (via
// the slot), and false when a group barrier gave up.
template <typename T, bool kHasW, int kBT>
__device__ __noinline__ bool batch_refresh(const BatchArgs<T>& A, BatchSmem<T, kBT>& sm, BGroup* gp, BSlot* sl, int g, int m,
                              long long lo, long long hi, long long ct0, long long ntk,
                              unsigned long long& target, unsigned long long limit_ns, double& l1r) {
    __shared__ double scratch[32];
    // (H was added to with red.global by the group: read it from L2)
    for (long long i = lo + threadIdx.x; i < hi; i += kBT) A.hsrc[i] = __ldcg(A.H + i) * A.s[i];
    if (!group_barrier<kBT>(gp, g, target, limit_ns)) return false;
    pull_tiles<double, double, kHasW, true, kBT>(A.y, A.hsrc, A.t_ptr, A.t_src, A.t_w, A.ct_r + ct0, A.ct_e + ct0,
                                                 ntk, m, g, sm.pull64);
    if (!group_barrier<kBT>(gp, g, target, limit_ns)) return false;
    double l1 = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kBT) {
        const double ex = __ldcg(A.y + i) - __ldcg(A.H + i);
        const T v = (T)ex;
        A.c[i] = v;
        A.y[i] = 0.0;
        l1 += fabs((double)v);
    }
    l1 = block_sum(l1, scratch);
    if (threadIdx.x == 0 && l1 != 0.0) atomicAdd(&sl->l1r, l1);
    if (!group_barrier<kBT>(gp, g, target, limit_ns)) return false;
    if (threadIdx.x == 0) l1r = __ldcg(&sl->l1r);
    return true;
}

// The whole solve of chain k as member m of its group of g blocks.
template <typename T, bool kHasW, int kBT>
__device__ void batch_chain(const BatchArgs<T>& A, const Control& ctl, BatchSmem<T, kBT>& sm, BCtl& bc, int k,
                            int m, int g, unsigned long long t_start, long long mask_base) {
    __shared__ T tscratch[4 * 32];
    __shared__ unsigned long long base_sh;
    constexpr bool kF32 = std::is_same<T, float>::value;
    const long long a = A.node_ptr[k], b = A.node_ptr[k + 1];
    const long long nk = b - a;
    const long long e_lo = A.row_ptr[a];
    const long long nnz_k = A.row_ptr[b] - e_lo;
    const long long cbase = e_lo / kPushChunk + k;
    const long long ct0 = A.ct_off[k];
    const long long ntk = A.ct_off[k + 1] - ct0 - 1;
    long long lo, hi;
    member_share<kBT>(a, b, m, g, lo, hi);
    BGroup* gp = A.grp + k;
    ChainState* ch = A.cs + k;
    const unsigned long long limit = ctl.barrier_limit_ns;
    const bool link = ctl.sched == SCHED_LINK;
    const int r = ctl.r;
    if (threadIdx.x == 0) {
        bc.moves = ch->moves;
        bc.solve_moves = 0;
        bc.s_edges = bc.s_green = bc.s_push = bc.s_pull = bc.s_refr = 0;
        bc.hsum = ch->hsum;
        bc.habs = ch->habs;
        bc.tol = ch->tol;
        bc.fresh = ch->fresh;
        bc.l1r = ch->l1r;
        bc.stall_mark = kNoMark;
        bc.stall_count = 0;
        bc.target = 0ull;
        bc.p = 0;
        bc.stop = -1;
        bc.want_refresh = 0;
        bc.l1 = bc.sum = bc.sumr = bc.theta = 0.0;
        bc.theta_f = 0.f;
    }
    __syncthreads();
    bool ok = true;
    for (;;) {
        BSlot* sl = &gp->slot[bc.p];
        // ------------------------------------------------------ stats
        {
            T sa = T(0), ss = T(0), spr = T(0);
            // kNodesPerThread nodes a thread, all loads issued before any sum
            constexpr long long kUnit = (long long)kBT * kNodesPerThread;
            for (long long it0 = lo; it0 < hi; it0 += kUnit) {
                T v[kNodesPerThread], idg[kNodesPerThread];
#pragma unroll
                for (int q = 0; q < kNodesPerThread; ++q) {
                    const long long i = it0 + q * kBT + threadIdx.x;
                    v[q] = i < hi ? __ldcg(A.c + i) : T(0);
                    idg[q] = (link && i < hi) ? __ldg(A.ideg + i) : T(0);
                }
#pragma unroll
                for (int q = 0; q < kNodesPerThread; ++q) {
                    const T av = fabs(v[q]);
                    sa += av;
                    ss += v[q];
                    const T tv = link ? av * idg[q] : av;
                    if (link && r == 1) spr += tv;
                    else if (r == 2) spr += tv * tv;
                    else if (r > 2) spr += pow_r(tv, r);
                }
            }
            T v3[4] = {sa, ss, spr, T(0)};
            block_sum_n<T, 4>(v3, tscratch);
            if (threadIdx.x == 0) {
                if (v3[0] != T(0)) atomicAdd(&sl->a, (double)v3[0]);
                if (v3[1] != T(0)) atomicAdd(&sl->s, (double)v3[1]);
                if (v3[2] != T(0)) atomicAdd(&sl->pr, (double)v3[2]);
                if (m == 0) sl->tstamp = globaltimer();
            }
        }
        if (!(ok = group_barrier<kBT>(gp, g, bc.target, limit))) break;
        // ---------------------------------------------------- control
        if (threadIdx.x == 0) {
            if (m == 0) {
                // every member is done with the other slot (the last move's)
                BSlot* o = &gp->slot[bc.p ^ 1];
                o->a = o->s = o->pr = o->msum = o->mabs = o->l1r = 0.0;
                o->reserve = o->chunk_next = 0ull;
            }
            const double l1 = __ldcg(&sl->a), sum = __ldcg(&sl->s), pr = __ldcg(&sl->pr);
            const unsigned long long now = __ldcg(&sl->tstamp);
            const double sumr = (r == 1 && !link) ? l1 : pr;
            bc.l1 = l1;
            bc.sum = sum;
            bc.sumr = sumr;
            if (bc.solve_moves == 0 && bc.fresh && bc.l1r == 0.0) bc.l1r = l1;  // step 0's cash
            int stop = -1, act = 0;
            const bool degenerate = !(fabs(bc.hsum) > 1e-12 * bc.habs) || bc.habs == 0.0;
            const bool converged = bc.moves >= 1 && l1 / fabs(bc.hsum) < bc.tol;
            if (degenerate) stop = ST_DEGENERATE;
            else if (converged) {
                if (ctl.mixed && !bc.fresh) act = 1;
                else stop = ST_OK;
            } else if (bc.solve_moves >= ctl.max_steps) stop = ST_NOCONV;
            else if ((double)(now - t_start) > ctl.time_limit_ns) stop = ST_TIMEOUT;
            if (stop >= 0) act = 2;
            bc.want_refresh = 0;
            if (act == 0 && ctl.mixed &&
                ((ctl.refresh_factor > 0.0 && l1 < ctl.refresh_factor * bc.l1r) ||
                 cash_stalled(l1, bc.stall_mark, bc.stall_count, ctl.stall_moves)))
                bc.want_refresh = 1;
            bc.stop = stop;
            bc.act = act;
            int sched = ctl.sched;
            if (ctl.safety_every > 0 && ((bc.solve_moves + 1) % ctl.safety_every) == 0) sched = SCHED_ALL_GREEN;
            double th = 0.0;
            if (sched == SCHED_THRESHOLD || sched == SCHED_LINK) {
                const double mean = sumr / (double)nk;
                th = ctl.theta_arg > 0.0 ? ctl.theta_arg
                                         : (r == 1 ? ctl.theta_scale * mean : ctl.theta_scale * pow(mean, 1.0 / r));
            }
            bc.sched = sched;
            bc.theta = th;
            bc.theta_f = (sched == SCHED_LINK) ? __double2float_rn(th) : __double2float_ru(th);
            bc.ax = sched_aux(ctl, nk, bc.moves, l1, sched);
            // MASK: the k-th move of the solve takes set (cursor + k) mod period
            bc.mask_off = (sched == SCHED_MASK) ? ((mask_base + bc.solve_moves) % ctl.n_masks) : 0;
        }
        __syncthreads();
        if (bc.act == 2) break;
        if (bc.act == 1) {
            // re-derive, then test again with fresh statistics
            double l1r = 0.0;
            if (!(ok = batch_refresh<T, kHasW, kBT>(A, sm, gp, sl, g, m, lo, hi, ct0, ntk, bc.target, limit, l1r)))
                break;
            if (threadIdx.x == 0) {
                bc.l1r = l1r;
                bc.fresh = 1;
                bc.stall_mark = kNoMark;
                bc.stall_count = 0;
                bc.s_refr++;
                bc.p ^= 1;
            }
            __syncthreads();
            continue;
        }
        // ----------------------------------------------------- select
        {
            const int sched = bc.sched;
            const T th = kF32 ? (T)bc.theta_f : (T)bc.theta;
            const unsigned char* mask = nullptr;
            if (sched == SCHED_MASK) mask = A.masks + (size_t)bc.mask_off * (size_t)A.node_ptr[A.nchains];
            const SchedAux ax = bc.ax;
            T msum = T(0), mabs = T(0);
            const bool dense = sched == SCHED_ALL_GREEN;
            const T* scale = row_scale(A.sf, A.s, T(0));
            for (long long it0 = lo; it0 < hi; it0 += (long long)kBT * kNodesPerThread) {
                long long rb[kNodesPerThread];
                int rdeg[kNodesPerThread];
                T val[kNodesPerThread], sc[kNodesPerThread];
                bool gq[kNodesPerThread];
                unsigned long long mine = 0ull;
                // every load of the range before the first red_add below
#pragma unroll
                for (int q = 0; q < kNodesPerThread; ++q) {
                    const long long i = it0 + q * kBT + threadIdx.x;
                    const bool in = i < hi;
                    val[q] = in ? __ldcg(A.c + i) : T(0);
                    sc[q] = in ? __ldg(scale + i) : T(0);
                    rb[q] = (in && !dense) ? __ldg(A.row_ptr + i) : 0;
                    rdeg[q] = (in && !dense) ? (int)(__ldg(A.row_ptr + i + 1) - rb[q]) : 0;
                    const T idg = (in && sched == SCHED_LINK) ? __ldg(A.ideg + i) : T(0);
                    gq[q] = in && green_test_v<T>(sched, val[q], idg, i - a, th, mask ? mask + a : nullptr, ax);
                    if (gq[q] && !dense) mine += ((unsigned long long)rdeg[q] << kCountBits) + 1ull;
                }
                if (dense) {
#pragma unroll
                    for (int q = 0; q < kNodesPerThread; ++q) {
                        const long long i = it0 + q * kBT + threadIdx.x;
                        if (i >= hi) continue;
                        const T v = val[q];
                        A.c[i] = T(0);
                        red_add(A.H + i, (double)v);
                        msum += v;
                        mabs += fabs(v);
                        A.mt[i] = v * sc[q];
                    }
                    continue;
                }
                unsigned long long tot;
                const unsigned long long pre = block_exscan<kBT>(mine, &tot);
                if (threadIdx.x == 0) base_sh = tot ? atomicAdd(&sl->reserve, tot) : 0ull;
                __syncthreads();
                const unsigned long long base = base_sh + pre;
                long long kk = (long long)(base & ((1ull << kCountBits) - 1ull));
                long long ee = (long long)(base >> kCountBits);
#pragma unroll
                for (int q = 0; q < kNodesPerThread; ++q) {
                    const long long i = it0 + q * kBT + threadIdx.x;
                    if (i >= hi) continue;
                    if (gq[q]) {
                        const T v = val[q];
                        const T mtil = v * sc[q];
                        A.c[i] = T(0);
                        red_add(A.H + i, (double)v);
                        msum += v;
                        mabs += fabs(v);
                        A.mt[i] = mtil;
                        A.f_eoff[a + kk] = ee;
                        A.f_base[a + kk] = rb[q] - ee;
                        A.f_m[a + kk] = mtil;
                        const long long b0 = (ee + kPushChunk - 1) / kPushChunk;
                        const long long b1 = (ee + rdeg[q] + kPushChunk - 1) / kPushChunk;
                        for (long long cb = b0; cb < b1; ++cb) A.chunk_row[cbase + cb] = (int)kk;
                        ++kk;
                        ee += rdeg[q];
                    } else {
                        A.mt[i] = T(0);
                    }
                }
                __syncthreads();  // base_sh is rewritten next
            }
            T v2[4] = {msum, mabs, T(0), T(0)};
            block_sum_n<T, 4>(v2, tscratch);
            if (threadIdx.x == 0) {
                if (v2[0] != T(0)) atomicAdd(&sl->msum, (double)v2[0]);
                if (v2[1] != T(0)) atomicAdd(&sl->mabs, (double)v2[1]);
            }
        }
        if (!(ok = group_barrier<kBT>(gp, g, bc.target, limit))) break;
        // ------------------------------------------------ choose move
        if (threadIdx.x == 0) {
            const unsigned long long rsv = __ldcg(&sl->reserve);
            long long green = (long long)(rsv & ((1ull << kCountBits) - 1ull));
            long long edges = (long long)(rsv >> kCountBits);
            if (bc.sched == SCHED_ALL_GREEN) {
                green = nk;
                edges = nnz_k;
            }
            bc.hsum += __ldcg(&sl->msum);
            bc.habs += __ldcg(&sl->mabs);
            bc.moves++;
            bc.solve_moves++;
            bc.fresh = 0;
            bc.green = green;
            bc.edges = edges;
            bc.s_green += green;
            bc.s_edges += edges;
            int mode;
            if (green == 0) mode = MODE_NONE;
            else if (bc.sched == SCHED_ALL_GREEN || (double)edges >= ctl.pull_crossover * (double)nnz_k)
                mode = MODE_PULL;
            else
                mode = MODE_PUSH;
            if (mode == MODE_PUSH) bc.s_push++;
            if (mode == MODE_PULL) bc.s_pull++;
            bc.mode = mode;
        }
        __syncthreads();
        // -------------------------------------------------------- move
        if (bc.mode == MODE_PUSH)
            push_chunks<T, kHasW, true, kBT>(A.c, A.col, A.w, A.f_eoff + a, A.f_base + a, A.f_m + a,
                                             A.chunk_row + cbase, bc.edges, bc.green, m, g, sm.push, nullptr,
                                             g > 1 ? &sl->chunk_next : nullptr);
        else if (bc.mode == MODE_PULL)
            pull_tiles<T, T, kHasW, true, kBT>(A.c, A.mt, A.t_ptr, A.t_src, A.t_w, A.ct_r + ct0, A.ct_e + ct0, ntk,
                                               m, g, sm.pull, g > 1 ? &sl->chunk_next : nullptr);
        if (!(ok = group_barrier<kBT>(gp, g, bc.target, limit))) break;
        if (bc.want_refresh) {
            double l1r = 0.0;
            if (!(ok = batch_refresh<T, kHasW, kBT>(A, sm, gp, sl, g, m, lo, hi, ct0, ntk, bc.target, limit, l1r)))
                break;
            if (threadIdx.x == 0) {
                bc.l1r = l1r;
                bc.fresh = 1;
                bc.stall_mark = kNoMark;
                bc.stall_count = 0;
                bc.s_refr++;
            }
        }
        if (threadIdx.x == 0) bc.p ^= 1;
        __syncthreads();
    }
    // member 0 records the chain's result
    if (threadIdx.x == 0 && m == 0) {
        const int stop = ok ? bc.stop : ST_TIMEOUT;
        ch->moves = bc.moves;
        ch->hsum = bc.hsum;
        ch->habs = bc.habs;
        ch->l1 = bc.l1;
        ch->sum = bc.sum;
        ch->sumr = bc.sumr;
        ch->theta = bc.theta;
        ch->theta_f = bc.theta_f;
        ch->fresh = bc.fresh;
        ch->l1r = bc.l1r;
        ch->s_moves = bc.solve_moves;
        ch->s_edges = bc.s_edges;
        ch->s_green = bc.s_green;
        ch->s_push = bc.s_push;
        ch->s_pull = bc.s_pull;
        ch->s_refr = bc.s_refr;
        ch->status = stop;
        ch->done = 1;
    }
    __syncthreads();
}

template <typename T, bool kHasW, int kBT>
__global__ void __launch_bounds__(kBT, 1024 / kBT) k_bsweep(BatchArgs<T> A) {
    __shared__ BatchSmem<T, kBT> sm;
    __shared__ BCtl bc;
    __shared__ Control ctl;
    __shared__ long long s_entry;
    __shared__ unsigned long long s_t0;
    __shared__ long long s_mask_base;
    {
        const unsigned int* src = reinterpret_cast<const unsigned int*>(&A.st->ctl);
        unsigned int* dst = reinterpret_cast<unsigned int*>(&ctl);
        for (int k = threadIdx.x; k < (int)(sizeof(Control) / 4); k += blockDim.x) dst[k] = src[k];
        if (threadIdx.x == 0) {
            s_t0 = A.st->t_start;
            s_mask_base = A.st->mask_cursor;
        }
    }
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_entry = (long long)atomicAdd(A.q_next, 1ull);
        __syncthreads();
        const long long e = s_entry;
        __syncthreads();
        if (e >= A.q_len) break;
        const int k = A.q_chain[e];
        const int m = A.q_member[e];
        const int g = A.g_of[k];
        // Test of the bounded group wait: the last member of a group leaves
        // without arriving, so the others' first wait runs out.
        if (ctl.test_skip_barrier && g > 1 && m == g - 1) continue;
        batch_chain<T, kHasW, kBT>(A, ctl, sm, bc, k, m, g, s_t0, s_mask_base);
    }
}

// Before a persistent batch solve: the solve's start time and every chain
// running (single block).
__global__ void k_bstart(DevState* st) {
    st->t_start = globaltimer();
}

// After it: the batch's totals from the chains (one block, fixed order):
// status = the worst chain's (OK < NOCONV < DEGENERATE < TIMEOUT), moves =
// the most any chain made, edges / green / push / pull / re-derivations
// summed, ||C||_1 and H 1 summed over the chains.
__global__ void __launch_bounds__(kThreads) k_bfinish(DevState* st, const ChainState* cs, int nchains) {
    __shared__ double scratch[32];
    __shared__ int s_worst;
    __shared__ unsigned long long s_moves;
    if (threadIdx.x == 0) {
        s_worst = 0;
        s_moves = 0ull;
    }
    __syncthreads();
    double l1 = 0.0, hs = 0.0, sm = 0.0;
    long long ed = 0, gr = 0, pu = 0, pl = 0, rf = 0, mv = 0;
    for (int k = threadIdx.x; k < nchains; k += blockDim.x) {
        const ChainState& c = cs[k];
        l1 += c.l1;
        hs += c.hsum;
        sm += c.sum;
        ed += c.s_edges;
        gr += c.s_green;
        pu += c.s_push;
        pl += c.s_pull;
        rf += c.s_refr;
        if (c.moves > mv) mv = c.moves;
        atomicMax(&s_worst, status_rank(c.status));
        atomicMax(&s_moves, (unsigned long long)c.s_moves);
    }
    l1 = block_sum(l1, scratch);
    hs = block_sum(hs, scratch);
    sm = block_sum(sm, scratch);
    const double edd = block_sum((double)ed, scratch), grd = block_sum((double)gr, scratch);
    const double pud = block_sum((double)pu, scratch), pld = block_sum((double)pl, scratch);
    const double rfd = block_sum((double)rf, scratch);
    __shared__ unsigned long long s_mv;
    if (threadIdx.x == 0) s_mv = 0ull;
    __syncthreads();
    atomicMax(&s_mv, (unsigned long long)mv);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->l1 = l1;
        st->sum = sm;
        st->hsum = hs;
        st->solve_moves = (long long)s_moves;
        st->iters = (long long)s_moves;
        st->moves = (long long)s_mv;
        st->mask_cursor += (long long)s_moves;
        st->tot_edges += (long long)edd;
        st->tot_green += (long long)grd;
        st->push_moves += (long long)pud;
        st->pull_moves += (long long)pld;
        st->refreshes += (long long)rfd;
        st->mode = MODE_NONE;
        st->status = rank_status(s_worst);
        st->done = 1;
    }
}

// v[k] = row_ptr[node_ptr[k]] for k < m: the links before each chain.
__global__ void k_gather_rows(const long long* __restrict__ row_ptr, const long long* __restrict__ node_ptr,
                              long long m, long long* __restrict__ v) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += (long long)gridDim.x * blockDim.x)
        v[k] = row_ptr[node_ptr[k]];
}

// Per-chain merge-path tiles of kItems items: chain k's ntiles_k + 1 tile
// boundaries, ntiles_k = ceil((n_k + nnz_k) / kItems) (at least 1), laid out
// from ct_off[k]. cnt[k + 1] = ntiles_k + 1 (for the scan that gives ct_off).
__global__ void k_chain_tile_counts(const long long* __restrict__ node_ptr, const long long* __restrict__ t_ptr,
                                    int nchains, long long items, long long* __restrict__ cnt) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nchains; k += gridDim.x * blockDim.x) {
        const long long a = node_ptr[k], b = node_ptr[k + 1];
        const long long tot = (b - a) + (t_ptr[b] - t_ptr[a]);
        long long nt = (tot + items - 1) / items;
        if (nt < 1) nt = 1;
        cnt[k + 1] = nt + 1;
    }
}

// Boundary t of all chains' tile tables: its chain (binary search on
// ct_off), the diagonal d = min(j items, chain items) with j its index in
// the chain's table, split as in k_mp_partition over the chain's rows.
__global__ void k_chain_tiles(const long long* __restrict__ node_ptr, const long long* __restrict__ t_ptr,
                              const long long* __restrict__ ct_off, int nchains, long long items,
                              long long* __restrict__ ct_r, long long* __restrict__ ct_e) {
    const long long total = ct_off[nchains];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = nchains - 1;  // last chain with ct_off <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ct_off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int k = lo;
        const long long a = node_ptr[k], b = node_ptr[k + 1];
        const long long nk = b - a, e_a = t_ptr[a], mk = t_ptr[b] - e_a;
        const long long j = t - ct_off[k];
        const long long d = min(j * items, nk + mk);
        long long l = max(0ll, d - mk), h = min(d, nk);
        while (l < h) {
            const long long mid = (l + h) >> 1;
            if (t_ptr[a + mid + 1] - e_a >= d - mid) h = mid; else l = mid + 1;
        }
        ct_r[t] = a + l;
        ct_e[t] = e_a + (d - l);
    }
}

}  // namespace rlgl
