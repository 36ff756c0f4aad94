// The persistent sweep: the moves of a single-chain solve (the loop of
// Alg. 1 with its stop test) in one cooperative kernel, so that a move
// costs three grid barriers (two with the stale threshold) instead of three
// to four kernel launches, their drain and their serial last-block tails.
//
// Every block runs every phase of a move on its share of the work:
//   stats   : its slice of the nodes; block sums go to one FP64 atomic per
//             statistic in the move's slot;
//   barrier ; every block reads the totals and takes the same decisions
//             (stop, re-derivation, theta) from the same numbers;
//   [top-k] : TOPFRAC only: the radix passes of the exact k-th largest |C|,
//             each a count over the block's nodes and a barrier;
//   select  : its node ranges, staged in shared memory by asynchronous
//             copies (the same compaction as k_select);
//   barrier ; every block reads the frontier size and picks push or pull;
//   push    : its share of the frontier's edge chunks, or
//   pull    : its share of the merge-path tiles;
//   barrier.
// With the stale threshold (Control::theta_lag) a move after the first of a
// launch has no stats phase and no first barrier: its select gathers the
// statistics of the cash it reads, and the next move's threshold and
// decisions come from them, taken while the block waits at the last
// barrier.
// The kernel returns when the solve stops (it then ends the graph's loop) or
// when the FP32 cash of the MIXED path must be re-derived in FP64 (the
// graph's re-derivation runs and the loop launches the sweep again).
//
// Co-residency: the kernel is launched cooperatively with at most as many
// blocks as fit on the GPU at once. Every barrier wait is bounded in time;
// a wait that gives up raises an abort flag on which every block leaves,
// and the solve ends with the status ST_BARRIER.
#pragma once
#include <cstddef>

#include "rlgl_kernels.cuh"

namespace rlgl {

constexpr int kSweepMinBlocks = 4;  // blocks per SM (launch bounds)
constexpr int ST_BARRIER = 9;

// Per-move accumulators, zero at rest. Two slots alternate: the slot of
// move t is cleared by block 0 during move t + 1, after the first barrier,
// when every block has finished reading it.
// Every group of fields that all blocks update or read at one time sits on
// its own 128-byte line, and so does the barrier: the blocks' atomics on one
// line do not queue behind those on another or behind the barrier's polls,
// and the fields read together after a barrier are pairs in 16 bytes (one
// request per pair, the pairs in parallel).
// (An alignment specifier applies to every declarator of its declaration:
// one field per declaration here.)
struct SweepSlot {
    alignas(128) double a;       // ||C||_1 of the cash
    double pr;                   // sum v^r of the cash
    alignas(128) double msum;    // sum m_i of the moved cash
    double mabs;                 // sum |m_i|
    alignas(128) unsigned long long reserve;  // packed frontier reservation
    unsigned long long tstamp;   // block 0's timer at the end of its stats (or select)
    alignas(128) double s;       // sum C
    unsigned long long chunk_next;  // next push chunk (or pull tile) to hand out
    unsigned long long range_next;  // select of large chains: next node range to hand out
};
static_assert(offsetof(SweepSlot, pr) == offsetof(SweepSlot, a) + 8 && offsetof(SweepSlot, a) % 16 == 0,
              "a, pr: one 16-byte pair");
static_assert(offsetof(SweepSlot, mabs) == offsetof(SweepSlot, msum) + 8 && offsetof(SweepSlot, msum) % 16 == 0,
              "msum, mabs: one 16-byte pair");
static_assert(offsetof(SweepSlot, tstamp) == offsetof(SweepSlot, reserve) + 8 &&
                  offsetof(SweepSlot, reserve) % 16 == 0,
              "reserve, tstamp: one 16-byte pair");

struct alignas(128) GridBar {
    unsigned long long arrived;  // arrivals since the solve began (grid size per barrier)
    unsigned int abort;          // a wait gave up: every block leaves
    unsigned int parity;         // slot of the next move (kept across launches)
    unsigned int tk_pass;        // top-k radix passes made so far (kept across launches)
};

// The two 8-byte fields at p (16-byte aligned), read from L2 in one request.
__device__ __forceinline__ double2 ldcg_pair(const void* p) {
    return __ldcg(reinterpret_cast<const double2*>(p));
}

struct SweepState {
    GridBar bar;
    SweepSlot slot[3];  // the general sweep alternates slots 0 and 1; the all-green sweep rotates all three
    // TOPFRAC: the radix passes' digit histograms (zero at rest), three in
    // rotation: pass q adds into q mod 3, every block reads it after the
    // pass's barrier, and block 0 then clears (q + 2) mod 3, which every
    // block read before that barrier and pass q + 2 will fill after the next.
    unsigned int tk_hist[3][kRadixBins];
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: the arrival half of a grid barrier. Makes the block's writes
// visible (fence) and adds one to the arrival count (no value returned);
// target grows by the grid size, the count once every block has arrived.
__device__ __forceinline__ void bar_arrive(GridBar* bar, unsigned long long& target) {
    target += gridDim.x;
    __threadfence();
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], 1;" ::"l"(&bar->arrived) : "memory");
}

// Thread 0: the waiting half of a grid barrier. Polls the arrival count
// until it reaches target, at most limit_ns; a wait that runs out raises the
// abort flag, and a raised flag ends every other wait. Returns 0 when the
// sweep must stop.
__device__ __forceinline__ int bar_wait(GridBar* bar, unsigned long long target,
                                        unsigned long long limit_ns) {
    int ok = 1;
    const unsigned long long t0 = globaltimer();
    unsigned int spins = 0;
    while (ld_acquire_u64(&bar->arrived) < target) {
        if ((++spins & 15u) == 0u) {
            if (ld_acquire_u32(&bar->abort)) {
                ok = 0;
                break;
            }
            if (globaltimer() - t0 > limit_ns) {
                atomicExch(&bar->abort, 1u);
                ok = 0;
                break;
            }
        }
        __nanosleep(32);
    }
    return ok;
}

// Grid-wide barrier of a cooperative launch: the count only grows, so no
// block has to reset or release anything. `target` is the block's expected
// arrival count (kept by thread 0). `work` runs in thread 0 between its
// arrival and its wait (off the critical path unless this block arrives
// last). The wait is bounded by limit_ns; returns false (in every thread of
// the block) when the sweep must stop. When ts is given, thread 0 stores its
// arrival and release times in ts[0], ts[1].
template <typename F>
__device__ __forceinline__ bool grid_barrier_with(GridBar* bar, unsigned long long& target,
                                                  unsigned long long limit_ns, unsigned long long* ts,
                                                  F&& work) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (ts) ts[0] = globaltimer();
        bar_arrive(bar, target);
        work();
        s_ok = bar_wait(bar, target, limit_ns);
        if (ts) ts[1] = globaltimer();
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ bool grid_barrier(GridBar* bar, unsigned long long& target,
                                             unsigned long long limit_ns,
                                             unsigned long long* ts = nullptr) {
    return grid_barrier_with(bar, target, limit_ns, ts, []() {});
}

template <typename T>
struct SweepArgs {
    T* c;
    double* H;
    const double* s;
    const float* sf;
    const long long* row_ptr;
    const T* ideg;
    const unsigned char* masks;
    T* mt;
    T* mt2;      // power sweep: the moved cash of every other move
    T* facc;     // power sweep: sums of rows split across tiles (zero at rest)
    long long* f_eoff;
    long long* f_base;
    T* f_m;
    int* chunk_row;
    const int* col;
    const float* w;
    const long long* t_ptr;
    const int* t_src;
    const float* t_w;
    const long long* tile_r;
    const long long* tile_e;
    long long ntiles;
    const long long* wtile_r;  // power sweep: merge-path tiles of a warp
    const long long* wtile_e;
    long long nwtiles;
    DevState* st;
    SweepState* sw;
    MoveRecord* log;
    unsigned long long cond_loop;
    unsigned long long cond_refresh;
    int use_cond;
    int n;
    int vec_ok;
    const int* hubs;  // hub table of the push (nullptr: none)
};

// Shared cache of the select phase when the chain has at most kIters
// block-iterations (2 for FP32 cash, 1 for FP64, so that a block's static
// shared memory stays within 48 KB): the block's node ranges (contiguous,
// kNodesPerIter nodes each) keep their cash, 1/d, row offsets and test
// results between the counting pass and the writing pass, and every warp's
// green count and edge sum for each of its node groups sits there. The
// arrays are filled by asynchronous 16-byte copies.
constexpr int kSelRp = kNodesPerIter + 2;  // row offsets of a range (+1, padded to 16 bytes)
template <typename T>
struct SelSmem {
    static constexpr int kIters = sizeof(T) == 4 ? 2 : 1;
    static constexpr int kNodes = kIters * kNodesPerIter;
    alignas(16) T val[kNodes];
    alignas(16) T idg[kNodes];
    alignas(16) T sv[kNodes];  // s_i in the cash type (1 / row weight)
    alignas(16) long long rp[kIters][kSelRp];
    unsigned char g[kNodes];
    unsigned long long wsum[kIters * kNodesPerThread * (kThreads / 32)];  // packed (edges << kCountBits) | count
};

// Asynchronous copy of `bytes` (1..16) from global to shared memory, the
// rest of the 16 destination bytes zero-filled; both addresses 16-byte
// aligned. Completed by cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Waits until at most the most recent committed group is in flight.
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// s_i in the cash type: FP32 on the MIXED path, FP64 on the FP64 path.
__device__ __forceinline__ const float* row_scale(const float* sf, const double*, float) { return sf; }
__device__ __forceinline__ const double* row_scale(const float*, const double* s, double) { return s; }

// Warp sum of the packed (edges << kCountBits) | count of the green lanes:
// the count from the ballot, the edges from two 32-bit warp reductions of
// the degree's 16-bit halves (no overflow for any int32 degrees).
__device__ __forceinline__ unsigned long long warp_pack_sum(bool g, int rdeg) {
    const unsigned int cnt = __popc(__ballot_sync(0xffffffffu, g));
    const unsigned int lo = __reduce_add_sync(0xffffffffu, g ? ((unsigned int)rdeg & 0xffffu) : 0u);
    const unsigned int hi = __reduce_add_sync(0xffffffffu, g ? ((unsigned int)rdeg >> 16) : 0u);
    return ((((unsigned long long)hi << 16) + lo) << kCountBits) + cnt;
}

// Exclusive prefix over the warp's lanes of x >= 0 (x < 2^31).
__device__ __forceinline__ long long warp_exscan_deg(int x) {
    const int lane = threadIdx.x & 31;
    if (__all_sync(0xffffffffu, x < (1 << 26))) {
        // 32 x 2^26 = 2^31: the sums fit 32 bits
        int y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        return (long long)(y - x);
    }
    long long y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long z = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += z;
    }
    return y - x;
}

// Copies elements [e0, e0 + count) of src (count elements of type E in
// 16-byte pieces; the array holds `avail` elements from index 0) into dst,
// zero past the array's end. Every thread of the block takes pieces.
template <typename E>
__device__ __forceinline__ void stage_range(E* dst, const E* src, long long e0, int count, long long avail) {
    constexpr int kPer = 16 / (int)sizeof(E);
    const int pieces = (count + kPer - 1) / kPer;
    for (int u = threadIdx.x; u < pieces; u += blockDim.x) {
        const long long e = e0 + (long long)u * kPer;
        const long long left = (avail - e) * (long long)sizeof(E);
        E* d = dst + u * kPer;
        if (left >= 16) cp_async16(d, src + e, 16);
        else if (left > 0) cp_async16(d, src + e, (int)left);
        else *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Select on this block's node slices (the single-chain form of k_select):
// green nodes give their cash (m_i = C_i, C_i <- 0, H_i += m_i) and get
// frontier entries and push-chunk starts; mt holds m~_i (0 for red nodes).
// Two passes over the block's nodes: the first counts green nodes and their
// edges, one atomic per block reserves the block's frontier range, the
// second writes it. For the first two block-iterations (cached in shared
// memory) the frontier slots follow node order within each warp, so a
// warp's frontier writes are contiguous; beyond, each thread's green nodes
// take consecutive slots. Returns the block's sums of m_i and |m_i| in
// thread 0. With acc_stats (the stale threshold), also the block's sums of
// the statistics of the cash before the move, from the same loads:
// ba = sum |C_i| and bpr = sum v_i^r as the statistics pass forms them
// (v_i = |C_i| / d_i when link, else |C_i|; bpr stays 0 for r = 1 without
// link, whose sum is ba).
// x^r for the rare exponents r > 2, out of line so that the select loop
// does not carry pow's registers.
template <typename T>
__device__ __noinline__ T pow_r(T x, int r) {
    return pow(x, (T)r);
}

template <typename T>
__device__ __forceinline__ void sweep_select(const SweepArgs<T>& A, int sched, T th,
                                             const unsigned char* mask, const SchedAux& ax,
                                             SweepSlot* sl, SelSmem<T>& cs, bool acc_stats,
                                             bool link, int r, double& bmsum, double& bmabs,
                                             double& ba, double& bpr) {
    __shared__ T tscratch[4 * 32];
    __shared__ unsigned long long base_sh;
    // rows with many push chunks: their chunk starts are written by the
    // whole block after the second pass instead of by one thread
    constexpr int kLongRows = 16;
    constexpr int kLongChunks = 8;
    __shared__ int s_nlong;
    __shared__ long long s_long[kLongRows][3];  // frontier row, first chunk, end chunk
    const int n = A.n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T msum = T(0), mabs = T(0), sa = T(0), spr = T(0);
    // the statistics pass's terms (stats_slice)
    auto stat = [&](T v, T idg) {
        const T av = fabs(v);
        sa += av;
        const T tv = link ? av * idg : av;
        if (link && r == 1) spr += tv;
        else if (r == 2) spr += tv * tv;
        else if (r > 2) spr += pow_r(tv, r);
    };
    auto finish = [&]() {
        T v4[4] = {msum, mabs, sa, spr};
        block_sum_n<T, 4>(v4, tscratch);
        bmsum = (double)v4[0];
        bmabs = (double)v4[1];
        ba = (double)v4[2];
        bpr = (double)v4[3];
    };
    if (sched == SCHED_ALL_GREEN) {
        // every node moves; the pull needs no frontier
        for (long long it0 = (long long)blockIdx.x * kNodesPerIter; it0 < n;
             it0 += (long long)gridDim.x * kNodesPerIter) {
            // every load of the range first: red_add orders later loads after it
            T val[kNodesPerThread], idg[kNodesPerThread], scv[kNodesPerThread];
#pragma unroll
            for (int q = 0; q < kNodesPerThread; ++q) {
                const long long i = it0 + q * kThreads + threadIdx.x;
                val[q] = i < n ? __ldcg(A.c + i) : T(0);
                idg[q] = (i < n && link) ? __ldg(A.ideg + i) : T(0);
                scv[q] = i < n ? moved_per_weight(T(1), A.s, A.sf, i) : T(0);
            }
#pragma unroll
            for (int q = 0; q < kNodesPerThread; ++q) {
                const long long i = it0 + q * kThreads + threadIdx.x;
                if (i >= n) continue;
                const T v = val[q];
                if (acc_stats) stat(v, idg[q]);
                A.c[i] = T(0);
                red_add(A.H + i, (double)v);  // no load: the L2 adds
                msum += v;
                mabs += fabs(v);
                A.mt[i] = v * scv[q];
            }
        }
        finish();
        return;
    }
    if ((long long)n > (long long)gridDim.x * SelSmem<T>::kNodes && SelSmem<T>::kIters >= 2) {
        // Large chains, FP32 cash: node ranges of kNodesPerIter one after
        // another through the two stages of the shared cache, the next
        // range's asynchronous copies in flight while this one is tested,
        // reserved and written. One reservation per range: a count pass over
        // all of them first would read the nodes from memory twice. Block b
        // takes ranges b and b + G, then grabs the next free range from a
        // counter (the grab issued a range ahead), so that blocks end within
        // a fraction of a range of one another.
        const bool with_idg = sched == SCHED_LINK;
        // unweighted chains: s_i = 1/d_i, bit for bit the staged 1/d
        const bool scale_is_idg = with_idg && A.w == nullptr;
        const T* scale = scale_is_idg ? cs.idg : cs.sv;
        const long long G = gridDim.x;
        const long long nranges = ((long long)n + kNodesPerIter - 1) / kNodesPerIter;
        __shared__ long long s_grab[2];
        auto stage = [&](int buf, long long r) {
            const long long it0 = r * kNodesPerIter;
            stage_range<T>(cs.val + buf * kNodesPerIter, A.c, it0, kNodesPerIter, n);
            if (with_idg) stage_range<T>(cs.idg + buf * kNodesPerIter, A.ideg, it0, kNodesPerIter, n);
            if (!scale_is_idg)
                stage_range<T>(cs.sv + buf * kNodesPerIter, row_scale(A.sf, A.s, T(0)), it0, kNodesPerIter, n);
            stage_range<long long>(cs.rp[buf], A.row_ptr, it0, kSelRp, (long long)n + 1);
            cp_async_commit();
        };
        // n > G x kNodes: ranges b and b + G exist for every block
        long long cur = blockIdx.x, nxt = blockIdx.x + G;
        stage(0, cur);
        stage(1, nxt);
        for (int j = 0;; ++j) {
            const int buf = j & 1;
            const long long it0 = cur * kNodesPerIter;
            // the range after next, staged at the end of this iteration: the
            // grab's reply is first used there, so its round trip overlaps
            // this range's work
            unsigned long long grab = 0ull;
            if (threadIdx.x == 0 && nxt >= 0) grab = atomicAdd(&sl->range_next, 1ull);
            if (nxt >= 0) cp_async_wait_prev();
            else cp_async_wait_all();
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kNodesPerThread; ++q) {
                const int loc = q * kThreads + threadIdx.x;
                const int slot = buf * kNodesPerIter + loc;
                const long long i = it0 + loc;
                const T v = cs.val[slot];
                const T idg = with_idg ? cs.idg[slot] : T(0);
                const int rdeg = (int)(cs.rp[buf][loc + 1] - cs.rp[buf][loc]);
                const bool g = (i < n) && green_test_v<T>(sched, v, idg, i, th, mask, ax);
                if (acc_stats && i < n) stat(v, idg);
                cs.g[slot] = g ? 1 : 0;
                const unsigned long long w = warp_pack_sum(g, rdeg);
                if (lane == 0) cs.wsum[q * (kThreads / 32) + wid] = w;
            }
            __syncthreads();
            if (wid == 0) {
                // kNodesPerThread x warps = 32 groups: one warp-wide scan
                const unsigned long long v = cs.wsum[lane];
                unsigned long long x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                cs.wsum[lane] = x - v;
                const unsigned long long run = __shfl_sync(0xffffffffu, x, 31);
                if (lane == 0) {
                    base_sh = run ? atomicAdd(&sl->reserve, run) : 0ull;
                    s_nlong = 0;
                }
            }
            __syncthreads();
            const unsigned long long base = base_sh;
#pragma unroll
            for (int q = 0; q < kNodesPerThread; ++q) {
                const int loc = q * kThreads + threadIdx.x;
                const int slot = buf * kNodesPerIter + loc;
                const long long i = it0 + loc;
                const T v = cs.val[slot];
                const long long rb = cs.rp[buf][loc];
                const int rdeg = (int)(cs.rp[buf][loc + 1] - rb);
                const bool g = cs.g[slot] != 0;
                const unsigned int bal = __ballot_sync(0xffffffffu, g);
                if (bal == 0u) {  // no green node in this warp's group
                    if (i < n) A.mt[i] = T(0);
                    continue;
                }
                const long long xe = warp_exscan_deg(g ? rdeg : 0);
                const unsigned long long wb = base + cs.wsum[q * (kThreads / 32) + wid];
                const long long kk = (long long)(wb & ((1ull << kCountBits) - 1ull)) + __popc(bal & ((1u << lane) - 1u));
                const long long ee = (long long)(wb >> kCountBits) + xe;
                if (i >= n) continue;
                if (g) {
                    const T mtil = v * scale[slot];
                    A.c[i] = T(0);
                    red_add(A.H + i, (double)v);  // no load: the L2 adds
                    msum += v;
                    mabs += fabs(v);
                    A.mt[i] = mtil;
                    A.f_eoff[kk] = ee;
                    A.f_base[kk] = rb - ee;
                    A.f_m[kk] = mtil;
                    const long long b0 = (ee + kPushChunk - 1) / kPushChunk;
                    const long long b1 = (ee + rdeg + kPushChunk - 1) / kPushChunk;
                    int ls = -1;
                    if (b1 - b0 > kLongChunks) {
                        ls = atomicAdd(&s_nlong, 1);
                        if (ls < kLongRows) {
                            s_long[ls][0] = kk;
                            s_long[ls][1] = b0;
                            s_long[ls][2] = b1;
                        }
                    }
                    if (ls < 0 || ls >= kLongRows)
                        for (long long b = b0; b < b1; ++b) A.chunk_row[b] = (int)kk;
                } else {
                    A.mt[i] = T(0);
                }
            }
            if (threadIdx.x == 0 && nxt >= 0) s_grab[buf] = 2 * G + (long long)grab;
            __syncthreads();
            // this stage is free: the range after next goes into it
            long long after = nxt >= 0 ? s_grab[buf] : -1;
            if (after >= nranges) after = -1;
            if (after >= 0) stage(buf, after);
            const int nlong = s_nlong < kLongRows ? s_nlong : kLongRows;
            for (int q = 0; q < nlong; ++q)
                for (long long b = s_long[q][1] + threadIdx.x; b < s_long[q][2]; b += blockDim.x)
                    A.chunk_row[b] = (int)s_long[q][0];
            cur = nxt;
            nxt = after;
            if (cur < 0) break;
        }
        finish();
        return;
    }
    if ((long long)n > (long long)gridDim.x * SelSmem<T>::kNodes) {
        // Large chains, FP64 cash (more block-iterations than the cache holds): one pass
        // with one reservation per block-iteration, so that the nodes are
        // read once (a second pass would read them again from memory).
        for (long long it0 = (long long)blockIdx.x * kNodesPerIter; it0 < n;
             it0 += (long long)gridDim.x * kNodesPerIter) {
            long long rb[kNodesPerThread];
            int rdeg[kNodesPerThread];
            T val[kNodesPerThread], idg[kNodesPerThread], scv[kNodesPerThread];
            bool g[kNodesPerThread];
#pragma unroll
            for (int q = 0; q < kNodesPerThread; ++q) {
                const long long i = it0 + q * kThreads + threadIdx.x;
                rb[q] = (i < n) ? __ldg(A.row_ptr + i) : 0;
                rdeg[q] = (i < n) ? (int)(__ldg(A.row_ptr + i + 1) - rb[q]) : 0;
                val[q] = (i < n) ? __ldcg(A.c + i) : T(0);
                idg[q] = (i < n && sched == SCHED_LINK) ? __ldg(A.ideg + i) : T(0);
                // s_i now: red_add below orders every later load after it
                scv[q] = (i < n) ? moved_per_weight(T(1), A.s, A.sf, i) : T(0);
            }
            unsigned long long mine = 0ull;
#pragma unroll
            for (int q = 0; q < kNodesPerThread; ++q) {
                const long long i = it0 + q * kThreads + threadIdx.x;
                g[q] = (i < n) && green_test_v<T>(sched, val[q], idg[q], i, th, mask, ax);
                if (g[q]) mine += ((unsigned long long)rdeg[q] << kCountBits) + 1ull;
                if (acc_stats && i < n) stat(val[q], idg[q]);
            }
            unsigned long long total;
            const unsigned long long pre = block_exscan(mine, &total);
            if (threadIdx.x == 0) base_sh = total ? atomicAdd(&sl->reserve, total) : 0ull;
            __syncthreads();
            const unsigned long long base = base_sh + pre;
            long long k = (long long)(base & ((1ull << kCountBits) - 1ull));
            long long e = (long long)(base >> kCountBits);
#pragma unroll
            for (int q = 0; q < kNodesPerThread; ++q) {
                const long long i = it0 + q * kThreads + threadIdx.x;
                if (i >= n) continue;
                if (g[q]) {
                    const T v = val[q];
                    const T mtil = v * scv[q];
                    A.c[i] = T(0);
                    red_add(A.H + i, (double)v);  // no load: the L2 adds
                    msum += v;
                    mabs += fabs(v);
                    A.mt[i] = mtil;
                    A.f_eoff[k] = e;
                    A.f_base[k] = rb[q] - e;
                    A.f_m[k] = mtil;
                    const long long b0 = (e + kPushChunk - 1) / kPushChunk;
                    const long long b1 = (e + rdeg[q] + kPushChunk - 1) / kPushChunk;
                    for (long long b = b0; b < b1; ++b) A.chunk_row[b] = (int)k;
                    ++k;
                    e += rdeg[q];
                } else {
                    A.mt[i] = T(0);
                }
            }
            __syncthreads();  // base_sh is rewritten by the next iteration
        }
        finish();
        return;
    }
    // Cached path (n <= grid x kNodes): at most kIters ranges.
    // Pass 1 stages every range's cash, 1/d and row offsets in shared
    // memory at once (one round trip, no registers held), then tests and
    // counts from there, per warp and node group.
    const bool with_idg = sched == SCHED_LINK;
    const bool scale_is_idg = with_idg && A.w == nullptr;  // s_i = 1/d_i
    const T* scale = scale_is_idg ? cs.idg : cs.sv;
    int nj = 0;
    for (int j = 0; j < SelSmem<T>::kIters; ++j) {
        const long long it0 = ((long long)blockIdx.x + (long long)j * gridDim.x) * kNodesPerIter;
        if (it0 >= n) break;
        ++nj;
        stage_range<T>(cs.val + j * kNodesPerIter, A.c, it0, kNodesPerIter, n);
        if (with_idg) stage_range<T>(cs.idg + j * kNodesPerIter, A.ideg, it0, kNodesPerIter, n);
        if (!scale_is_idg)
            stage_range<T>(cs.sv + j * kNodesPerIter, row_scale(A.sf, A.s, T(0)), it0, kNodesPerIter, n);
        stage_range<long long>(cs.rp[j], A.row_ptr, it0, kSelRp, (long long)n + 1);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int j = 0; j < nj; ++j) {
        const long long it0 = ((long long)blockIdx.x + (long long)j * gridDim.x) * kNodesPerIter;
#pragma unroll
        for (int q = 0; q < kNodesPerThread; ++q) {
            const int loc = q * kThreads + threadIdx.x;
            const int slot = j * kNodesPerIter + loc;
            const long long i = it0 + loc;
            const T v = cs.val[slot];
            const T idg = with_idg ? cs.idg[slot] : T(0);
            const int rdeg = (int)(cs.rp[j][loc + 1] - cs.rp[j][loc]);
            const bool g = (i < n) && green_test_v<T>(sched, v, idg, i, th, mask, ax);
            if (acc_stats && i < n) stat(v, idg);
            cs.g[slot] = g ? 1 : 0;
            const unsigned long long w = warp_pack_sum(g, rdeg);
            if (lane == 0) cs.wsum[(j * kNodesPerThread + q) * (kThreads / 32) + wid] = w;
        }
    }
    const int ncached = nj * kNodesPerThread * (kThreads / 32);
    __syncthreads();
    // exclusive prefix of the groups' counts in group order, and one
    // reservation for the whole block (warp 0)
    if (wid == 0) {
        unsigned long long run = 0ull;
        for (int g0 = 0; g0 < ncached; g0 += 32) {
            const int gi = g0 + lane;
            const unsigned long long v = gi < ncached ? cs.wsum[gi] : 0ull;
            unsigned long long x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (gi < ncached) cs.wsum[gi] = run + x - v;
            run += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) {
            base_sh = run ? atomicAdd(&sl->reserve, run) : 0ull;
            s_nlong = 0;
        }
    }
    __syncthreads();
    const unsigned long long base = base_sh;
    // pass 2: write (frontier slots in node order within each warp)
    for (int j = 0; j < nj; ++j) {
        const long long it0 = ((long long)blockIdx.x + (long long)j * gridDim.x) * kNodesPerIter;
#pragma unroll
        for (int q = 0; q < kNodesPerThread; ++q) {
            const int loc = q * kThreads + threadIdx.x;
            const int slot = j * kNodesPerIter + loc;
            const long long i = it0 + loc;
            const T v = cs.val[slot];
            const long long rb = cs.rp[j][loc];
            const int rdeg = (int)(cs.rp[j][loc + 1] - rb);
            const bool g = cs.g[slot] != 0;
            const unsigned int bal = __ballot_sync(0xffffffffu, g);
            if (bal == 0u) {  // no green node in this warp's group
                if (i < n) A.mt[i] = T(0);
                continue;
            }
            const long long xe = warp_exscan_deg(g ? rdeg : 0);
            const unsigned long long wb = base + cs.wsum[(j * kNodesPerThread + q) * (kThreads / 32) + wid];
            const long long kk = (long long)(wb & ((1ull << kCountBits) - 1ull)) + __popc(bal & ((1u << lane) - 1u));
            const long long ee = (long long)(wb >> kCountBits) + xe;
            if (i >= n) continue;
            if (g) {
                const T mtil = v * scale[slot];
                A.c[i] = T(0);
                red_add(A.H + i, (double)v);  // no load: the L2 adds
                msum += v;
                mabs += fabs(v);
                A.mt[i] = mtil;
                A.f_eoff[kk] = ee;
                A.f_base[kk] = rb - ee;
                A.f_m[kk] = mtil;
                const long long b0 = (ee + kPushChunk - 1) / kPushChunk;
                const long long b1 = (ee + rdeg + kPushChunk - 1) / kPushChunk;
                int ls = -1;
                if (b1 - b0 > kLongChunks) {
                    ls = atomicAdd(&s_nlong, 1);
                    if (ls < kLongRows) {
                        s_long[ls][0] = kk;
                        s_long[ls][1] = b0;
                        s_long[ls][2] = b1;
                    }
                }
                if (ls < 0 || ls >= kLongRows)
                    for (long long b = b0; b < b1; ++b) A.chunk_row[b] = (int)kk;
            } else {
                A.mt[i] = T(0);
            }
        }
    }
    __syncthreads();
    const int nlong = s_nlong < kLongRows ? s_nlong : kLongRows;
    for (int q = 0; q < nlong; ++q)
        for (long long b = s_long[q][1] + threadIdx.x; b < s_long[q][2]; b += blockDim.x)
            A.chunk_row[b] = (int)s_long[q][0];
    finish();
}

template <typename T>
union SweepSmem {
    PushSmem<T> push;
    PullSmem<T> pull;
    SelSmem<T> sel;
    unsigned int hist[kRadixBins];  // TOPFRAC: the block's digit histogram
};

// TOPFRAC inside the sweep: one pass of the exact k-th largest |C| by radix
// select over the IEEE bit patterns of |C| (the phase form is k_radix_pass).
// The block counts the digit at `shift` (`width` bits) of the keys that
// match `prefix` above it, over its grid-stride share of the nodes (equal
// digits of a warp merged with __match_any_sync, one shared-memory add per
// distinct digit), and adds its nonzero counts to the pass's histogram.
template <typename T>
__device__ __forceinline__ void sweep_radix_count(const T* c, int n, unsigned int* ghist, unsigned long long prefix,
                                                  int shift, int width, unsigned int* h) {
    const int nbins = 1 << width;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const int hi_shift = shift + width;
    const unsigned long long mask = (unsigned long long)(nbins - 1);
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const long long i = base + lane;
        int digit = -1;
        if (i < n) {
            // the cash other blocks moved last move: from L2
            const unsigned long long k = (unsigned long long)KeyOf<T>::key(__ldcg(c + i));
            const bool match = (hi_shift >= KeyOf<T>::bits) || ((k >> hi_shift) == (prefix >> hi_shift));
            if (match) digit = (int)((k >> shift) & mask);
        }
        const unsigned int peers = __match_any_sync(0xffffffffu, digit);
        if (digit >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[digit], (unsigned int)__popc(peers));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (h[b]) atomicAdd(&ghist[b], h[b]);
}

// After the pass's barrier: the bucket of the remaining k-th largest key,
// the same in every block (the same counts, the same scan). Thread t owns 8
// bins counted from the top; thread 0 gets the new prefix and remainder.
__device__ __forceinline__ void sweep_radix_pick(const unsigned int* ghist, int shift, int width,
                                                 unsigned long long& prefix, long long& remain) {
    __shared__ int found;
    __shared__ long long above_found;
    if (threadIdx.x == 0) found = -1;
    constexpr int per = kRadixBins / kThreads;  // 8
    const int nbins = 1 << width;
    const int top = nbins - 1 - (int)threadIdx.x * per;
    unsigned long long mine = 0;
    unsigned int hb[per];
#pragma unroll
    for (int q = 0; q < per; ++q) {
        const int b = top - q;
        hb[q] = (b >= 0) ? __ldcg(&ghist[b]) : 0u;
        mine += hb[q];
    }
    unsigned long long total;
    const unsigned long long above = block_exscan(mine, &total);
    const long long rem = remain;
    if ((long long)above < rem && (long long)(above + mine) >= rem) {
        long long cum = (long long)above;
#pragma unroll
        for (int q = 0; q < per; ++q) {
            const int b = top - q;
            if (b >= 0 && cum + (long long)hb[q] >= rem) {
                found = b;
                above_found = cum;
                break;
            }
            cum += hb[q];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int digit = found >= 0 ? found : 0;
        const long long cum = found >= 0 ? above_found : 0;
        prefix |= (unsigned long long)digit << shift;
        remain = rem - cum;
    }
}

// The evolving scalars of the solve, one copy per block in shared memory,
// kept by the block's thread 0. Every block's copy goes through the same
// updates from the same values read after the barriers, so all copies stay
// identical and every block takes the same decisions.
struct SweepCtl {
    long long moves, solve_moves, iters, mask_cursor;
    long long tot_green, tot_edges, push_moves, pull_moves;
    long long green, edges;
    double hsum, habs, theta, l1;
    double stall_mark;
    long long stall_count;
    unsigned long long t_start;
    float theta_f;
    int fresh, sched, mode;
    int leave;         // 1: return now (stop, or re-derive before testing again)
    int want_refresh;  // return after this move for a re-derivation
    int p;             // slot parity
    unsigned long long target;  // expected arrival count at the next barrier
    unsigned long long ts[7];  // block 0: move start, then arrival / release at each barrier
    SchedAux ax;       // this move's block-round-robin range and PC constants
    long long mask_off;  // MASK: offset of this move's mask
    // stale threshold: the statistics of the cash before the last move
    double lag_l1, lag_sumr;
    unsigned long long lag_now;  // block 0's timer when they were taken
    int have_lag;      // a move of this launch has set them
    int stop_after;    // status to stop with after this move (-1: none)
    int lag_stop;      // stale threshold: the next move's stop before it selects (-1: none)
    int pre_done;      // the next move's decisions are taken (sweep_lag_control)
    // TOPFRAC: this move's radix select
    unsigned long long tk_prefix;
    long long tk_remain;
    unsigned int tk_pass;  // passes made by the solve so far (histogram rotation)
};

// This move's schedule, threshold and schedule constants from the
// statistics l1 = ||C||_1 and sumr = sum v^r (thread 0; the same in every
// block).
__device__ __forceinline__ void sweep_theta(SweepCtl& sc, const Control& ctl, int n, double l1, double sumr) {
    const int r = ctl.r;
    int sched = ctl.sched;
    if (ctl.safety_every > 0 && ((sc.solve_moves + 1) % ctl.safety_every) == 0) sched = SCHED_ALL_GREEN;
    double theta = 0.0;
    if (sched == SCHED_THRESHOLD || sched == SCHED_LINK) {
        const double mean = sumr / (double)n;
        theta = ctl.theta_arg > 0.0 ? ctl.theta_arg
                                    : (r == 1 ? ctl.theta_scale * mean : ctl.theta_scale * pow(mean, 1.0 / r));
    }
    sc.sched = sched;
    sc.theta = theta;
    sc.ax = sched_aux(ctl, n, sc.moves, l1, sched);
    sc.mask_off = (sched == SCHED_MASK) ? (sc.mask_cursor % ctl.n_masks) * (long long)n : 0;
    sc.theta_f = (sched == SCHED_LINK) ? __double2float_rn(theta) : __double2float_ru(theta);
}

// The decisions of a move of the stale threshold that need no new
// statistics (thread 0): degenerate history, max_steps, time; the threshold
// from the statistics of the cash before the previous move. Every input is
// known once the previous move has read its totals, so this runs while the
// block waits at that move's last barrier.
__device__ __forceinline__ void sweep_lag_control(SweepCtl& sc, const Control& ctl, int n) {
    sc.iters++;
    int stop = -1;
    const bool degenerate = !(fabs(sc.hsum) > 1e-12 * sc.habs) || sc.habs == 0.0;
    if (degenerate) stop = ST_DEGENERATE;
    else if (sc.solve_moves >= ctl.max_steps) stop = ST_NOCONV;
    else if ((double)(sc.lag_now - sc.t_start) > ctl.time_limit_ns || sc.iters > ctl.max_iters)
        stop = ST_TIMEOUT;
    sc.lag_stop = stop;
    sc.leave = stop >= 0 ? 1 : 0;
    sc.want_refresh = 0;
    sweep_theta(sc, ctl, n, sc.lag_l1, sc.lag_sumr);
    sc.pre_done = 1;
}

__device__ __forceinline__ void clear_slot(SweepSlot* o) {
    o->a = 0.0;
    o->s = 0.0;
    o->pr = 0.0;
    o->msum = 0.0;
    o->mabs = 0.0;
    o->reserve = 0ull;
    o->chunk_next = 0ull;
    o->range_next = 0ull;
}

template <typename T, bool kHasW>
__global__ void __launch_bounds__(kThreads, kSweepMinBlocks) k_sweep(SweepArgs<T> A) {
    DevState* st = A.st;
    SweepState* sw = A.sw;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (st->done) {
        if (A.use_cond && lead) cudaGraphSetConditional(A.cond_loop, 0u);
        return;
    }
    __shared__ SweepSmem<T> sm;
    __shared__ T tscratch[32];
    __shared__ SweepCtl sc;
    // The solve's parameters, copied once: after every barrier a global read
    // would go to L2 again (and 600 blocks would queue on the same lines).
    __shared__ Control ctl;
    __shared__ double s_l1_refresh;
    {
        const unsigned int* src = reinterpret_cast<const unsigned int*>(&st->ctl);
        unsigned int* dst = reinterpret_cast<unsigned int*>(&ctl);
        for (int k = threadIdx.x; k < (int)(sizeof(Control) / 4); k += blockDim.x) dst[k] = src[k];
        if (threadIdx.x == 0) s_l1_refresh = st->l1_refresh;
    }
    const int n = A.n;
    constexpr bool kF32 = std::is_same<T, float>::value;
    if (threadIdx.x == 0) {
        sc.moves = st->moves;
        sc.solve_moves = st->solve_moves;
        sc.iters = st->iters;
        sc.mask_cursor = st->mask_cursor;
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
        // Every barrier adds exactly the grid size, and no barrier can
        // complete before this block arrives: rounding down what has arrived
        // gives the count at the start of this launch.
        const unsigned long long arr = ld_acquire_u64(&sw->bar.arrived);
        sc.target = arr - arr % gridDim.x;
        sc.p = (int)(sw->bar.parity & 1u);
        sc.tk_pass = sw->bar.tk_pass;
        sc.have_lag = 0;
        sc.stop_after = -1;
        sc.pre_done = 0;
    }
    __syncthreads();
    // Test of the bounded wait: the last block leaves without arriving, so
    // the others' first barrier wait runs out.
    if (ctl.test_skip_barrier && blockIdx.x == gridDim.x - 1 && gridDim.x > 1) return;

    for (;;) {
        SweepSlot* sl = &sw->slot[sc.p];
        if (lead) sc.ts[0] = globaltimer();
        // A move of the stale threshold (after the first of the launch)
        // skips the statistics pass and its barrier: its select takes the
        // statistics of the cash before the previous move and gathers its
        // own cash's for the stop test.
        const bool lagged = ctl.theta_lag && sc.have_lag;
        if (!lagged) {
        // ---------------------------------------------------------- stats
        {
            const bool link = ctl.sched == SCHED_LINK;
            T a = T(0), s = T(0), pr = T(0);
            stats_slice<T, true>(A.c, A.ideg, n, link, ctl.r, A.vec_ok,
                                 blockIdx.x * (long long)blockDim.x + threadIdx.x,
                                 (long long)gridDim.x * blockDim.x, a, s, pr);
            const T ba = block_sum(a, tscratch);
            const T bs = block_sum(s, tscratch);
            const T bp = block_sum(pr, tscratch);
            if (threadIdx.x == 0) {
                if (ba != T(0)) atomicAdd(&sl->a, (double)ba);
                if (bs != T(0)) atomicAdd(&sl->s, (double)bs);
                if (bp != T(0)) atomicAdd(&sl->pr, (double)bp);
                if (blockIdx.x == 0) sl->tstamp = globaltimer();
            }
        }
        if (!grid_barrier(&sw->bar, sc.target, ctl.barrier_limit_ns, blockIdx.x == 0 ? sc.ts + 1 : nullptr)) break;

        // -------------------------------------------------------- control
        if (threadIdx.x == 0) {
            if (blockIdx.x == 0) clear_slot(&sw->slot[sc.p ^ 1]);
            const int r = ctl.r;
            const bool link = ctl.sched == SCHED_LINK;
            const double2 apr = ldcg_pair(&sl->a);
            const double2 rts = ldcg_pair(&sl->reserve);
            const double sum = __ldcg(&sl->s);
            const double l1 = apr.x;
            const double sumr = (r == 1 && !link) ? l1 : apr.y;
            sc.l1 = l1;
            const unsigned long long now = (unsigned long long)__double_as_longlong(rts.y);
            if (sc.iters == 0) sc.t_start = now;
            sc.iters++;
            int stop = -1;
            bool skip = false, want_refresh = false;
            const bool degenerate = !(fabs(sc.hsum) > 1e-12 * sc.habs) || sc.habs == 0.0;
            const bool converged = sc.moves >= 1 && l1 / fabs(sc.hsum) < ctl.tol;
            if (degenerate) {
                stop = ST_DEGENERATE;
            } else if (converged) {
                if (ctl.mixed && !sc.fresh) {
                    want_refresh = true;  // re-derive, then test again
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
            sc.leave = (stop >= 0 || skip) ? 1 : 0;
            sc.want_refresh = want_refresh ? 1 : 0;
            sweep_theta(sc, ctl, n, l1, sumr);
            // the next move of the stale threshold takes these statistics
            sc.lag_l1 = l1;
            sc.lag_sumr = sumr;
            sc.lag_now = now;
            if (blockIdx.x == 0) {
                st->l1 = l1;
                st->sum = sum;
                st->sumr = sumr;
                st->iters = sc.iters;
                st->t_start = sc.t_start;
                st->stall_mark = sc.stall_mark;
                st->stall_count = sc.stall_count;
                if (sc.leave) {
                    st->mode = MODE_NONE;
                    sw->bar.parity = (unsigned int)(sc.p ^ 1);
                    sw->bar.tk_pass = sc.tk_pass;
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
                }
            }
        }
        __syncthreads();
        if (sc.leave) return;
        } else {
        // ------------------------------------- control (stale threshold)
        // the tests that need no new statistics, the threshold from the
        // previous move's
        if (lead) sc.ts[1] = sc.ts[2] = sc.ts[0];
        if (threadIdx.x == 0) {
            if (!sc.pre_done) sweep_lag_control(sc, ctl, n);
            sc.pre_done = 0;
            const int stop = sc.lag_stop;
            if (blockIdx.x == 0 && stop >= 0) {
                // this move's slot is still clear: the next launch may take it
                st->iters = sc.iters;
                st->mode = MODE_NONE;
                sw->bar.parity = (unsigned int)sc.p;
                sw->bar.tk_pass = sc.tk_pass;
                st->done = 1;
                st->status = stop;
                if (A.use_cond) {
                    cudaGraphSetConditional(A.cond_loop, 0u);
                    if (ctl.mixed) cudaGraphSetConditional(A.cond_refresh, 0u);
                }
            }
        }
        __syncthreads();
        if (sc.leave) return;
        }

        // ------------------------------------------------ top-k threshold
        // TOPFRAC: theta = the exact k-th largest |C| (k = ceil(f N)), one
        // radix pass and one grid barrier per digit
        if (sc.sched == SCHED_TOPFRAC) {
            if (threadIdx.x == 0) {
                const double f = (ctl.theta_arg > 0.0 && ctl.theta_arg <= 1.0) ? ctl.theta_arg : ctl.top_frac;
                long long k = (long long)ceil(f * (double)n);
                if (k < 1) k = 1;
                if (k > n) k = n;
                sc.tk_prefix = 0ull;
                sc.tk_remain = k;
            }
            __syncthreads();
            bool bar_ok = true;
            for (int hi = KeyOf<T>::bits; hi > 0; hi -= kRadixBits) {
                const int width = hi >= kRadixBits ? kRadixBits : hi;
                const int shift = hi - width;
                const unsigned int q = sc.tk_pass;
                sweep_radix_count<T>(A.c, n, sw->tk_hist[q % 3u], sc.tk_prefix, shift, width, sm.hist);
                if (!(bar_ok = grid_barrier(&sw->bar, sc.target, ctl.barrier_limit_ns))) break;
                if (blockIdx.x == 0) {
                    unsigned int* old = sw->tk_hist[(q + 2u) % 3u];
                    for (int b = threadIdx.x; b < kRadixBins; b += blockDim.x) old[b] = 0u;
                }
                sweep_radix_pick(sw->tk_hist[q % 3u], shift, width, sc.tk_prefix, sc.tk_remain);
                if (threadIdx.x == 0) sc.tk_pass = q + 1u;
                __syncthreads();
            }
            if (!bar_ok) break;
            if (threadIdx.x == 0) {
                sc.theta = KeyOf<T>::value(sc.tk_prefix);
                sc.theta_f = __double2float_ru(sc.theta);
            }
            __syncthreads();
        }

        // --------------------------------------------------------- select
        {
            const int sched = sc.sched;
            const T th = kF32 ? (T)sc.theta_f : (T)sc.theta;
            const unsigned char* mask = (sched == SCHED_MASK) ? A.masks + sc.mask_off : nullptr;
            const SchedAux& ax = sc.ax;
            double bmsum, bmabs, ba, bpr;
            const bool link = ctl.sched == SCHED_LINK;
            sweep_select<T>(A, sched, th, mask, ax, sl, sm.sel, lagged, link, ctl.r, bmsum, bmabs, ba, bpr);
            if (threadIdx.x == 0) {
                if (bmsum != 0.0) atomicAdd(&sl->msum, bmsum);
                if (bmabs != 0.0) atomicAdd(&sl->mabs, bmabs);
                if (lagged) {
                    if (ba != 0.0) atomicAdd(&sl->a, ba);
                    if (bpr != 0.0) atomicAdd(&sl->pr, bpr);
                    if (blockIdx.x == 0) sl->tstamp = globaltimer();
                }
            }
        }
        if (!grid_barrier(&sw->bar, sc.target, ctl.barrier_limit_ns, blockIdx.x == 0 ? sc.ts + 3 : nullptr)) break;

        // ---------------------------------------------------- choose move
        if (threadIdx.x == 0) {
            const int sched = sc.sched;
            // every total of the move in one round of paired loads
            const double2 mm = ldcg_pair(&sl->msum);
            const double2 rts = ldcg_pair(&sl->reserve);
            const double2 apr = ldcg_pair(&sl->a);
            const unsigned long long rsv = (unsigned long long)__double_as_longlong(rts.x);
            long long green = (long long)(rsv & ((1ull << kCountBits) - 1ull));
            long long edges = (long long)(rsv >> kCountBits);
            if (sched == SCHED_ALL_GREEN) {
                green = n;
                edges = ctl.nnz;
            }
            const double ms = mm.x, ma = mm.y;
            if (lagged) {
                // stop test and re-derivation triggers on this move's cash
                // C_t (gathered by the select), against H_t 1; the move is
                // made whatever they say
                const int r = ctl.r;
                const bool link = ctl.sched == SCHED_LINK;
                const double l1 = apr.x;
                const double sumr = (r == 1 && !link) ? l1 : apr.y;
                const unsigned long long now = (unsigned long long)__double_as_longlong(rts.y);
                const bool converged = sc.moves >= 1 && l1 / fabs(sc.hsum) < ctl.tol;
                bool want_refresh = false;
                if (converged) {
                    if (ctl.mixed && !sc.fresh) want_refresh = true;  // re-derive, then test again
                    else sc.stop_after = ST_OK;
                } else if (ctl.mixed &&
                           ((ctl.refresh_factor > 0.0 && l1 < ctl.refresh_factor * s_l1_refresh) ||
                            cash_stalled(l1, sc.stall_mark, sc.stall_count, ctl.stall_moves))) {
                    want_refresh = true;
                }
                sc.want_refresh = want_refresh ? 1 : 0;
                sc.l1 = l1;
                sc.lag_l1 = l1;
                sc.lag_sumr = sumr;
                sc.lag_now = now;
                if (blockIdx.x == 0) {
                    st->l1 = l1;
                    st->sumr = sumr;
                    st->iters = sc.iters;
                    st->stall_mark = sc.stall_mark;
                    st->stall_count = sc.stall_count;
                    // every block is done with the other slot (the last move's)
                    clear_slot(&sw->slot[sc.p ^ 1]);
                }
            }
            if (ctl.theta_lag) sc.have_lag = 1;
            sc.hsum += ms;
            sc.habs += ma;
            sc.moves++;
            sc.solve_moves++;
            sc.tot_green += green;
            sc.tot_edges += edges;
            sc.fresh = 0;
            if (sched == SCHED_MASK) sc.mask_cursor++;
            int mode;
            if (green == 0) mode = MODE_NONE;
            else if (sched == SCHED_ALL_GREEN || (double)edges >= ctl.pull_crossover * (double)ctl.nnz)
                mode = MODE_PULL;
            else
                mode = MODE_PUSH;
            if (mode == MODE_PUSH) sc.push_moves++;
            if (mode == MODE_PULL) sc.pull_moves++;
            sc.mode = mode;
            sc.green = green;
            sc.edges = edges;
            if (blockIdx.x == 0) {
                st->theta = sc.theta;
                st->theta_f = sc.theta_f;
                st->green = green;
                st->edges = edges;
                st->hsum = sc.hsum;
                st->habs = sc.habs;
                st->last_mabs = ma;
                st->moves = sc.moves;
                st->solve_moves = sc.solve_moves;
                st->tot_green = sc.tot_green;
                st->tot_edges = sc.tot_edges;
                st->push_moves = sc.push_moves;
                st->pull_moves = sc.pull_moves;
                st->fresh = 0;
                st->skip_move = 0;
                st->mask_cursor = sc.mask_cursor;
                st->mode = mode;
                MoveRecord rec;
                rec.move = sc.moves - 1;
                rec.green = green;
                rec.edges = edges;
                rec.mode = mode;
                rec.pad = 0;
                rec.theta = sc.theta;
                rec.l1 = st->l1;
                rec.hsum = sc.hsum;
                for (int q = 0; q < 4; ++q) rec.phase_us[q] = (float)(sc.ts[q + 1] - sc.ts[q]) * 1e-3f;
                rec.phase_us[4] = rec.phase_us[5] = 0.f;
                A.log[rec.move % kLogCap] = rec;
            }
        }
        __syncthreads();

        // ----------------------------------------------------------- move
        if (sc.mode == MODE_PUSH)
            push_chunks<T, kHasW, true>(A.c, A.col, A.w, A.f_eoff, A.f_base, A.f_m, A.chunk_row,
                                        sc.edges, sc.green, blockIdx.x, gridDim.x, sm.push,
                                        A.hubs, &sl->chunk_next);
        else if (sc.mode == MODE_PULL)
            pull_tiles<T, T, kHasW, true>(A.c, A.mt, A.t_ptr, A.t_src, A.t_w, A.tile_r, A.tile_e,
                                          A.ntiles, blockIdx.x, gridDim.x, sm.pull, &sl->chunk_next);
        // the stale threshold's next move: its decisions while this block waits
        if (!grid_barrier_with(&sw->bar, sc.target, ctl.barrier_limit_ns, blockIdx.x == 0 ? sc.ts + 5 : nullptr,
                               [&]() {
                                   if (ctl.theta_lag && sc.stop_after < 0 && !sc.want_refresh)
                                       sweep_lag_control(sc, ctl, n);
                               }))
            break;
        if (lead) {
            MoveRecord* rec = A.log + ((sc.moves - 1) % kLogCap);
            rec->phase_us[4] = (float)(sc.ts[5] - sc.ts[4]) * 1e-3f;
            rec->phase_us[5] = (float)(sc.ts[6] - sc.ts[5]) * 1e-3f;
        }
        if (sc.stop_after >= 0) {
            if (lead) {
                st->done = 1;
                st->status = sc.stop_after;
                st->mode = MODE_NONE;
                sw->bar.parity = (unsigned int)(sc.p ^ 1);
                sw->bar.tk_pass = sc.tk_pass;
                if (A.use_cond) {
                    cudaGraphSetConditional(A.cond_loop, 0u);
                    if (ctl.mixed) cudaGraphSetConditional(A.cond_refresh, 0u);
                }
            }
            return;
        }
        if (sc.want_refresh) {
            if (lead) {
                st->want_refresh = 1;
                sw->bar.parity = (unsigned int)(sc.p ^ 1);
                sw->bar.tk_pass = sc.tk_pass;
                if (A.use_cond) cudaGraphSetConditional(A.cond_refresh, 1u);
            }
            return;
        }
        if (threadIdx.x == 0) sc.p ^= 1;
        __syncthreads();
    }
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
