// librlgl: C ABI (include/rlgl.h) over the RLGL sweep kernels.
//
// The host side only validates arguments, owns device memory, enqueues
// kernels on the context's stream and reads results back; every step of a
// move runs in the kernels of rlgl_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/rlgl.h"
#include "rlgl_kernels.cuh"
#include "rlgl_batch.cuh"
#include "rlgl_power.cuh"
#include "rlgl_sweep.cuh"

using namespace rlgl;

namespace {

thread_local char g_thread_err[512] = "";

enum KClass { KC_STATS = 0, KC_SELECT, KC_PUSH, KC_PULL, KC_TOPK, KC_REFRESH, KC_SWEEP, KC_N };

struct ProfEv {
    int cls;
    cudaEvent_t a, b;
};

}  // namespace

struct rlgl_ctx {
    long long n = 0, nnz = 0;
    int prec = RLGL_FP64;
    bool has_w = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;
    cudaEvent_t done_ev = nullptr;  // end of the last asynchronous solve
    bool pending = false;           // an asynchronous solve not yet waited for
    int pending_sched = 0;
    long long pending_max = 0;
    int device = 0, sms = 0;
    // chain
    long long* row_ptr = nullptr;
    int* col = nullptr;
    float* w = nullptr;
    double* s = nullptr;
    float* sf = nullptr;     // s in FP32 (MIXED)
    void* ideg = nullptr;    // 1 / out-degree in the cash type
    long long* t_ptr = nullptr;
    int* t_src = nullptr;
    float* t_w = nullptr;
    long long* tile_r = nullptr;
    long long* tile_e = nullptr;
    long long ntiles = 0;
    long long* wtile_r = nullptr;  // the same split at warp tiles (power sweep, FP64 residual pull)
    long long* wtile_e = nullptr;
    long long nwtiles = 0;
    // state and scratch
    void* c = nullptr;       // cash, float (MIXED) or double (FP64)
    double* H = nullptr;
    void* mt = nullptr;      // dense moved cash m~ (cash type)
    double* y = nullptr;     // residual accumulator, all-zero at rest
    double* hsrc = nullptr;  // H_i s_i for residual pulls
    double* c0 = nullptr;    // recorded C_0 (rlgl_create_from_state), else null
    double* colsum = nullptr;  // (1 P)_j in FP64: step 0 from the uniform M_0
    long long* f_eoff = nullptr;
    long long* f_base = nullptr;
    void* f_m = nullptr;
    int* chunk_row = nullptr;
    double* part = nullptr;
    unsigned char* masks = nullptr;
    long long n_masks = 0;
    unsigned int* err = nullptr;
    MoveRecord* log = nullptr;
    DevState* st = nullptr;
    SweepState* sw = nullptr;  // grid barrier and per-move slots of the persistent sweep
    // batch of independent chains (nchains > 1): node -> chain map and
    // per-chain state; nchains == 1 is a single chain
    int nchains = 1;
    long long* node_ptr = nullptr;
    int* chain_of = nullptr;
    ChainState* cs = nullptr;
    double* bsums = nullptr;  // per-chain sum H, sum |H| [2 nchains]
    std::vector<int64_t> node_ptr_h;
    std::vector<int64_t> chain_nnz_h;  // links of each chain
    // persistent batch: per-chain merge-path tiles (for tiles of ct_items
    // items), the per-chain group barriers and slots, the work queue (built
    // for block size bq_block) and its counter, and the solve graph
    long long* ct_off = nullptr;
    long long* ct_r = nullptr;
    long long* ct_e = nullptr;
    long long ct_items = 0;
    BGroup* grp = nullptr;
    int* bq = nullptr;  // q_chain [q_len], q_member [q_len], g_of [nchains]
    long long q_len = 0;
    int bq_block = 0;
    int grid_batch = 0;
    unsigned long long* q_next = nullptr;
    cudaGraphExec_t batch_graph = nullptr;
    DevState* host_st = nullptr;  // pinned mirror
    Control* host_ctl = nullptr;  // pinned
    rlgl_params params{};
    // launch shapes
    int grid_nodes = 1, grid_select = 1, grid_push = 1, grid_pull = 1, grid_stats = 1;
    // solve graphs, one per schedule
    cudaGraphExec_t graph[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // solve graph of the persistent sweep (any schedule it serves) and its grid
    cudaGraphExec_t sweep_graph = nullptr;
    int grid_sweep = 0;
    // solve graph and grid of the all-green (power) sweep
    cudaGraphExec_t power_graph = nullptr;
    int grid_power = 0;
    int* hubs = nullptr;  // hub table of the push (kHubSlots ids, -1 empty), null when none
    int n_hubs = 0;
    // profiling
    int profiling = 0;
    std::vector<ProfEv> prof;
    double prof_ms[KC_N] = {0};
    long long prof_n[KC_N] = {0};
    char err_msg[512] = "";
};

// ------------------------------------------------------------------ errors

static rlgl_status fail(rlgl_ctx* ctx, rlgl_status s, const char* fmt, ...) {
    char* buf = ctx ? ctx->err_msg : g_thread_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    if (ctx) snprintf(g_thread_err, sizeof g_thread_err, "%s", ctx->err_msg);
    return s;
}

#define CK(ctx, call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? RLGL_ENOMEM : RLGL_ECUDA,   \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define CKL(ctx) CK(ctx, cudaGetLastError())

#define NOT_PENDING(ctx)                                                                   \
    do {                                                                                   \
        if ((ctx)->pending)                                                                \
            return fail((ctx), RLGL_EINVAL, "an asynchronous solve is pending: rlgl_wait"); \
    } while (0)

#define TRY(expr)                      \
    do {                               \
        rlgl_status s_ = (expr);       \
        if (s_ != RLGL_OK) return s_;  \
    } while (0)

// Device memory comes from one stream-ordered pool per device (allocations
// and frees are queued on the context's stream, so creating or destroying a
// context does not synchronise the whole device, as cudaMalloc/cudaFree may).
// Freed memory up to 4 GiB stays in the pool for the next context.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[128] = {nullptr};

static rlgl_status device_pool(rlgl_ctx* ctx) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (ctx->device < 0 || ctx->device >= 128) return fail(ctx, RLGL_EINVAL, "device id out of range");
    if (!g_pool[ctx->device]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        cudaMemPool_t pool;
        CK(ctx, cudaMemPoolCreate(&pool, &props));
        unsigned long long keep = 4ull << 30;
        CK(ctx, cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pool[ctx->device] = pool;
    }
    ctx->pool = g_pool[ctx->device];
    return RLGL_OK;
}

// Pinned host blocks for each context's device-state mirror, cut from slabs
// that live until the process exits and are recycled: releasing pinned
// memory (cudaFreeHost) may synchronise the whole device.
static constexpr size_t kPinBlock = ((sizeof(DevState) + sizeof(Control) + 255) / 256) * 256;
static std::mutex g_pin_mu;
static std::vector<void*> g_pin_free;

static void* pin_get() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        const int per_slab = 32;
        void* slab = nullptr;
        if (cudaMallocHost(&slab, kPinBlock * per_slab) != cudaSuccess) return nullptr;
        for (int k = per_slab - 1; k >= 0; --k) g_pin_free.push_back((char*)slab + k * kPinBlock);
    }
    void* p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}

static void pin_put(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

// Solve graphs of destroyed contexts. Destroying an executable graph that
// has been launched can wait for unrelated work on the device, which would
// stall a server that retires one request while others run; they are kept
// here until rlgl_release_retired() (a point where the caller knows the
// device is idle) or the end of the process.
static std::mutex g_retired_mu;
static std::vector<cudaGraphExec_t> g_retired;

static rlgl_status dalloc_bytes(rlgl_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    CK(ctx, cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream));
    return RLGL_OK;
}

template <typename P>
static rlgl_status dalloc(rlgl_ctx* ctx, P** p, size_t count) {
    return dalloc_bytes(ctx, (void**)p, count * sizeof(P));
}

static void dfree(rlgl_ctx* ctx, void* p) {
    if (p) cudaFreeAsync(p, ctx->stream);
}

static size_t cash_size(const rlgl_ctx* ctx) {
    return ctx->prec == RLGL_MIXED ? sizeof(float) : sizeof(double);
}

// ------------------------------------------------------------- profiling

static rlgl_status prof_begin(rlgl_ctx* ctx, int cls, ProfEv* ev) {
    if (!ctx->profiling) return RLGL_OK;
    ev->cls = cls;
    CK(ctx, cudaEventCreate(&ev->a));
    CK(ctx, cudaEventCreate(&ev->b));
    CK(ctx, cudaEventRecord(ev->a, ctx->stream));
    return RLGL_OK;
}

static rlgl_status prof_end(rlgl_ctx* ctx, ProfEv* ev) {
    if (!ctx->profiling) return RLGL_OK;
    CK(ctx, cudaEventRecord(ev->b, ctx->stream));
    ctx->prof.push_back(*ev);
    return RLGL_OK;
}

static rlgl_status prof_collect(rlgl_ctx* ctx) {
    if (ctx->prof.empty()) return RLGL_OK;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto& e : ctx->prof) {
        float ms = 0.f;
        CK(ctx, cudaEventElapsedTime(&ms, e.a, e.b));
        ctx->prof_ms[e.cls] += ms;
        ctx->prof_n[e.cls] += 1;
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    ctx->prof.clear();
    return RLGL_OK;
}

// ------------------------------------------------------------ enqueueing

// When capturing (graph) no profiling events are recorded.
struct Launch {
    rlgl_ctx* ctx;
    bool capture;
};

#define LAUNCH(L, cls, kernel_expr)                          \
    do {                                                     \
        ProfEv ev_{};                                        \
        if (!(L).capture) TRY(prof_begin((L).ctx, cls, &ev_)); \
        kernel_expr;                                         \
        CKL((L).ctx);                                        \
        if (!(L).capture) TRY(prof_end((L).ctx, &ev_));       \
    } while (0)

static int grid_for(long long work, int per_block, int cap);

// The FP64 residual pull (rlgl_power.cuh, warp tiles of the context's cash
// type) into y, guarded on the device like the rest of the re-derivation.
template <bool kHasW, int kIpt>
static void launch_rederive_pull_t(rlgl_ctx* ctx) {
    const int grid = grid_for(ctx->nwtiles, kWarpsPerBlock, ctx->sms * kPowerMinBlocks);
    k_rederive_pull<kHasW, kIpt><<<grid, kThreads, 0, ctx->stream>>>(
        ctx->y, ctx->hsrc, ctx->t_ptr, ctx->t_src, ctx->t_w, ctx->wtile_r, ctx->wtile_e, ctx->nwtiles, ctx->st);
}

static void launch_rederive_pull(rlgl_ctx* ctx) {
    constexpr int kF = power_ipt(4), kD = power_ipt(8);
    if (ctx->prec == RLGL_MIXED) {
        if (ctx->has_w) launch_rederive_pull_t<true, kF>(ctx);
        else launch_rederive_pull_t<false, kF>(ctx);
    } else {
        if (ctx->has_w) launch_rederive_pull_t<true, kD>(ctx);
        else launch_rederive_pull_t<false, kD>(ctx);
    }
}

template <typename T>
static rlgl_status enqueue_refresh(Launch L) {
    rlgl_ctx* ctx = L.ctx;
    const int n = (int)ctx->n;
    LAUNCH(L, KC_REFRESH,
           (k_refresh_src<<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(ctx->H, ctx->s, n,
                                                                          ctx->hsrc, ctx->st)));
    LAUNCH(L, KC_REFRESH, launch_rederive_pull(ctx));
    LAUNCH(L, KC_REFRESH,
           (k_refresh_apply<T><<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(
               (T*)ctx->c, ctx->H, ctx->y, ctx->c0, n, ctx->st, ctx->part)));
    return RLGL_OK;
}

static int grid_for(long long work, int per_block, int cap);

// Cash and 1/degree arrays start on 16-byte boundaries (vector loads).
static int vec_aligned(const rlgl_ctx* ctx) {
    return ((uintptr_t)ctx->c % 16 == 0) && ((uintptr_t)ctx->ideg % 16 == 0) ? 1 : 0;
}

// Graph handles of one solve graph (0 in eager mode).
struct Conds {
    unsigned long long loop = 0, refresh = 0, mode = 0;
    int use = 0;
};

// stats, [top-k passes], select.
template <typename T>
static rlgl_status enqueue_head(Launch L, int sched, const Conds& cd) {
    rlgl_ctx* ctx = L.ctx;
    const int n = (int)ctx->n;
    const BatchView bv{ctx->chain_of, ctx->cs, ctx->nchains};
    if (ctx->nchains > 1)
        LAUNCH(L, KC_STATS,
               (k_bstats<T><<<ctx->grid_select, kThreads, 0, ctx->stream>>>(
                   (const T*)ctx->c, (const T*)ctx->ideg, n, ctx->st, bv, cd.loop, cd.refresh,
                   cd.use)));
    else
        LAUNCH(L, KC_STATS,
               (k_stats<T><<<ctx->grid_stats, kThreads, 0, ctx->stream>>>(
                   (const T*)ctx->c, (const T*)ctx->ideg, n, ctx->st, ctx->part, cd.loop, cd.refresh,
                   cd.use, vec_aligned(ctx))));
    if (sched == RLGL_TOPFRAC) {
        const int bits = KeyOf<T>::bits;
        for (int hi = bits; hi > 0; hi -= kRadixBits) {
            int width = hi >= kRadixBits ? kRadixBits : hi;
            int shift = hi - width;
            LAUNCH(L, KC_TOPK,
                   (k_radix_pass<T><<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(
                       (const T*)ctx->c, n, ctx->st, shift, width)));
        }
    }
    if (ctx->nchains > 1)
        LAUNCH(L, KC_SELECT,
               (k_select<T, true><<<ctx->grid_select, kThreads, 0, ctx->stream>>>(
                   (T*)ctx->c, ctx->H, ctx->s, ctx->sf, ctx->row_ptr, (const T*)ctx->ideg, ctx->masks, n,
                   (T*)ctx->mt, ctx->f_eoff, ctx->f_base, (T*)ctx->f_m, ctx->chunk_row, ctx->st,
                   ctx->part, ctx->log, cd.mode, cd.use, bv)));
    else
        LAUNCH(L, KC_SELECT,
               (k_select<T, false><<<ctx->grid_select, kThreads, 0, ctx->stream>>>(
                   (T*)ctx->c, ctx->H, ctx->s, ctx->sf, ctx->row_ptr, (const T*)ctx->ideg, ctx->masks, n,
                   (T*)ctx->mt, ctx->f_eoff, ctx->f_base, (T*)ctx->f_m, ctx->chunk_row, ctx->st,
                   ctx->part, ctx->log, cd.mode, cd.use, bv)));
    return RLGL_OK;
}

template <typename T>
static rlgl_status enqueue_push(Launch L) {
    rlgl_ctx* ctx = L.ctx;
    if (ctx->has_w)
        LAUNCH(L, KC_PUSH,
               (k_push<T, true><<<ctx->grid_push, kThreads, 0, ctx->stream>>>(
                   (T*)ctx->c, ctx->col, ctx->w, ctx->f_eoff, ctx->f_base, (const T*)ctx->f_m,
                   ctx->chunk_row, ctx->st, ctx->n_hubs ? ctx->hubs : nullptr)));
    else
        LAUNCH(L, KC_PUSH,
               (k_push<T, false><<<ctx->grid_push, kThreads, 0, ctx->stream>>>(
                   (T*)ctx->c, ctx->col, ctx->w, ctx->f_eoff, ctx->f_base, (const T*)ctx->f_m,
                   ctx->chunk_row, ctx->st, ctx->n_hubs ? ctx->hubs : nullptr)));
    return RLGL_OK;
}

template <typename T>
static rlgl_status enqueue_pull(Launch L) {
    rlgl_ctx* ctx = L.ctx;
    if (ctx->has_w)
        LAUNCH(L, KC_PULL,
               (k_pull<T, T, true, 0><<<ctx->grid_pull, kThreads, 0, ctx->stream>>>(
                   (T*)ctx->c, (const T*)ctx->mt, ctx->t_ptr, ctx->t_src, ctx->t_w, ctx->tile_r,
                   ctx->tile_e, ctx->ntiles, ctx->st)));
    else
        LAUNCH(L, KC_PULL,
               (k_pull<T, T, false, 0><<<ctx->grid_pull, kThreads, 0, ctx->stream>>>(
                   (T*)ctx->c, (const T*)ctx->mt, ctx->t_ptr, ctx->t_src, ctx->t_w, ctx->tile_r,
                   ctx->tile_e, ctx->ntiles, ctx->st)));
    return RLGL_OK;
}

// A persistent kernel (rlgl_sweep.cuh, rlgl_power.cuh): one cooperative
// launch of `grid` blocks, never more than fit on the device at once.
template <typename T>
static rlgl_status launch_coop(rlgl_ctx* ctx, int grid, void (*kernel)(SweepArgs<T>), const SweepArgs<T>& a) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    memset(attr, 0, sizeof attr);
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(ctx, cudaLaunchKernelEx(&cfg, kernel, a));
    return RLGL_OK;
}

template <typename T>
static SweepArgs<T> sweep_args(rlgl_ctx* ctx, const Conds& cd) {
    SweepArgs<T> a;
    a.c = (T*)ctx->c;
    a.H = ctx->H;
    a.s = ctx->s;
    a.sf = ctx->sf;
    a.row_ptr = ctx->row_ptr;
    a.ideg = (const T*)ctx->ideg;
    a.masks = ctx->masks;
    a.mt = (T*)ctx->mt;
    a.mt2 = (T*)ctx->hsrc;  // free while no re-derivation runs
    a.facc = (T*)ctx->f_m;  // the power sweep clears it at every launch
    a.f_eoff = ctx->f_eoff;
    a.f_base = ctx->f_base;
    a.f_m = (T*)ctx->f_m;
    a.chunk_row = ctx->chunk_row;
    a.col = ctx->col;
    a.w = ctx->w;
    a.t_ptr = ctx->t_ptr;
    a.t_src = ctx->t_src;
    a.t_w = ctx->t_w;
    a.tile_r = ctx->tile_r;
    a.tile_e = ctx->tile_e;
    a.ntiles = ctx->ntiles;
    a.wtile_r = ctx->wtile_r;
    a.wtile_e = ctx->wtile_e;
    a.nwtiles = ctx->nwtiles;
    a.st = ctx->st;
    a.sw = ctx->sw;
    a.log = ctx->log;
    a.cond_loop = cd.loop;
    a.cond_refresh = cd.refresh;
    a.use_cond = cd.use;
    a.n = (int)ctx->n;
    a.vec_ok = vec_aligned(ctx);
    a.hubs = ctx->n_hubs ? ctx->hubs : nullptr;
    return a;
}

template <typename T>
static rlgl_status enqueue_sweep(Launch L, const Conds& cd) {
    rlgl_ctx* ctx = L.ctx;
    const SweepArgs<T> a = sweep_args<T>(ctx, cd);
    if (ctx->has_w)
        LAUNCH(L, KC_SWEEP, TRY((launch_coop<T>(ctx, ctx->grid_sweep, k_sweep<T, true>, a))));
    else
        LAUNCH(L, KC_SWEEP, TRY((launch_coop<T>(ctx, ctx->grid_sweep, k_sweep<T, false>, a))));
    return RLGL_OK;
}

// The all-green (power) sweep of rlgl_power.cuh.
template <typename T>
static rlgl_status enqueue_power(Launch L, const Conds& cd) {
    rlgl_ctx* ctx = L.ctx;
    const SweepArgs<T> a = sweep_args<T>(ctx, cd);
    if (ctx->has_w)
        LAUNCH(L, KC_SWEEP, TRY((launch_coop<T>(ctx, ctx->grid_power, k_power<T, true>, a))));
    else
        LAUNCH(L, KC_SWEEP, TRY((launch_coop<T>(ctx, ctx->grid_power, k_power<T, false>, a))));
    return RLGL_OK;
}

// The persistent batch solve (rlgl_batch.cuh) with blocks of BT threads.
template <typename T>
static BatchArgs<T> batch_args(rlgl_ctx* ctx) {
    BatchArgs<T> a;
    a.c = (T*)ctx->c;
    a.H = ctx->H;
    a.s = ctx->s;
    a.sf = ctx->sf;
    a.row_ptr = ctx->row_ptr;
    a.ideg = (const T*)ctx->ideg;
    a.masks = ctx->masks;
    a.mt = (T*)ctx->mt;
    a.f_eoff = ctx->f_eoff;
    a.f_base = ctx->f_base;
    a.f_m = (T*)ctx->f_m;
    a.chunk_row = ctx->chunk_row;
    a.col = ctx->col;
    a.w = ctx->w;
    a.t_ptr = ctx->t_ptr;
    a.t_src = ctx->t_src;
    a.t_w = ctx->t_w;
    a.ct_r = ctx->ct_r;
    a.ct_e = ctx->ct_e;
    a.ct_off = ctx->ct_off;
    a.node_ptr = ctx->node_ptr;
    a.cs = ctx->cs;
    a.grp = ctx->grp;
    a.q_chain = ctx->bq;
    a.q_member = ctx->bq + ctx->q_len;
    a.g_of = ctx->bq + 2 * ctx->q_len;
    a.q_len = ctx->q_len;
    a.q_next = ctx->q_next;
    a.y = ctx->y;
    a.hsrc = ctx->hsrc;
    a.st = ctx->st;
    a.nchains = ctx->nchains;
    return a;
}

template <typename T, bool kHasW, int BT>
static rlgl_status launch_bsweep_t(rlgl_ctx* ctx, const BatchArgs<T>& a) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)ctx->grid_batch);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    memset(attr, 0, sizeof attr);
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(ctx, cudaLaunchKernelEx(&cfg, k_bsweep<T, kHasW, BT>, a));
    return RLGL_OK;
}

template <typename T>
static rlgl_status enqueue_bsweep(rlgl_ctx* ctx) {
    const BatchArgs<T> a = batch_args<T>(ctx);
    switch (ctx->bq_block) {
        case 128: return ctx->has_w ? launch_bsweep_t<T, true, 128>(ctx, a) : launch_bsweep_t<T, false, 128>(ctx, a);
        case 512: return ctx->has_w ? launch_bsweep_t<T, true, 512>(ctx, a) : launch_bsweep_t<T, false, 512>(ctx, a);
        default: return ctx->has_w ? launch_bsweep_t<T, true, 256>(ctx, a) : launch_bsweep_t<T, false, 256>(ctx, a);
    }
}

template <typename T, bool kHasW>
static int bsweep_fit_t(int bt) {
    int nb = 0;
    cudaError_t e;
    switch (bt) {
        case 128: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bsweep<T, kHasW, 128>, 128, 0); break;
        case 512: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bsweep<T, kHasW, 512>, 512, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bsweep<T, kHasW, 256>, 256, 0); break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

static int bsweep_fit(rlgl_ctx* ctx, int bt) {
    if (ctx->prec == RLGL_MIXED) return ctx->has_w ? bsweep_fit_t<float, true>(bt) : bsweep_fit_t<float, false>(bt);
    return ctx->has_w ? bsweep_fit_t<double, true>(bt) : bsweep_fit_t<double, false>(bt);
}

// Blocks of the sweep: all that fit on the device at once (the occupancy of
// the instantiation this context uses), fewer for a small chain, where each
// block still gets at least one block-iteration of nodes.
template <typename T>
static int sweep_fit(rlgl_ctx* ctx) {
    int nb = 0;
    cudaError_t e = ctx->has_w
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<T, true>, kThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<T, false>, kThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

static int sweep_grid(rlgl_ctx* ctx) {
    const int nb = ctx->prec == RLGL_MIXED ? sweep_fit<float>(ctx) : sweep_fit<double>(ctx);
    if (nb < 1) return 0;
    const long long fit = (long long)nb * ctx->sms;
    long long work = ctx->n > ctx->nnz / 8 ? ctx->n : ctx->nnz / 8;
    long long want = (work + kNodesPerIter - 1) / kNodesPerIter;
    if (want < 1) want = 1;
    return (int)(want < fit ? want : fit);
}

// Blocks of the power sweep: all that fit, fewer when the chain has fewer
// merge-path tiles (and node block-iterations) than that.
template <typename T>
static int power_fit(rlgl_ctx* ctx) {
    int nb = 0;
    cudaError_t e = ctx->has_w
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_power<T, true>, kThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_power<T, false>, kThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

static int power_grid(rlgl_ctx* ctx) {
    const int nb = ctx->prec == RLGL_MIXED ? power_fit<float>(ctx) : power_fit<double>(ctx);
    if (nb < 1) return 0;
    const long long fit = (long long)nb * ctx->sms;
    long long want = ctx->ntiles;
    const long long nodes = (ctx->n + kNodesPerIter - 1) / kNodesPerIter;
    if (nodes > want) want = nodes;
    if (want < 1) want = 1;
    return (int)(want < fit ? want : fit);
}

// Whether a solve with this schedule runs as the persistent sweep.
static bool use_sweep(const rlgl_ctx* ctx, int sched) {
    return ctx->params.persistent && ctx->nchains <= 1 && ctx->grid_sweep > 0 &&
           !(sched == RLGL_TOPFRAC && ctx->params.theta_lag);
}

// Whether it runs as the all-green (power) sweep: all-green with the plain
// stop rule (the stale threshold's order of move and stop test is the
// general sweep's).
static bool use_power(const rlgl_ctx* ctx, int sched) {
    return use_sweep(ctx, sched) && sched == RLGL_ALL_GREEN && !ctx->params.theta_lag && ctx->grid_power > 0;
}

// One eager iteration of Alg. 1: stats [top-k] select push pull. Every kernel
// checks the device state and returns at once when it has nothing to do.
template <typename T>
static rlgl_status enqueue_iteration(Launch L, int sched) {
    Conds none;
    TRY(enqueue_head<T>(L, sched, none));
    TRY(enqueue_push<T>(L));
    TRY(enqueue_pull<T>(L));
    return RLGL_OK;
}

static rlgl_status iteration(rlgl_ctx* ctx, bool capture, int sched, unsigned long long, int) {
    Launch L{ctx, capture};
    if (ctx->prec == RLGL_MIXED) return enqueue_iteration<float>(L, sched);
    return enqueue_iteration<double>(L, sched);
}

static rlgl_status forced_refresh(rlgl_ctx* ctx, bool apply) {
    k_set_refresh_flags<<<1, 1, 0, ctx->stream>>>(ctx->st, 1, apply ? 1 : 0);
    CKL(ctx);
    Launch L{ctx, false};
    if (ctx->prec == RLGL_MIXED) return enqueue_refresh<float>(L);
    return enqueue_refresh<double>(L);
}

static void drop_graphs(rlgl_ctx* ctx) {
    for (auto& g : ctx->graph)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    if (ctx->sweep_graph) {
        cudaGraphExecDestroy(ctx->sweep_graph);
        ctx->sweep_graph = nullptr;
    }
    if (ctx->power_graph) {
        cudaGraphExecDestroy(ctx->power_graph);
        ctx->power_graph = nullptr;
    }
    if (ctx->batch_graph) {
        cudaGraphExecDestroy(ctx->batch_graph);
        ctx->batch_graph = nullptr;
    }
}

static rlgl_status read_state(rlgl_ctx* ctx) {
    CK(ctx, cudaMemcpyAsync(ctx->host_st, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost,
                            ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return RLGL_OK;
}

static void fill_control(rlgl_ctx* ctx, Control* c, int sched, double theta, double tol,
                         long long max_steps, int solving) {
    memset(c, 0, sizeof *c);
    c->tol = tol;
    c->theta_arg = theta;
    c->theta_scale = ctx->params.theta_scale;
    c->top_frac = ctx->params.top_frac;
    c->pull_crossover = ctx->params.pull_crossover;
    c->refresh_factor = ctx->params.refresh_factor;
    c->time_limit_ns = ctx->params.time_limit_s * 1e9;
    c->max_steps = max_steps;
    c->max_iters = 2 * max_steps + 16;
    c->nnz = ctx->nnz;
    c->rr_blocks = ctx->params.rr_blocks;
    c->pc_frac = ctx->params.pc_frac;
    c->seed = ctx->params.seed;
    c->barrier_limit_ns = (unsigned long long)(ctx->params.barrier_limit_s * 1e9);
    c->test_skip_barrier = ctx->params.test_skip_barrier;
    c->stall_moves = ctx->params.stall_moves;
    c->theta_lag = solving ? ctx->params.theta_lag : 0;
    c->sched = sched;
    c->r = ctx->params.r;
    c->safety_every = solving ? ctx->params.safety_every : 0;
    c->solving = solving;
    c->mixed = ctx->prec == RLGL_MIXED;
    c->n_masks = (int)(ctx->n_masks > 0 ? ctx->n_masks : 1);
}

__global__ void k_begin(DevState* st) {
    st->base_green = st->tot_green;
    st->base_edges = st->tot_edges;
    st->base_push = st->push_moves;
    st->base_pull = st->pull_moves;
    st->base_refreshes = st->refreshes;
    st->done = 0;
    st->status = 0;
    st->iters = 0;
    st->solve_moves = 0;
    st->skip_move = 0;
    st->mode = 0;
    st->want_refresh = 0;
    st->force_refresh = 0;
    st->apply_refresh = 0;
    st->green = 0;
    st->edges = 0;
    st->stall_mark = kNoMark;
    st->stall_count = 0;
}

static rlgl_status begin(rlgl_ctx* ctx, int sched, double theta, double tol, long long max_steps,
                         int solving, double chain_tol = -1.0) {
    fill_control(ctx, ctx->host_ctl, sched, theta, tol, max_steps, solving);
    CK(ctx, cudaMemcpyAsync(&ctx->st->ctl, ctx->host_ctl, sizeof(Control), cudaMemcpyHostToDevice,
                            ctx->stream));
    k_begin<<<1, 1, 0, ctx->stream>>>(ctx->st);
    CKL(ctx);
    if (ctx->nchains > 1) {
        k_bbegin<<<grid_for(ctx->nchains, kThreads, 1024), kThreads, 0, ctx->stream>>>(
            ctx->cs, ctx->nchains, chain_tol, 0);
        CKL(ctx);
    }
    return RLGL_OK;
}

// --------------------------------------------------------------- create

static rlgl_status upload(rlgl_ctx* ctx, void* dst, const void* src, size_t bytes, rlgl_memspace sp) {
    if (bytes == 0) return RLGL_OK;
    CK(ctx, cudaMemcpyAsync(dst, src, bytes,
                            sp == RLGL_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            ctx->stream));
    return RLGL_OK;
}

static int grid_for(long long work, int per_block, int cap) {
    long long g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Exclusive prefix sum in place over x[0..m) (x[m-1] then holds the total of
// the first m-1 inputs); used on counts laid out as cnt[j + 1].
static rlgl_status device_inclusive_scan(rlgl_ctx* ctx, long long* x, long long m) {
    long long nb = (m + kNodesPerIter - 1) / kNodesPerIter;
    long long* tot = nullptr;
    TRY(dalloc(ctx, &tot, (size_t)nb));
    k_scan_blocks<<<(unsigned)nb, kThreads, 0, ctx->stream>>>(x, m, tot);
    CKL(ctx);
    k_scan_tot<<<1, kThreads, 0, ctx->stream>>>(tot, nb);
    CKL(ctx);
    k_scan_add<<<(unsigned)nb, kThreads, 0, ctx->stream>>>(x, m, tot);
    CKL(ctx);
    dfree(ctx, tot);  // stream-ordered
    return RLGL_OK;
}

// Step 0 (Eq. init): H = M_0, C_1 = M_0 (P - I). The uniform M_0 (NULL; per
// chain in a batch) is set on the device from the precomputed column sums;
// a given M_0 goes through the FP64 re-derivation C = C_0 + H (P - I) with
// C_0 = 0.
static rlgl_status set_step0(rlgl_ctx* ctx, const double* m0, rlgl_memspace sp) {
    const long long n = ctx->n;
    if (ctx->c0) {
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(ctx, ctx->c0);
        ctx->c0 = nullptr;
        drop_graphs(ctx);  // captured launches hold the C_0 pointer
    }
    CK(ctx, cudaMemsetAsync(ctx->st, 0, sizeof(DevState), ctx->stream));
    if (m0) {
        TRY(upload(ctx, ctx->H, m0, (size_t)n * sizeof(double), sp));
        CK(ctx, cudaMemsetAsync(ctx->c, 0, (size_t)n * cash_size(ctx), ctx->stream));
        TRY(forced_refresh(ctx, true));
        k_hist_sums<<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(ctx->H, (int)n, ctx->st, ctx->part, 1);
    } else {
        // (also sums H into the state, as k_hist_sums does)
        const int* chain_of = ctx->nchains > 1 ? ctx->chain_of : nullptr;
        const long long* node_ptr = ctx->nchains > 1 ? ctx->node_ptr : nullptr;
        if (ctx->prec == RLGL_MIXED)
            k_step0_uniform<float><<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(
                (float*)ctx->c, ctx->H, ctx->colsum, (int)n, chain_of, node_ptr, ctx->st, ctx->part);
        else
            k_step0_uniform<double><<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(
                (double*)ctx->c, ctx->H, ctx->colsum, (int)n, chain_of, node_ptr, ctx->st, ctx->part);
    }
    CKL(ctx);
    if (ctx->nchains > 1) {
        const BatchView bv{ctx->chain_of, ctx->cs, ctx->nchains};
        k_bbegin<<<grid_for(ctx->nchains, kThreads, 1024), kThreads, 0, ctx->stream>>>(
            ctx->cs, ctx->nchains, -1.0, 1);
        k_bhist_sums<<<ctx->grid_select, kThreads, 0, ctx->stream>>>(ctx->H, (int)n, bv);
        k_bhist_finish<<<grid_for(ctx->nchains, kThreads, 1024), kThreads, 0, ctx->stream>>>(bv, 1, nullptr);
        CKL(ctx);
    }
    return RLGL_OK;
}

static rlgl_status build_sweep_graph(rlgl_ctx* ctx, bool power);

// eager_graph: build the single-chain sweep's solve graph on the host while
// the device builds the in-link copy (the graph holds no parameter, only the
// context's buffers and grids).
static rlgl_status create_common(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                 const float* w, rlgl_precision prec, rlgl_memspace src,
                                 void* stream, rlgl_ctx** out, bool eager_graph = false) {
    if (!out) return fail(nullptr, RLGL_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n >= (1ll << kCountBits)) return fail(nullptr, RLGL_EINVAL, "n=%lld out of range [1, 2^27)", (long long)n);
    if (nnz < 1 || nnz >= (1ll << 37)) return fail(nullptr, RLGL_EINVAL, "nnz=%lld out of range", (long long)nnz);
    if (!row_ptr || !col) return fail(nullptr, RLGL_EINVAL, "row_ptr/col is NULL");
    if (prec != RLGL_FP64 && prec != RLGL_MIXED) return fail(nullptr, RLGL_EINVAL, "bad precision");
    if (src != RLGL_HOST && src != RLGL_DEVICE) return fail(nullptr, RLGL_EINVAL, "bad memspace");
    rlgl_ctx* ctx = new (std::nothrow) rlgl_ctx();
    if (!ctx) return fail(nullptr, RLGL_ENOMEM, "host allocation failed");
    *out = ctx;  // freed by the caller wrapper on failure
    ctx->n = n;
    ctx->nnz = nnz;
    ctx->prec = prec;
    ctx->has_w = (w != nullptr);
    rlgl_default_params(&ctx->params);
    CK(ctx, cudaGetDevice(&ctx->device));
    CK(ctx, cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device));
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        CK(ctx, cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    TRY(device_pool(ctx));
    CK(ctx, cudaEventCreateWithFlags(&ctx->done_ev, cudaEventDisableTiming));
    const int cap = ctx->sms * 8 < kMaxGrid ? ctx->sms * 8 : kMaxGrid;
    ctx->grid_nodes = grid_for(n, kThreads, cap);
    ctx->grid_select = grid_for(n, kNodesPerIter, cap);
    ctx->grid_stats = grid_for(n, kThreads * 8, ctx->sms * 2);  // about 8+ nodes per thread
    // push/pull grids grow with the work up to a few blocks per SM, so that a
    // small chain does not launch hundreds of idle blocks (which would also
    // crowd out other contexts' work on the device)
    ctx->grid_push = grid_for(nnz, kPushChunk, ctx->sms * 4);
    ctx->grid_pull = grid_for(n + nnz, kMpItems, ctx->sms * 8);
    ctx->grid_sweep = sweep_grid(ctx);
    ctx->grid_power = power_grid(ctx);
    const size_t cs = cash_size(ctx);

    TRY(dalloc(ctx, &ctx->row_ptr, (size_t)n + 1));
    TRY(dalloc(ctx, &ctx->col, (size_t)nnz));
    if (ctx->has_w) TRY(dalloc(ctx, &ctx->w, (size_t)nnz));
    TRY(dalloc(ctx, &ctx->s, (size_t)n));
    if (prec == RLGL_MIXED) TRY(dalloc(ctx, &ctx->sf, (size_t)n));
    TRY(dalloc_bytes(ctx, &ctx->ideg, (size_t)n * cs));
    TRY(dalloc(ctx, &ctx->t_ptr, (size_t)n + 1));
    TRY(dalloc(ctx, &ctx->t_src, (size_t)nnz));
    if (ctx->has_w) TRY(dalloc(ctx, &ctx->t_w, (size_t)nnz));
    ctx->ntiles = (n + nnz + kMpItems - 1) / kMpItems;  // (grid_pull above uses the same count)
    TRY(dalloc(ctx, &ctx->tile_r, (size_t)ctx->ntiles + 1));
    TRY(dalloc(ctx, &ctx->tile_e, (size_t)ctx->ntiles + 1));
    const long long witems = 32 * power_ipt((int)cs);
    ctx->nwtiles = (n + nnz + witems - 1) / witems;
    TRY(dalloc(ctx, &ctx->wtile_r, (size_t)ctx->nwtiles + 1));
    TRY(dalloc(ctx, &ctx->wtile_e, (size_t)ctx->nwtiles + 1));
    TRY(dalloc_bytes(ctx, &ctx->c, (size_t)n * cs));
    TRY(dalloc(ctx, &ctx->H, (size_t)n));
    TRY(dalloc_bytes(ctx, &ctx->mt, (size_t)n * cs));
    TRY(dalloc(ctx, &ctx->y, (size_t)n));
    TRY(dalloc(ctx, &ctx->hsrc, (size_t)n));
    TRY(dalloc(ctx, &ctx->colsum, (size_t)n));
    TRY(dalloc(ctx, &ctx->f_eoff, (size_t)n));
    TRY(dalloc(ctx, &ctx->f_base, (size_t)n));
    TRY(dalloc_bytes(ctx, &ctx->f_m, (size_t)n * cs));
    TRY(dalloc(ctx, &ctx->chunk_row, (size_t)(nnz / kPushChunk + 2)));
    TRY(dalloc(ctx, &ctx->part, (size_t)(4 * kMaxGrid + 8)));
    TRY(dalloc(ctx, &ctx->err, 1));
    TRY(dalloc(ctx, &ctx->log, (size_t)kLogCap));
    TRY(dalloc(ctx, &ctx->st, 1));
    TRY(dalloc(ctx, &ctx->sw, 1));
    // the sweep reads slot fields in 16-byte pairs and stages the cash, 1/d
    // and row offsets with 16-byte copies (pool allocations are aligned far
    // beyond that)
    if ((((uintptr_t)ctx->sw | (uintptr_t)ctx->c | (uintptr_t)ctx->ideg | (uintptr_t)ctx->row_ptr) & 15u) != 0)
        return fail(ctx, RLGL_ENOMEM, "device buffers not 16-byte aligned");
    ctx->host_st = static_cast<DevState*>(pin_get());
    if (!ctx->host_st) return fail(ctx, RLGL_ENOMEM, "pinned host allocation failed");
    ctx->host_ctl = reinterpret_cast<Control*>(reinterpret_cast<char*>(ctx->host_st) + sizeof(DevState));
    CK(ctx, cudaMemsetAsync(ctx->y, 0, (size_t)n * sizeof(double), ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->err, 0, sizeof(unsigned int), ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->st, 0, sizeof(DevState), ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->sw, 0, sizeof(SweepState), ctx->stream));

    TRY(upload(ctx, ctx->row_ptr, row_ptr, ((size_t)n + 1) * sizeof(long long), src));
    TRY(upload(ctx, ctx->col, col, (size_t)nnz * sizeof(int), src));
    if (ctx->has_w) TRY(upload(ctx, ctx->w, w, (size_t)nnz * sizeof(float), src));

    const int gv = grid_for(nnz, kThreads, ctx->sms * 16);
    k_validate<<<gv, kThreads, 0, ctx->stream>>>(ctx->row_ptr, ctx->col, ctx->w, n, nnz, ctx->err);
    CKL(ctx);
    unsigned int err = 0;
    CK(ctx, cudaMemcpyAsync(&err, ctx->err, sizeof err, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (err & 1u) return fail(ctx, RLGL_EINVAL, "row_ptr is not a valid CSR offset array");
    if (err & 4u) return fail(ctx, RLGL_EINVAL, "a column index is outside [0, n)");
    if (err & 2u) return fail(ctx, RLGL_ENOTSTOCHASTIC, "a row has no out-edge (P must be stochastic)");
    if (err & 8u) return fail(ctx, RLGL_ENOTSTOCHASTIC, "a weight is not positive and finite");

    const int gn = grid_for(n, kThreads, ctx->sms * 16);
    // long weighted rows go to a list (chunk_row and err serve as scratch
    // until the CSC build below) and get a block each
    CK(ctx, cudaMemsetAsync(ctx->err, 0, sizeof(unsigned int), ctx->stream));
    k_row_scale<<<gn, kThreads, 0, ctx->stream>>>(
        ctx->row_ptr, ctx->w, n, ctx->s, ctx->sf,
        prec == RLGL_MIXED ? (float*)ctx->ideg : nullptr,
        prec == RLGL_MIXED ? nullptr : (double*)ctx->ideg, ctx->chunk_row, ctx->err);
    CKL(ctx);
    if (ctx->has_w) {
        const long long max_long = nnz / kLongRowW + 1;  // rows longer than kLongRowW
        k_row_scale_long<<<(unsigned int)max_long, kThreads, 0, ctx->stream>>>(
            ctx->row_ptr, ctx->w, ctx->s, ctx->sf, ctx->chunk_row, ctx->err);
        CKL(ctx);
    }
    // In-link (CSC) copy: counts, scan, scatter.
    long long* cursor = nullptr;
    TRY(dalloc(ctx, &cursor, (size_t)n + 1));
    CK(ctx, cudaMemsetAsync(ctx->t_ptr, 0, ((size_t)n + 1) * sizeof(long long), ctx->stream));
    k_count_in<<<gv, kThreads, 0, ctx->stream>>>(ctx->col, nnz, ctx->t_ptr);
    CKL(ctx);
    rlgl_status sc = device_inclusive_scan(ctx, ctx->t_ptr, n + 1);
    if (sc != RLGL_OK) { dfree(ctx, cursor); return sc; }
    CK(ctx, cudaMemcpyAsync(cursor, ctx->t_ptr, ((size_t)n + 1) * sizeof(long long),
                            cudaMemcpyDeviceToDevice, ctx->stream));
    // Hub targets of the push: the nodes whose in-degree is at least
    // max(4096, n / 8, 32 x the mean), like the auxiliary node of a PageRank
    // chain, which every node feeds; up to one per slot of the direct-mapped
    // table (largest first). Summing a hub's additions per block costs the
    // push a check per link and a warp reduction per hub link: measured on
    // R-MAT 20 (per-link threshold, 79 moves), tables of the 64 nodes of
    // in-degree >= 1024, or of those >= 8192, made the solve 1.7x and 1.4x
    // slower than no table, so only nodes that a large share of all nodes
    // feed qualify. A histogram of log2(in-degree) gives the degree above
    // which at most a few thousand candidates lie; those are sorted here.
    {
        const double mean = (double)nnz / (double)n;
        double fl = 32.0 * mean;
        if (fl < 4096.0) fl = 4096.0;
        if (fl < (double)n / 8.0) fl = (double)n / 8.0;
        const long long floor_deg = (long long)fl;
        unsigned int* hist = nullptr;
        TRY(dalloc(ctx, &hist, 64 + 1));
        CK(ctx, cudaMemsetAsync(hist, 0, 65 * sizeof(unsigned int), ctx->stream));
        k_indeg_log2_hist<<<grid_for(n, kThreads, ctx->sms * 4), kThreads, 0, ctx->stream>>>(ctx->t_ptr, n, hist);
        CKL(ctx);
        unsigned int hh[64];
        CK(ctx, cudaMemcpyAsync(hh, hist, sizeof hh, cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        // the lowest power of two with at most 4096 nodes at or above it,
        // stopping once kHubSlots are there
        long long above = 0;
        int bin = 63, tbin = 63;
        for (; bin >= 0; --bin) {
            if (above + hh[bin] > 4096) break;
            above += hh[bin];
            tbin = bin;
            if (above >= kHubSlots) break;
        }
        long long thr = 1ll << (tbin < 62 ? tbin : 62);
        if (thr < floor_deg) thr = floor_deg;
        constexpr int kCap = 8192;
        int* cid = nullptr;
        long long* cdeg = nullptr;
        rlgl_status hs = dalloc(ctx, &cid, kCap);
        if (hs == RLGL_OK) hs = dalloc(ctx, &cdeg, kCap);
        if (hs != RLGL_OK) { dfree(ctx, hist); return hs; }
        CK(ctx, cudaMemsetAsync(hist + 64, 0, sizeof(unsigned int), ctx->stream));
        k_hub_candidates<<<grid_for(n, kThreads, ctx->sms * 4), kThreads, 0, ctx->stream>>>(ctx->t_ptr, n, thr, kCap,
                                                                                           cid, cdeg, hist + 64);
        CKL(ctx);
        unsigned int nc = 0;
        CK(ctx, cudaMemcpyAsync(&nc, hist + 64, sizeof nc, cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        if (nc > (unsigned int)kCap) nc = kCap;
        std::vector<int> ids(nc);
        std::vector<long long> dg(nc);
        if (nc) {
            CK(ctx, cudaMemcpyAsync(ids.data(), cid, nc * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            CK(ctx, cudaMemcpyAsync(dg.data(), cdeg, nc * sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
            CK(ctx, cudaStreamSynchronize(ctx->stream));
        }
        dfree(ctx, cid);
        dfree(ctx, cdeg);
        dfree(ctx, hist);
        std::vector<int> order(nc);
        for (unsigned int k = 0; k < nc; ++k) order[k] = (int)k;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return dg[a] != dg[b] ? dg[a] > dg[b] : ids[a] < ids[b]; });
        int tab[kHubSlots];
        for (int t = 0; t < kHubSlots; ++t) tab[t] = -1;
        int got = 0;
        for (int k : order) {
            const int sl = hub_slot(ids[k]);
            if (tab[sl] < 0) {
                tab[sl] = ids[k];
                ++got;
            }
        }
        ctx->n_hubs = got;
        if (got) {
            TRY(dalloc(ctx, &ctx->hubs, kHubSlots));
            CK(ctx, cudaMemcpyAsync(ctx->hubs, tab, sizeof tab, cudaMemcpyHostToDevice, ctx->stream));
        }
    }
    // edge-balanced scatter (a warp per row would leave one warp with every
    // edge of a hub row)
    const long long nch = (nnz + kPushChunk - 1) / kPushChunk;
    k_chunk_rows<<<grid_for(nch + 1, kThreads, ctx->sms * 8), kThreads, 0, ctx->stream>>>(
        ctx->row_ptr, n, nnz, ctx->chunk_row);
    k_csc_scatter<<<grid_for(nch, 1, ctx->sms * 8), kThreads, 0, ctx->stream>>>(
        ctx->row_ptr, ctx->col, ctx->w, nnz, ctx->chunk_row, cursor, ctx->t_src, ctx->t_w);
    CKL(ctx);
    const int gt = grid_for(ctx->ntiles + 1, kThreads, ctx->sms * 16);
    k_mp_partition<<<gt, kThreads, 0, ctx->stream>>>(ctx->t_ptr, n, nnz, ctx->ntiles, kMpItems, ctx->tile_r,
                                                      ctx->tile_e);
    const int gw = grid_for(ctx->nwtiles + 1, kThreads, ctx->sms * 16);
    k_mp_partition<<<gw, kThreads, 0, ctx->stream>>>(ctx->t_ptr, n, nnz, ctx->nwtiles,
                                                      32 * power_ipt((int)cash_size(ctx)), ctx->wtile_r,
                                                      ctx->wtile_e);
    CKL(ctx);
    CK(ctx, cudaMemsetAsync(ctx->colsum, 0, (size_t)n * sizeof(double), ctx->stream));
    if (ctx->has_w)
        k_colsum_tiles<true><<<ctx->grid_pull, kThreads, 0, ctx->stream>>>(
            ctx->colsum, ctx->s, ctx->t_ptr, ctx->t_src, ctx->t_w, ctx->tile_r, ctx->tile_e, ctx->ntiles);
    else
        k_colsum_tiles<false><<<ctx->grid_pull, kThreads, 0, ctx->stream>>>(
            ctx->colsum, ctx->s, ctx->t_ptr, ctx->t_src, ctx->t_w, ctx->tile_r, ctx->tile_e, ctx->ntiles);
    CKL(ctx);
    if (eager_graph && ctx->params.persistent && build_sweep_graph(ctx, false) != RLGL_OK) {
        // (the first solve tries again and falls back to the phase kernels)
        cudaGetLastError();
        ctx->err_msg[0] = '\0';
    }
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    dfree(ctx, cursor);
    return RLGL_OK;
}

extern "C" {

rlgl_status rlgl_default_params(rlgl_params* p) {
    if (!p) return RLGL_EINVAL;
    p->theta_scale = 1.0;
    p->r = 1;
    p->top_frac = 0.01;
    p->pull_crossover = 0.9;
    p->safety_every = 0;
    p->refresh_factor = 1e-4;
    p->time_limit_s = 600.0;
    p->rr_blocks = 8;
    p->pc_frac = 0.05;
    p->seed = 0;
    p->persistent = 1;
    p->barrier_limit_s = 2.0;
    p->test_skip_barrier = 0;
    p->stall_moves = 32;
    p->theta_lag = 0;
    p->batch_block = 256;
    return RLGL_OK;
}

rlgl_status rlgl_create(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                        const float* w, const double* m0, rlgl_precision prec, rlgl_memspace src,
                        void* stream, rlgl_ctx** out) {
    rlgl_ctx* ctx = nullptr;
    rlgl_status s = create_common(n, nnz, row_ptr, col, w, prec, src, stream, &ctx, true);
    if (s == RLGL_OK) s = set_step0(ctx, m0, src);
    if (s != RLGL_OK) {
        if (ctx) snprintf(g_thread_err, sizeof g_thread_err, "%s", ctx->err_msg);
        rlgl_destroy(ctx);
        if (out) *out = nullptr;
        return s;
    }
    *out = ctx;
    return RLGL_OK;
}

rlgl_status rlgl_create_from_state(int64_t n, int64_t nnz, const int64_t* row_ptr,
                                   const int32_t* col, const float* w, const double* c,
                                   const double* h, rlgl_precision prec, rlgl_memspace src,
                                   void* stream, rlgl_ctx** out) {
    if (!c || !h) return fail(nullptr, RLGL_EINVAL, "c/h is NULL");
    rlgl_ctx* ctx = nullptr;
    rlgl_status s = create_common(n, nnz, row_ptr, col, w, prec, src, stream, &ctx);
    auto bail = [&](rlgl_status st) {
        if (ctx) snprintf(g_thread_err, sizeof g_thread_err, "%s", ctx->err_msg);
        rlgl_destroy(ctx);
        if (out) *out = nullptr;
        return st;
    };
    if (s != RLGL_OK) return bail(s);
    // Check the total of c on the host, then record C_0 = c - h (P - I).
    std::vector<double> hc((size_t)n);
    if (src == RLGL_DEVICE) {
        if (cudaMemcpy(hc.data(), c, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            return bail(fail(ctx, RLGL_ECUDA, "reading c failed"));
    } else {
        memcpy(hc.data(), c, (size_t)n * sizeof(double));
    }
    double tot = 0.0, l1 = 0.0;
    for (double v : hc) { tot += v; l1 += fabs(v); }
    if (fabs(tot) > 1e-12 * (l1 > 1.0 ? l1 : 1.0))
        return bail(fail(ctx, RLGL_EINVAL, "sum of c is %g, not zero", tot));
    if ((s = upload(ctx, ctx->H, h, (size_t)n * sizeof(double), src)) != RLGL_OK) return bail(s);
    if ((s = dalloc(ctx, &ctx->c0, (size_t)n)) != RLGL_OK) return bail(s);
    if (cudaMemcpyAsync(ctx->c0, hc.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess)
        return bail(fail(ctx, RLGL_ECUDA, "upload of c failed"));
    // y = H P by the residual pull (forced, measuring), then C_0 and C.
    k_set_refresh_flags<<<1, 1, 0, ctx->stream>>>(ctx->st, 1, 0);
    k_refresh_src<<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(ctx->H, ctx->s, (int)n, ctx->hsrc, ctx->st);
    launch_rederive_pull(ctx);
    if (ctx->prec == RLGL_MIXED)
        k_record_c0<float><<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(ctx->c0, ctx->H, ctx->y, (float*)ctx->c, (int)n, ctx->st);
    else
        k_record_c0<double><<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(ctx->c0, ctx->H, ctx->y, (double*)ctx->c, (int)n, ctx->st);
    k_hist_sums<<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(ctx->H, (int)n, ctx->st, ctx->part, 1);
    if (cudaGetLastError() != cudaSuccess) return bail(fail(ctx, RLGL_ECUDA, "launch failed"));
    // The cash is exactly what was given (fresh), and a resumed state counts
    // as t >= 2 for the stopping rule.
    int one = 1;
    long long mv = 1;
    if (cudaMemcpyAsync(&ctx->st->fresh, &one, sizeof one, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(&ctx->st->moves, &mv, sizeof mv, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(&ctx->st->l1_refresh, &l1, sizeof l1, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        return bail(fail(ctx, RLGL_ECUDA, "state init failed"));
    if ((s = read_state(ctx)) != RLGL_OK) return bail(s);
    *out = ctx;
    return RLGL_OK;
}

rlgl_status rlgl_batch_create(int64_t n_chains, const int64_t* node_ptr, int64_t n, int64_t nnz,
                              const int64_t* row_ptr, const int32_t* col, const float* w,
                              rlgl_precision prec, rlgl_memspace src, void* stream, rlgl_ctx** out) {
    if (!out) return fail(nullptr, RLGL_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_chains < 1 || n_chains > (1ll << 30) || !node_ptr)
        return fail(nullptr, RLGL_EINVAL, "n_chains out of range or node_ptr NULL");
    std::vector<int64_t> np((size_t)n_chains + 1);
    if (src == RLGL_DEVICE) {
        if (cudaMemcpy(np.data(), node_ptr, np.size() * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(nullptr, RLGL_ECUDA, "reading node_ptr failed");
    } else {
        memcpy(np.data(), node_ptr, np.size() * sizeof(int64_t));
    }
    if (np[0] != 0 || np[(size_t)n_chains] != n) return fail(nullptr, RLGL_EINVAL, "node_ptr must run from 0 to n");
    for (int64_t k = 0; k < n_chains; ++k)
        if (np[(size_t)k + 1] <= np[(size_t)k]) return fail(nullptr, RLGL_EINVAL, "chain %lld is empty", (long long)k);
    rlgl_ctx* ctx = nullptr;
    rlgl_status s = create_common(n, nnz, row_ptr, col, w, prec, src, stream, &ctx);
    auto bail = [&](rlgl_status st) {
        if (ctx) snprintf(g_thread_err, sizeof g_thread_err, "%s", ctx->err_msg);
        rlgl_destroy(ctx);
        return st;
    };
    if (s != RLGL_OK) return bail(s);
    ctx->nchains = (int)n_chains;
    ctx->node_ptr_h = np;
    // the push chunk index of a batch holds every chain's own part
    // (chain k's chunks start at its first link / kPushChunk + k)
    dfree(ctx, ctx->chunk_row);
    ctx->chunk_row = nullptr;
    if ((s = dalloc(ctx, &ctx->chunk_row, (size_t)(nnz / kPushChunk + n_chains + 2))) != RLGL_OK) return bail(s);
    if ((s = dalloc(ctx, &ctx->node_ptr, (size_t)n_chains + 1)) != RLGL_OK) return bail(s);
    if ((s = dalloc(ctx, &ctx->chain_of, (size_t)n)) != RLGL_OK) return bail(s);
    if ((s = dalloc(ctx, &ctx->cs, (size_t)n_chains)) != RLGL_OK) return bail(s);
    if ((s = dalloc(ctx, &ctx->bsums, 2 * (size_t)n_chains)) != RLGL_OK) return bail(s);
    std::vector<ChainState> cs((size_t)n_chains);
    memset(cs.data(), 0, cs.size() * sizeof(ChainState));
    for (int64_t k = 0; k < n_chains; ++k) {
        cs[(size_t)k].n = np[(size_t)k + 1] - np[(size_t)k];
        cs[(size_t)k].tol = 1e-12;
    }
    if (cudaMemcpyAsync(ctx->node_ptr, np.data(), np.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(ctx->cs, cs.data(), cs.size() * sizeof(ChainState), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess)
        return bail(fail(ctx, RLGL_ECUDA, "upload of chain data failed"));
    k_chain_of<<<grid_for(n, kThreads, ctx->sms * 16), kThreads, 0, ctx->stream>>>(ctx->node_ptr, (int)n_chains, n,
                                                                                  ctx->chain_of);
    unsigned int zero = 0, err = 0;
    if (cudaMemcpyAsync(ctx->err, &zero, sizeof zero, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        return bail(fail(ctx, RLGL_ECUDA, "memset failed"));
    k_check_blocks<<<grid_for(n * 32, kThreads, ctx->sms * 16), kThreads, 0, ctx->stream>>>(
        ctx->row_ptr, ctx->col, ctx->chain_of, n, ctx->err);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&err, ctx->err, sizeof err, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return bail(fail(ctx, RLGL_ECUDA, "chain map failed"));
    if (err) return bail(fail(ctx, RLGL_EINVAL, "an edge leaves its chain: the CSR must be block-diagonal"));
    {
        // each chain's links (row_ptr at the chain boundaries), for the
        // persistent batch's work queue
        long long* eb = nullptr;
        if ((s = dalloc(ctx, &eb, (size_t)n_chains + 1)) != RLGL_OK) return bail(s);
        k_gather_rows<<<grid_for(n_chains + 1, kThreads, 1024), kThreads, 0, ctx->stream>>>(
            ctx->row_ptr, ctx->node_ptr, n_chains + 1, eb);
        std::vector<long long> ebh((size_t)n_chains + 1);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(ebh.data(), eb, ebh.size() * sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            dfree(ctx, eb);
            return bail(fail(ctx, RLGL_ECUDA, "reading the chains' link offsets failed"));
        }
        dfree(ctx, eb);
        ctx->chain_nnz_h.resize((size_t)n_chains);
        for (int64_t k = 0; k < n_chains; ++k) ctx->chain_nnz_h[(size_t)k] = ebh[(size_t)k + 1] - ebh[(size_t)k];
    }
    if ((s = set_step0(ctx, nullptr, RLGL_HOST)) != RLGL_OK) return bail(s);  // uniform per chain
    *out = ctx;
    return RLGL_OK;
}

rlgl_status rlgl_batch_set_tol(rlgl_ctx* ctx, const double* tol) {
    if (!ctx || !tol) return fail(ctx, RLGL_EINVAL, "NULL argument");
    if (ctx->nchains < 2) return fail(ctx, RLGL_EINVAL, "not a batch");
    std::vector<ChainState> cs((size_t)ctx->nchains);
    CK(ctx, cudaMemcpyAsync(cs.data(), ctx->cs, cs.size() * sizeof(ChainState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < ctx->nchains; ++k) {
        if (!(tol[k] >= 0.0)) return fail(ctx, RLGL_EINVAL, "tol[%d] < 0", k);
        cs[(size_t)k].tol = tol[k];
    }
    CK(ctx, cudaMemcpyAsync(ctx->cs, cs.data(), cs.size() * sizeof(ChainState), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return RLGL_OK;
}

rlgl_status rlgl_batch_chains(rlgl_ctx* ctx, int32_t* status, int64_t* moves, double* resid) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    if (ctx->nchains < 2) return fail(ctx, RLGL_EINVAL, "not a batch");
    std::vector<ChainState> cs((size_t)ctx->nchains);
    CK(ctx, cudaMemcpyAsync(cs.data(), ctx->cs, cs.size() * sizeof(ChainState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < ctx->nchains; ++k) {
        const ChainState& c = cs[(size_t)k];
        if (status) status[k] = c.done ? c.status : -1;
        if (moves) moves[k] = c.moves;
        if (resid) resid[k] = c.hsum != 0.0 ? c.l1 / fabs(c.hsum) : INFINITY;
    }
    return RLGL_OK;
}

rlgl_status rlgl_reset(rlgl_ctx* ctx, const double* m0, rlgl_memspace src) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    NOT_PENDING(ctx);
    return set_step0(ctx, m0, src);  // NULL: uniform (within each chain of a batch)
}

rlgl_status rlgl_set_masks(rlgl_ctx* ctx, const uint8_t* masks, int64_t period, rlgl_memspace src) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    NOT_PENDING(ctx);
    if (!masks || period < 1) return fail(ctx, RLGL_EINVAL, "masks is NULL or period < 1");
    if (ctx->masks) { dfree(ctx, ctx->masks); ctx->masks = nullptr; }
    TRY(dalloc(ctx, &ctx->masks, (size_t)(period * ctx->n)));
    TRY(upload(ctx, ctx->masks, masks, (size_t)(period * ctx->n), src));
    ctx->n_masks = period;
    static const long long zero = 0;
    CK(ctx, cudaMemcpyAsync(&ctx->st->mask_cursor, &zero, sizeof zero, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);  // captured launches hold the mask pointer
    return RLGL_OK;
}

static rlgl_status check_sched(rlgl_ctx* ctx, rlgl_schedule sched) {
    if (sched < RLGL_ALL_GREEN || sched > RLGL_PC)
        return fail(ctx, RLGL_EINVAL, "bad schedule %d", (int)sched);
    if ((sched == RLGL_TOPFRAC || sched == RLGL_BLOCK_RR || sched == RLGL_PC) && ctx->nchains > 1)
        return fail(ctx, RLGL_EINVAL, "schedule %d is not available for a batch of chains", (int)sched);
    if (sched == RLGL_MASK && !ctx->masks) return fail(ctx, RLGL_EINVAL, "RLGL_MASK needs rlgl_set_masks");
    return RLGL_OK;
}

rlgl_status rlgl_step(rlgl_ctx* ctx, rlgl_schedule sched, double theta, rlgl_step_info* info) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    NOT_PENDING(ctx);
    TRY(check_sched(ctx, sched));
    TRY(begin(ctx, sched, theta, 0.0, 1, 0));
    TRY(iteration(ctx, false, sched, 0ull, 0));
    if (info) {
        TRY(read_state(ctx));
        DevState* h = ctx->host_st;
        info->green = h->green;
        info->edges_pushed = h->edges;
        info->mode = h->mode;
        info->theta = h->theta;
        // statistics of the new cash
        TRY(begin(ctx, sched, theta, 0.0, 1, 0));
        Launch L{ctx, false};
        if (ctx->prec == RLGL_MIXED)
            LAUNCH(L, KC_STATS, (k_stats<float><<<ctx->grid_stats, kThreads, 0, ctx->stream>>>(
                                    (const float*)ctx->c, (const float*)ctx->ideg, (int)ctx->n, ctx->st, ctx->part, 0ull, 0ull, 0,
                                    vec_aligned(ctx))));
        else
            LAUNCH(L, KC_STATS, (k_stats<double><<<ctx->grid_stats, kThreads, 0, ctx->stream>>>(
                                    (const double*)ctx->c, (const double*)ctx->ideg, (int)ctx->n, ctx->st, ctx->part, 0ull, 0ull, 0,
                                    vec_aligned(ctx))));
        TRY(read_state(ctx));
        info->l1_cash = h->l1;
        info->sum_cash = h->sum;
        info->sum_hist = h->hsum;
    }
    return RLGL_OK;
}

}  // extern "C"

// Captures what `body` enqueues into graph g after the nodes deps; returns
// the leaf nodes of the capture in *leaves (when given).
template <typename F>
static rlgl_status capture_into(rlgl_ctx* ctx, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                                F&& body, std::vector<cudaGraphNode_t>* leaves) {
    CK(ctx, cudaStreamBeginCaptureToGraph(ctx->stream, g, deps, nullptr, nd,
                                          cudaStreamCaptureModeRelaxed));
    rlgl_status s = body();
    if (s == RLGL_OK && leaves) {
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* d = nullptr;
        size_t n = 0;
        cudaError_t e = cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, nullptr, &d, nullptr, &n);
        if (e == cudaSuccess) leaves->assign(d, d + n);
        else s = fail(ctx, RLGL_ECUDA, "cudaStreamGetCaptureInfo: %s", cudaGetErrorString(e));
    }
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &out);
    if (s != RLGL_OK) return s;
    CK(ctx, e);
    return RLGL_OK;
}

// Adds a conditional node (type, `size` bodies) to g after deps.
static rlgl_status add_conditional(rlgl_ctx* ctx, cudaGraph_t g, const cudaGraphNode_t* deps,
                                   size_t nd, cudaGraphConditionalHandle h,
                                   cudaGraphConditionalNodeType type, unsigned size,
                                   cudaGraphNode_t* node, cudaGraph_t* bodies) {
    // cudaGraphNodeParams holds a union without a default constructor:
    // build it in zeroed storage.
    alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
    memset(pbuf, 0, sizeof pbuf);
    cudaGraphNodeParams* p = reinterpret_cast<cudaGraphNodeParams*>(pbuf);
    p->type = cudaGraphNodeTypeConditional;
    p->conditional.handle = h;
    p->conditional.type = type;
    p->conditional.size = size;
    CK(ctx, cudaGraphAddNode(node, g, deps, nullptr, nd, p));
    for (unsigned k = 0; k < size; ++k) bodies[k] = p->conditional.phGraph_out[k];
    return RLGL_OK;
}

// The solve graph: WHILE(loop) { [IF(refresh) {re-derive C}] stats [top-k]
// select IF/ELSE(mode) {pull} {push} }. k_stats ends the loop and requests
// the refresh of the next iteration; k_select picks pull or push.
template <typename T>
static rlgl_status build_graph_t(rlgl_ctx* ctx, int sched, cudaGraph_t g) {
    Conds cd;
    cd.use = 1;
    cudaGraphConditionalHandle hw;
    CK(ctx, cudaGraphConditionalHandleCreate(&hw, g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNode_t wnode;
    cudaGraph_t body;
    TRY(add_conditional(ctx, g, nullptr, 0, hw, cudaGraphCondTypeWhile, 1, &wnode, &body));
    cd.loop = (unsigned long long)hw;
    cudaGraphConditionalHandle hr = 0, hm;
    CK(ctx, cudaGraphConditionalHandleCreate(&hm, body, 0u, cudaGraphCondAssignDefault));
    cd.mode = (unsigned long long)hm;
    std::vector<cudaGraphNode_t> deps;
    Launch L{ctx, true};
    if (ctx->prec == RLGL_MIXED) {
        CK(ctx, cudaGraphConditionalHandleCreate(&hr, body, 0u, cudaGraphCondAssignDefault));
        cd.refresh = (unsigned long long)hr;
        cudaGraphNode_t rnode;
        cudaGraph_t rbody;
        TRY(add_conditional(ctx, body, nullptr, 0, hr, cudaGraphCondTypeIf, 1, &rnode, &rbody));
        TRY(capture_into(ctx, rbody, nullptr, 0, [&] { return enqueue_refresh<T>(L); }, nullptr));
        deps.push_back(rnode);
    }
    std::vector<cudaGraphNode_t> leaves;
    TRY(capture_into(ctx, body, deps.data(), deps.size(),
                     [&] { return enqueue_head<T>(L, sched, cd); }, &leaves));
    cudaGraphNode_t mnode;
    cudaGraph_t mbody[2];
    TRY(add_conditional(ctx, body, leaves.data(), leaves.size(), hm, cudaGraphCondTypeIf, 2, &mnode,
                        mbody));
    TRY(capture_into(ctx, mbody[0], nullptr, 0, [&] { return enqueue_pull<T>(L); }, nullptr));
    TRY(capture_into(ctx, mbody[1], nullptr, 0, [&] { return enqueue_push<T>(L); }, nullptr));
    return RLGL_OK;
}

// The sweep's solve graph: WHILE(loop) { [IF(refresh) {re-derive C}] sweep }.
// The sweep ends the loop when the solve stops and requests the
// re-derivation when it returns for one. power: the all-green sweep.
template <typename T>
static rlgl_status build_sweep_graph_t(rlgl_ctx* ctx, cudaGraph_t g, bool power) {
    Conds cd;
    cd.use = 1;
    cudaGraphConditionalHandle hw;
    CK(ctx, cudaGraphConditionalHandleCreate(&hw, g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNode_t wnode;
    cudaGraph_t body;
    TRY(add_conditional(ctx, g, nullptr, 0, hw, cudaGraphCondTypeWhile, 1, &wnode, &body));
    cd.loop = (unsigned long long)hw;
    std::vector<cudaGraphNode_t> deps;
    Launch L{ctx, true};
    if (ctx->prec == RLGL_MIXED) {
        cudaGraphConditionalHandle hr;
        CK(ctx, cudaGraphConditionalHandleCreate(&hr, body, 0u, cudaGraphCondAssignDefault));
        cd.refresh = (unsigned long long)hr;
        cudaGraphNode_t rnode;
        cudaGraph_t rbody;
        TRY(add_conditional(ctx, body, nullptr, 0, hr, cudaGraphCondTypeIf, 1, &rnode, &rbody));
        TRY(capture_into(ctx, rbody, nullptr, 0, [&] { return enqueue_refresh<T>(L); }, nullptr));
        deps.push_back(rnode);
    }
    TRY(capture_into(ctx, body, deps.data(), deps.size(),
                     [&] { return power ? enqueue_power<T>(L, cd) : enqueue_sweep<T>(L, cd); }, nullptr));
    return RLGL_OK;
}

static rlgl_status build_sweep_graph(rlgl_ctx* ctx, bool power) {
    cudaGraph_t g = nullptr;
    CK(ctx, cudaGraphCreate(&g, 0));
    rlgl_status s = (ctx->prec == RLGL_MIXED) ? build_sweep_graph_t<float>(ctx, g, power)
                                              : build_sweep_graph_t<double>(ctx, g, power);
    if (s != RLGL_OK) {
        cudaGraphDestroy(g);
        return s;
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    CK(ctx, e);
    (power ? ctx->power_graph : ctx->sweep_graph) = exec;
    return RLGL_OK;
}

// Whether a batch solve runs as the persistent batch kernel.
static bool use_bsweep(const rlgl_ctx* ctx, int sched) {
    return ctx->params.persistent && ctx->nchains > 1 && sched != RLGL_TOPFRAC && !ctx->params.theta_lag;
}

// The persistent batch's per-chain tiles (for its block size) and work
// queue: chains sorted by size (rows + links), largest first; chain k gets
// g_k = ceil(w_k / W) blocks (W = the batch's work over the grid), at most
// 16 and at most its tiles, and the groups of more than one block together
// take no more than the grid, so all of them start at once.
static rlgl_status batch_prepare(rlgl_ctx* ctx) {
    const int bt = ctx->params.batch_block;
    const long long items = (long long)bt * mp_ipt(bt);
    const int nc = ctx->nchains;
    if (ctx->ct_items != items) {
        if (!ctx->ct_off) TRY(dalloc(ctx, &ctx->ct_off, (size_t)nc + 1));
        CK(ctx, cudaMemsetAsync(ctx->ct_off, 0, ((size_t)nc + 1) * sizeof(long long), ctx->stream));
        k_chain_tile_counts<<<grid_for(nc, kThreads, 1024), kThreads, 0, ctx->stream>>>(ctx->node_ptr, ctx->t_ptr, nc,
                                                                                      items, ctx->ct_off);
        CKL(ctx);
        TRY(device_inclusive_scan(ctx, ctx->ct_off, (long long)nc + 1));
        long long total = 0;
        CK(ctx, cudaMemcpyAsync(&total, ctx->ct_off + nc, sizeof total, cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->ct_r) { dfree(ctx, ctx->ct_r); ctx->ct_r = nullptr; }
        if (ctx->ct_e) { dfree(ctx, ctx->ct_e); ctx->ct_e = nullptr; }
        TRY(dalloc(ctx, &ctx->ct_r, (size_t)total));
        TRY(dalloc(ctx, &ctx->ct_e, (size_t)total));
        k_chain_tiles<<<grid_for(total, kThreads, ctx->sms * 8), kThreads, 0, ctx->stream>>>(
            ctx->node_ptr, ctx->t_ptr, ctx->ct_off, nc, items, ctx->ct_r, ctx->ct_e);
        CKL(ctx);
        ctx->ct_items = items;
    }
    if (ctx->bq_block != bt) {
        const int nb = bsweep_fit(ctx, bt);
        if (nb < 1) return fail(ctx, RLGL_ECUDA, "the persistent batch kernel does not fit on an SM");
        const long long G = (long long)nb * ctx->sms;
        std::vector<double> wk((size_t)nc);
        double W = 0.0;
        for (int k = 0; k < nc; ++k) {
            wk[(size_t)k] = (double)(ctx->node_ptr_h[(size_t)k + 1] - ctx->node_ptr_h[(size_t)k]) +
                            (double)ctx->chain_nnz_h[(size_t)k];
            W += wk[(size_t)k];
        }
        W = W / (double)G;
        if (W < 1.0) W = 1.0;
        std::vector<int> order((size_t)nc), g((size_t)nc);
        for (int k = 0; k < nc; ++k) {
            order[(size_t)k] = k;
            long long gk = (long long)ceil(wk[(size_t)k] / W);
            const long long tiles = (long long)ceil(wk[(size_t)k] / (double)items);
            if (gk > 16) gk = 16;
            if (gk > tiles) gk = tiles;
            if (gk < 1) gk = 1;
            g[(size_t)k] = (int)gk;
        }
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return wk[(size_t)x] > wk[(size_t)y]; });
        for (;;) {
            long long multi = 0;
            for (int k = 0; k < nc; ++k)
                if (g[(size_t)k] > 1) multi += g[(size_t)k];
            if (multi <= G) break;
            for (int k = 0; k < nc; ++k)
                if (g[(size_t)k] > 1) g[(size_t)k] /= 2;
        }
        long long E = 0;
        for (int k = 0; k < nc; ++k) E += g[(size_t)k];
        std::vector<int> q((size_t)(2 * E + nc));
        long long e = 0;
        for (int k : order)
            for (int m = 0; m < g[(size_t)k]; ++m) {
                q[(size_t)e] = k;
                q[(size_t)(E + e)] = m;
                ++e;
            }
        for (int k = 0; k < nc; ++k) q[(size_t)(2 * E + k)] = g[(size_t)k];
        if (ctx->bq) { CK(ctx, cudaStreamSynchronize(ctx->stream)); dfree(ctx, ctx->bq); ctx->bq = nullptr; }
        TRY(dalloc(ctx, &ctx->bq, q.size()));
        CK(ctx, cudaMemcpyAsync(ctx->bq, q.data(), q.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        ctx->q_len = E;
        ctx->grid_batch = (int)(E < G ? E : G);
        ctx->bq_block = bt;
        if (ctx->batch_graph) {
            cudaGraphExecDestroy(ctx->batch_graph);
            ctx->batch_graph = nullptr;
        }
    }
    if (!ctx->grp) TRY(dalloc(ctx, &ctx->grp, (size_t)nc));
    if (!ctx->q_next) TRY(dalloc(ctx, &ctx->q_next, 1));
    return RLGL_OK;
}

// The persistent batch's solve graph: clear the groups and the queue
// counter, take the start time, the batch kernel, the totals.
template <typename T>
static rlgl_status enqueue_batch_solve(rlgl_ctx* ctx) {
    CK(ctx, cudaMemsetAsync(ctx->grp, 0, (size_t)ctx->nchains * sizeof(BGroup), ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->q_next, 0, sizeof(unsigned long long), ctx->stream));
    k_bstart<<<1, 1, 0, ctx->stream>>>(ctx->st);
    CKL(ctx);
    TRY(enqueue_bsweep<T>(ctx));
    k_bfinish<<<1, kThreads, 0, ctx->stream>>>(ctx->st, ctx->cs, ctx->nchains);
    CKL(ctx);
    return RLGL_OK;
}

static rlgl_status build_batch_graph(rlgl_ctx* ctx) {
    cudaGraph_t g = nullptr;
    CK(ctx, cudaGraphCreate(&g, 0));
    rlgl_status s = capture_into(ctx, g, nullptr, 0, [&] {
        return ctx->prec == RLGL_MIXED ? enqueue_batch_solve<float>(ctx) : enqueue_batch_solve<double>(ctx);
    }, nullptr);
    if (s != RLGL_OK) {
        cudaGraphDestroy(g);
        return s;
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    CK(ctx, e);
    ctx->batch_graph = exec;
    return RLGL_OK;
}

static rlgl_status build_graph(rlgl_ctx* ctx, int sched) {
    cudaGraph_t g = nullptr;
    CK(ctx, cudaGraphCreate(&g, 0));
    rlgl_status s = (ctx->prec == RLGL_MIXED) ? build_graph_t<float>(ctx, sched, g)
                                              : build_graph_t<double>(ctx, sched, g);
    if (s != RLGL_OK) {
        cudaGraphDestroy(g);
        return s;
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    CK(ctx, e);
    ctx->graph[sched] = exec;
    return RLGL_OK;
}

extern "C" {

static rlgl_status solve_launch(rlgl_ctx* ctx, rlgl_schedule sched, double theta, double tol,
                                int64_t max_steps) {
    TRY(check_sched(ctx, sched));
    if (max_steps < 1 || max_steps > 100000000ll) return fail(ctx, RLGL_EINVAL, "max_steps out of range");
    const bool batch_tols = ctx->nchains > 1 && tol < 0.0;  // per-chain tolerances
    if (!(tol >= 0.0) && !batch_tols) return fail(ctx, RLGL_EINVAL, "tol must be >= 0");
    bool sweep = use_sweep(ctx, sched);
    const bool power = use_power(ctx, sched);
    cudaGraphExec_t& sg = power ? ctx->power_graph : ctx->sweep_graph;
    if (sweep && !sg && build_sweep_graph(ctx, power) != RLGL_OK) {
        // The device or driver would not take the cooperative kernel into a
        // graph: use one kernel per phase from now on (params.persistent
        // then reads 0, and rlgl_last_error keeps the reason).
        ctx->params.persistent = 0;
        ctx->grid_sweep = 0;
        ctx->grid_power = 0;
        sweep = false;
        cudaGetLastError();
    }
    if (!sweep && ctx->params.theta_lag)
        return fail(ctx, RLGL_EINVAL,
                    "theta_lag needs the persistent sweep and a threshold schedule (not TOPFRAC, batches or "
                    "persistent = 0)");
    const bool bsweep = use_bsweep(ctx, sched);
    if (bsweep) {
        TRY(batch_prepare(ctx));
        if (!ctx->batch_graph) TRY(build_batch_graph(ctx));
    } else if (!sweep && !ctx->graph[sched]) {
        TRY(build_graph(ctx, sched));
    }
    TRY(begin(ctx, sched, theta, batch_tols ? 0.0 : tol, max_steps, 1, batch_tols ? -1.0 : tol));
    if (sweep) CK(ctx, cudaMemsetAsync(ctx->sw, 0, sizeof(SweepState), ctx->stream));
    CK(ctx, cudaGraphLaunch(bsweep ? ctx->batch_graph : (sweep ? sg : ctx->graph[sched]), ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->host_st, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaEventRecord(ctx->done_ev, ctx->stream));
    ctx->pending = true;
    ctx->pending_max = max_steps;
    return RLGL_OK;
}

static rlgl_status solve_finish(rlgl_ctx* ctx, rlgl_solve_info* info) {
    ctx->pending = false;
    CK(ctx, cudaEventSynchronize(ctx->done_ev));
    const DevState* h = ctx->host_st;
    if (info) {
        info->moves = h->solve_moves;
        info->edges_pushed = h->tot_edges - h->base_edges;
        info->green_total = h->tot_green - h->base_green;
        info->push_moves = h->push_moves - h->base_push;
        info->pull_moves = h->pull_moves - h->base_pull;
        info->refreshes = h->refreshes - h->base_refreshes;
        info->iterations = h->iters;
        info->resid = h->hsum != 0.0 ? h->l1 / fabs(h->hsum) : INFINITY;
        info->l1_cash = h->l1;
        info->sum_hist = h->hsum;
    }
    switch (h->status) {
        case ST_OK: return RLGL_OK;
        case ST_DEGENERATE: return fail(ctx, RLGL_EDEGENERATE, "degenerate history: |H 1| ~ 0");
        case ST_NOCONV: return fail(ctx, RLGL_ENOCONV, "no convergence in %lld moves", ctx->pending_max);
        case ST_TIMEOUT: return fail(ctx, RLGL_ETIMEOUT, "solve exceeded its time limit");
        case ST_BARRIER:
            return fail(ctx, RLGL_ETIMEOUT, "a grid-barrier wait of the persistent sweep gave up");
        default: return fail(ctx, RLGL_ECUDA, "unexpected device status %d", h->status);
    }
}

rlgl_status rlgl_solve(rlgl_ctx* ctx, rlgl_schedule sched, double theta, double tol,
                       int64_t max_steps, rlgl_solve_info* info) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    NOT_PENDING(ctx);
    TRY(solve_launch(ctx, sched, theta, tol, max_steps));
    return solve_finish(ctx, info);
}

rlgl_status rlgl_solve_async(rlgl_ctx* ctx, rlgl_schedule sched, double theta, double tol,
                             int64_t max_steps) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    NOT_PENDING(ctx);
    return solve_launch(ctx, sched, theta, tol, max_steps);
}

rlgl_status rlgl_query(rlgl_ctx* ctx, int32_t* finished) {
    if (!ctx || !finished) return fail(ctx, RLGL_EINVAL, "NULL argument");
    if (!ctx->pending) {
        *finished = 1;
        return RLGL_OK;
    }
    cudaError_t e = cudaEventQuery(ctx->done_ev);
    if (e == cudaErrorNotReady) {
        *finished = 0;
        return RLGL_OK;
    }
    CK(ctx, e);
    *finished = 1;
    return RLGL_OK;
}

rlgl_status rlgl_wait(rlgl_ctx* ctx, rlgl_solve_info* info) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    if (!ctx->pending) return fail(ctx, RLGL_EINVAL, "no asynchronous solve to wait for");
    return solve_finish(ctx, info);
}

static rlgl_status batch_estimate(rlgl_ctx* ctx, double* pi_out, rlgl_memspace dst) {
    const int n = (int)ctx->n;
    const BatchView bv{ctx->chain_of, ctx->cs, ctx->nchains};
    k_bhist_sums<<<ctx->grid_select, kThreads, 0, ctx->stream>>>(ctx->H, n, bv);
    k_bhist_finish<<<grid_for(ctx->nchains, kThreads, 1024), kThreads, 0, ctx->stream>>>(bv, 0, ctx->bsums);
    CKL(ctx);
    std::vector<double> sums(2 * (size_t)ctx->nchains);
    CK(ctx, cudaMemcpyAsync(sums.data(), ctx->bsums, sums.size() * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    int bad = -1;
    for (int k = 0; k < ctx->nchains; ++k)
        if (!(fabs(sums[2 * k]) > 1e-12 * sums[2 * k + 1]) || sums[2 * k + 1] == 0.0) { bad = k; break; }
    if (bad >= 0) return fail(ctx, RLGL_EDEGENERATE, "degenerate history in chain %d", bad);
    double* out = (dst == RLGL_HOST) ? ctx->hsrc : pi_out;
    k_bscale<<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(ctx->H, n, ctx->chain_of, ctx->bsums, out);
    CKL(ctx);
    if (dst == RLGL_HOST)
        CK(ctx, cudaMemcpyAsync(pi_out, out, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return RLGL_OK;
}

// pi_i = H_i / sum_{k in [lo, hi)} H_k for i in [lo, hi), into pi_out[i - lo].
static rlgl_status estimate_range(rlgl_ctx* ctx, long long lo, long long hi, double* pi_out,
                                  rlgl_memspace dst) {
    const int m = (int)(hi - lo);
    const double* H = ctx->H + lo;
    k_hist_sums<<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(H, m, ctx->st, ctx->part, 0);
    CKL(ctx);
    double sums[2];
    CK(ctx, cudaMemcpyAsync(sums, ctx->part + 2 * kMaxGrid, sizeof sums, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (!(fabs(sums[0]) > 1e-12 * sums[1]) || sums[1] == 0.0)
        return fail(ctx, RLGL_EDEGENERATE, "degenerate history: H 1 = %g, sum|H| = %g", sums[0], sums[1]);
    double* out = pi_out;
    if (dst == RLGL_HOST) out = ctx->hsrc;  // staging (all scratch, rewritten before use)
    k_scale<<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>(H, m, ctx->part + 2 * kMaxGrid, out);
    CKL(ctx);
    if (dst == RLGL_HOST)
        CK(ctx, cudaMemcpyAsync(pi_out, out, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return RLGL_OK;
}

rlgl_status rlgl_estimate(rlgl_ctx* ctx, double* pi_out, rlgl_memspace dst) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    if (!pi_out) return fail(ctx, RLGL_EINVAL, "pi_out is NULL");
    if (dst != RLGL_HOST && dst != RLGL_DEVICE) return fail(ctx, RLGL_EINVAL, "bad memspace");
    NOT_PENDING(ctx);
    if (ctx->nchains > 1) return batch_estimate(ctx, pi_out, dst);
    return estimate_range(ctx, 0, ctx->n, pi_out, dst);
}

rlgl_status rlgl_estimate_range(rlgl_ctx* ctx, int64_t lo, int64_t hi, double* pi_out, rlgl_memspace dst) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    if (!pi_out) return fail(ctx, RLGL_EINVAL, "pi_out is NULL");
    if (dst != RLGL_HOST && dst != RLGL_DEVICE) return fail(ctx, RLGL_EINVAL, "bad memspace");
    if (ctx->nchains > 1) return fail(ctx, RLGL_EINVAL, "rlgl_estimate_range serves single chains");
    if (lo < 0 || hi > ctx->n || lo >= hi)
        return fail(ctx, RLGL_EINVAL, "node range [%lld, %lld) not inside [0, %lld)", (long long)lo,
                    (long long)hi, ctx->n);
    NOT_PENDING(ctx);
    return estimate_range(ctx, lo, hi, pi_out, dst);
}

rlgl_status rlgl_get_state(rlgl_ctx* ctx, double* c, double* h, rlgl_memspace dst) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    NOT_PENDING(ctx);
    const int n = (int)ctx->n;
    if (c) {
        double* out = (dst == RLGL_HOST) ? ctx->hsrc : c;
        if (ctx->prec == RLGL_MIXED)
            k_to_double<float><<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>((const float*)ctx->c, n, out);
        else
            k_to_double<double><<<ctx->grid_nodes, kThreads, 0, ctx->stream>>>((const double*)ctx->c, n, out);
        CKL(ctx);
        if (dst == RLGL_HOST)
            CK(ctx, cudaMemcpyAsync(c, out, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (h)
        CK(ctx, cudaMemcpyAsync(h, ctx->H, (size_t)n * sizeof(double),
                                dst == RLGL_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return RLGL_OK;
}

rlgl_status rlgl_invariant_residual(rlgl_ctx* ctx, double* l1) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    NOT_PENDING(ctx);
    TRY(forced_refresh(ctx, false));
    TRY(read_state(ctx));
    if (l1) *l1 = ctx->host_st->resid_l1;
    return RLGL_OK;
}

rlgl_status rlgl_refresh(rlgl_ctx* ctx, double* l1_before) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    NOT_PENDING(ctx);
    TRY(forced_refresh(ctx, true));
    TRY(read_state(ctx));
    if (l1_before) *l1_before = ctx->host_st->resid_l1;
    return RLGL_OK;
}

rlgl_status rlgl_set_params(rlgl_ctx* ctx, const rlgl_params* p) {
    if (!ctx || !p) return fail(ctx, RLGL_EINVAL, "NULL argument");
    if (!(p->theta_scale > 0.0) || p->r < 1 || !(p->top_frac > 0.0 && p->top_frac <= 1.0) ||
        !(p->pull_crossover >= 0.0) || p->safety_every < 0 || !(p->refresh_factor >= 0.0 && p->refresh_factor < 1.0) ||
        !(p->time_limit_s > 0.0) || (p->persistent != 0 && p->persistent != 1) || p->rr_blocks < 1 ||
        !(p->pc_frac > 0.0 && p->pc_frac <= 1e30) || !(p->barrier_limit_s > 0.0 && p->barrier_limit_s <= 60.0) ||
        (p->test_skip_barrier != 0 && p->test_skip_barrier != 1) || p->stall_moves < 0 ||
        (p->theta_lag != 0 && p->theta_lag != 1) ||
        (p->batch_block != 128 && p->batch_block != 256 && p->batch_block != 512))
        return fail(ctx, RLGL_EINVAL, "parameter out of range");
    ctx->params = *p;
    return RLGL_OK;
}

rlgl_status rlgl_get_params(const rlgl_ctx* ctx, rlgl_params* p) {
    if (!ctx || !p) return RLGL_EINVAL;
    *p = ctx->params;
    return RLGL_OK;
}

rlgl_status rlgl_profile(rlgl_ctx* ctx, int32_t mode) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    if (mode == 2) {
        TRY(prof_collect(ctx));
        for (int i = 0; i < KC_N; ++i) { ctx->prof_ms[i] = 0.0; ctx->prof_n[i] = 0; }
        return RLGL_OK;
    }
    ctx->profiling = mode ? 1 : 0;
    return RLGL_OK;
}

rlgl_status rlgl_kernel_times(rlgl_ctx* ctx, double* ms, int64_t* launches) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    TRY(prof_collect(ctx));
    for (int i = 0; i < KC_N; ++i) {
        if (ms) ms[i] = ctx->prof_ms[i];
        if (launches) launches[i] = ctx->prof_n[i];
    }
    return RLGL_OK;
}

namespace {
// Holds the stream until the host has queued a batch of launches (bounded
// wait: gives up after 30 s, the stream then simply continues).
struct Gate {
    std::atomic<int> open{0};
};
void CUDART_CB gate_wait(void* p) {
    Gate* g = static_cast<Gate*>(p);
    auto t0 = std::chrono::steady_clock::now();
    while (!g->open.load(std::memory_order_acquire)) {
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(30)) break;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}
}  // namespace

rlgl_status rlgl_profile_moves(rlgl_ctx* ctx, rlgl_schedule sched, double theta, int64_t moves) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    NOT_PENDING(ctx);
    TRY(check_sched(ctx, sched));
    if (moves < 0) return fail(ctx, RLGL_EINVAL, "moves < 0");
    const int prev = ctx->profiling;
    ctx->profiling = 1;
    TRY(begin(ctx, sched, theta, 0.0, moves > 0 ? moves : 1, 0));
    const int64_t batch = 16;
    rlgl_status s = RLGL_OK;
    for (int64_t m0 = 0; m0 < moves && s == RLGL_OK; m0 += batch) {
        Gate gate;
        CK(ctx, cudaLaunchHostFunc(ctx->stream, gate_wait, &gate));
        for (int64_t m = m0; m < moves && m < m0 + batch && s == RLGL_OK; ++m)
            s = iteration(ctx, false, sched, 0ull, 0);
        gate.open.store(1, std::memory_order_release);
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    ctx->profiling = prev;
    if (s != RLGL_OK) return s;
    return prof_collect(ctx);
}

}  // extern "C"

template <typename T>
static rlgl_status profile_sweep_t(rlgl_ctx* ctx, int64_t moves, bool power) {
    Launch L{ctx, false};
    Conds none;
    // every launch makes at least one move or ends the solve
    for (int64_t k = 0; k < moves + 4; ++k) {
        TRY(enqueue_refresh<T>(L));  // runs only when a re-derivation is pending
        if (power) TRY(enqueue_power<T>(L, none));
        else TRY(enqueue_sweep<T>(L, none));
        TRY(read_state(ctx));
        if (ctx->host_st->done) break;
    }
    return RLGL_OK;
}

extern "C" {

rlgl_status rlgl_profile_sweep(rlgl_ctx* ctx, rlgl_schedule sched, double theta, int64_t moves) {
    if (!ctx) return fail(nullptr, RLGL_EINVAL, "ctx is NULL");
    NOT_PENDING(ctx);
    TRY(check_sched(ctx, sched));
    if (moves < 1 || moves > 100000000ll) return fail(ctx, RLGL_EINVAL, "moves out of range");
    if (!use_sweep(ctx, sched))
        return fail(ctx, RLGL_EINVAL, "the persistent sweep does not serve this schedule or context");
    const int prev = ctx->profiling;
    ctx->profiling = 1;
    TRY(begin(ctx, sched, theta, 0.0, moves, 1));
    CK(ctx, cudaMemsetAsync(ctx->sw, 0, sizeof(SweepState), ctx->stream));
    const bool power = use_power(ctx, sched);
    rlgl_status s = ctx->prec == RLGL_MIXED ? profile_sweep_t<float>(ctx, moves, power)
                                            : profile_sweep_t<double>(ctx, moves, power);
    ctx->profiling = prev;
    if (s != RLGL_OK) return s;
    return prof_collect(ctx);
}

rlgl_status rlgl_move_log(rlgl_ctx* ctx, rlgl_move_record* out, int64_t count, int64_t* written) {
    if (!ctx || !out || count < 0) return fail(ctx, RLGL_EINVAL, "bad argument");
    static_assert(sizeof(rlgl_move_record) == sizeof(MoveRecord), "log record layout");
    TRY(read_state(ctx));
    long long total = ctx->host_st->moves;
    long long have = total < kLogCap ? total : kLogCap;
    long long k = count < have ? count : have;
    for (long long i = 0; i < k; ++i) {
        long long mv = total - k + i;
        CK(ctx, cudaMemcpyAsync(out + i, ctx->log + (mv % kLogCap), sizeof(MoveRecord),
                                cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (written) *written = k;
    return RLGL_OK;
}

int64_t rlgl_release_retired(void) {
    std::vector<cudaGraphExec_t> v;
    {
        std::lock_guard<std::mutex> lk(g_retired_mu);
        v.swap(g_retired);
    }
    for (auto g : v) cudaGraphExecDestroy(g);
    return (int64_t)v.size();
}

int64_t rlgl_footprint(int64_t n, int64_t nnz, int32_t weighted, rlgl_precision prec,
                       int64_t n_chains) {
    if (n < 1 || nnz < 1) return -1;
    const int64_t cs = prec == RLGL_MIXED ? 4 : 8;
    const int64_t ntiles = (n + nnz + kMpItems - 1) / kMpItems;
    const int64_t witems = 32 * power_ipt((int)cs);
    const int64_t nwtiles = (n + nnz + witems - 1) / witems;
    int64_t b = 0;
    b += 2 * ((n + 1) * 8 + nnz * 4 + (weighted ? nnz * 4 : 0));  // CSR and CSC
    b += n * (8 + (prec == RLGL_MIXED ? 4 : 0) + cs);                // s, sf, 1/deg
    b += 2 * (ntiles + 1) * 8 + 2 * (nwtiles + 1) * 8;               // merge-path tiles (block, warp)
    b += n * (cs + 8 + cs + 8 + 8 + 8 + 8 + cs + 8);                 // c H mt y hsrc f_eoff f_base f_m colsum
    b += (nnz / kPushChunk + 2) * 4;                                 // chunk index
    b += (4 * kMaxGrid + 8) * 8 + 8 + (int64_t)kLogCap * (int64_t)sizeof(MoveRecord) +
         (int64_t)sizeof(DevState) + (int64_t)sizeof(SweepState);
    if (n_chains > 1) b += (n_chains + 1) * 8 + n * 4 + n_chains * ((int64_t)sizeof(ChainState) + 16);
    return b;
}

void* rlgl_stream(const rlgl_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

const char* rlgl_last_error(const rlgl_ctx* ctx) { return ctx ? ctx->err_msg : g_thread_err; }

const char* rlgl_status_string(rlgl_status s) {
    switch (s) {
        case RLGL_OK: return "RLGL_OK";
        case RLGL_EINVAL: return "RLGL_EINVAL";
        case RLGL_ENOTSTOCHASTIC: return "RLGL_ENOTSTOCHASTIC";
        case RLGL_ENOMEM: return "RLGL_ENOMEM";
        case RLGL_ECUDA: return "RLGL_ECUDA";
        case RLGL_EDEGENERATE: return "RLGL_EDEGENERATE";
        case RLGL_ENOCONV: return "RLGL_ENOCONV";
        case RLGL_ETIMEOUT: return "RLGL_ETIMEOUT";
    }
    return "unknown status";
}

void rlgl_destroy(rlgl_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto& e : ctx->prof) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    {
        std::lock_guard<std::mutex> lk(g_retired_mu);
        for (auto& g : ctx->graph)
            if (g) g_retired.push_back(g);
        if (ctx->sweep_graph) g_retired.push_back(ctx->sweep_graph);
        if (ctx->power_graph) g_retired.push_back(ctx->power_graph);
        if (ctx->batch_graph) g_retired.push_back(ctx->batch_graph);
    }
    void* dev[] = {ctx->row_ptr, ctx->col, ctx->w, ctx->s, ctx->sf, ctx->ideg, ctx->t_ptr, ctx->t_src, ctx->t_w,
                   ctx->tile_r, ctx->tile_e, ctx->wtile_r, ctx->wtile_e, ctx->c, ctx->H, ctx->mt, ctx->y, ctx->hsrc, ctx->c0,
                   ctx->colsum,
                   ctx->f_eoff, ctx->f_base, ctx->f_m, ctx->chunk_row, ctx->part, ctx->masks,
                   ctx->err, ctx->log, ctx->st, ctx->sw, ctx->node_ptr, ctx->chain_of, ctx->cs,
                   ctx->bsums, ctx->ct_off, ctx->ct_r, ctx->ct_e, ctx->grp, ctx->bq, ctx->q_next, ctx->hubs};
    for (void* p : dev)
        dfree(ctx, p);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->done_ev) cudaEventDestroy(ctx->done_ev);
    pin_put(ctx->host_st);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

}  // extern "C"
