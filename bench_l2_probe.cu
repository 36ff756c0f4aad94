// Random-access rate probe: the ceiling against which the sweep's push and
// pull phases are measured. The chain of an R-MAT 20 solve lives in L2, so
// its moves are bound not by HBM bandwidth but by how many random 4-byte
// reductions (push) or loads (pull) the memory system completes per second.
// These two kernels do nothing else: m updates or loads at pseudo-random
// indices of an n-word array (indices from a xorshift sequence, all in
// range), grid-stride, 256 threads per block, each thread issuing eight
// independent accesses per pass. m must be large enough for the rate to be
// the steady state: with 4 M accesses (about 20 us) the launch's ramp and
// tail took a quarter of the time (210 G gathers/s against 290 G/s at 64 M).
//
// Built by bench.py into libbench_l2_probe.so beside it: measurement only,
// not part of the RLGL library.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kU = 8;  // independent accesses per thread and pass

__global__ void probe_scatter(float* __restrict__ c, const int* __restrict__ idx, long long m) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; k + (kU - 1) * stride < m; k += kU * stride) {
        int j[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) j[u] = __ldcs(idx + k + u * stride);
#pragma unroll
        for (int u = 0; u < kU; ++u)
            asm volatile("red.global.add.f32 [%0], %1;" ::"l"(c + j[u]), "f"(1.0f) : "memory");
    }
    for (; k < m; k += stride) asm volatile("red.global.add.f32 [%0], %1;" ::"l"(c + idx[k]), "f"(1.0f) : "memory");
}

__global__ void probe_gather(const float* __restrict__ c, const int* __restrict__ idx, long long m,
                             float* __restrict__ out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float s = 0.f;
    for (; k + (kU - 1) * stride < m; k += kU * stride) {
        int j[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) j[u] = __ldcs(idx + k + u * stride);
        float v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) v[u] = __ldcg(c + j[u]);
#pragma unroll
        for (int u = 0; u < kU; ++u) s += v[u];
    }
    for (; k < m; k += stride) s += __ldcg(c + idx[k]);
    if (s == -1.f) out[0] = s;  // keeps the loads
}

__global__ void probe_indices(int* idx, long long m, int n, unsigned long long seed) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x) {
        unsigned long long x = seed ^ (0x9E3779B97F4A7C15ull * (unsigned long long)(k + 1));
        x ^= x >> 33;
        x *= 0xFF51AFD7ED558CCDull;
        x ^= x >> 33;
        idx[k] = (int)(x % (unsigned long long)n);
    }
}

}  // namespace

// Best rate (G operations/s) over `reps` timed launches of the scatter
// (kind 0: red.global.add.f32) or the gather (kind 1: ld.global.cg) of m
// random accesses into n words, on the current device and default stream.
// Returns a negative value on a CUDA error. Allocates and frees its own
// buffers (n + m words).
extern "C" double l2_probe_rate(int kind, int n, long long m, int grid, int reps) {
    if (n < 1 || m < 1 || grid < 1 || reps < 1) return -1.0;
    float* c = nullptr;
    int* idx = nullptr;
    float* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    double best = -1.0;
    if (cudaMalloc(&c, (size_t)n * sizeof(float)) != cudaSuccess) return -1.0;
    if (cudaMalloc(&idx, (size_t)m * sizeof(int)) != cudaSuccess || cudaMalloc(&out, sizeof(float)) != cudaSuccess)
        goto done;
    cudaMemset(c, 0, (size_t)n * sizeof(float));
    probe_indices<<<1024, 256>>>(idx, m, n, 12345ull);
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int r = 0; r < reps + 1; ++r) {
        cudaEventRecord(a);
        if (kind == 0) probe_scatter<<<grid, 256>>>(c, idx, m);
        else probe_gather<<<grid, 256>>>(c, idx, m, out);
        cudaEventRecord(b);
        if (cudaEventSynchronize(b) != cudaSuccess) { best = -1.0; goto done; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double rate = (double)m / (ms * 1e-3) / 1e9;
        if (r > 0 && rate > best) best = rate;  // the first launch warms up
    }
done:
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(c);
    cudaFree(idx);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return best;
}
