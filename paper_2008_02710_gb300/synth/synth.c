/*
 * Seeded synthetic Markov-chain inputs (edge lists and CSR).
 *
 * This file holds input generation only: it draws graphs and raw edge
 * weights and lays them out as CSR. It does no step of the RLGL method
 * (no normalisation to transition probabilities, no cash, no history).
 *
 * Random numbers come from a counter-based generator: value(seed, stream, i)
 * is the SplitMix64 output function (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) applied to a key derived from
 * (seed, stream) and the counter i. Every draw depends only on its counter,
 * so results are identical on any machine and for any thread count.
 *
 * Only integer arithmetic decides graph structure; edge weights are
 * k * 2^-24 with k uniform on 1..2^24, which is exact in FP32.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

/* SplitMix64 output function. */
static inline uint64_t sm_mix(uint64_t z) {
    z += GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t rnd_key(uint64_t seed, uint64_t stream) {
    return sm_mix(sm_mix(seed) ^ (stream * 0xD1B54A32D192ED03ULL));
}

static inline uint64_t rnd_at(uint64_t key, uint64_t i) {
    return sm_mix(key + i * GOLDEN);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double unit_at(uint64_t key, uint64_t i) {
    return (double)(rnd_at(key, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* Uniform weight in (0, 1] on the grid k * 2^-24, exact in FP32. */
static inline float weight_at(uint64_t key, uint64_t i) {
    uint64_t k = (rnd_at(key, i) >> 40) + 1u; /* 1 .. 2^24 */
    return (float)((double)k * (1.0 / 16777216.0));
}

enum {
    S_DEG = 1, S_TGT = 2, S_W = 3, S_RMAT = 4, S_PERM = 5, S_POIS = 6,
    S_SIZE = 7, S_DELTA = 8, S_PL = 9, S_USER = 100
};

uint64_t synth_u64(uint64_t seed, uint64_t stream, uint64_t i) {
    return rnd_at(rnd_key(seed, stream), i);
}

double synth_unit(uint64_t seed, uint64_t stream, uint64_t i) {
    return unit_at(rnd_key(seed, stream), i);
}

/*
 * Tiny directed chain: node i gets d_i ~ U{1..8} out-edges to uniform
 * targets (with replacement; duplicates are kept and their weights add),
 * then the edge i -> (i+1) mod n and the self-loop i -> i. Every edge gets a
 * weight U(0,1]. Writes at most 10 n edges; returns the count.
 */
int64_t synth_tiny_edges(int64_t n, uint64_t seed, int32_t* src, int32_t* dst,
                         float* w, int64_t cap) {
    uint64_t kd = rnd_key(seed, S_DEG), kt = rnd_key(seed, S_TGT), kw = rnd_key(seed, S_W);
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t d = 1 + (int64_t)(rnd_at(kd, (uint64_t)i) % 8u);
        for (int64_t k = 0; k < d + 2; ++k) {
            if (m >= cap) return -1;
            int64_t j;
            if (k < d) j = (int64_t)(rnd_at(kt, (uint64_t)(i * 8 + k)) % (uint64_t)n);
            else if (k == d) j = (i + 1) % n;
            else j = i;
            src[m] = (int32_t)i;
            dst[m] = (int32_t)j;
            w[m] = weight_at(kw, (uint64_t)(i * 10 + k));
            ++m;
        }
    }
    return m;
}

/*
 * R-MAT edges (Chakrabarti, Zhan, Faloutsos 2004): for each of the `scale`
 * bit levels, pick a quadrant with probabilities (a, b, c, 1-a-b-c) and set
 * the source/destination bit accordingly (a: 0/0, b: 0/1, c: 1/0, d: 1/1).
 * No noise. Self-loops and duplicates are kept.
 */
void synth_rmat_edges(int32_t scale, int64_t m, double a, double b, double c,
                      uint64_t seed, int32_t* src, int32_t* dst) {
    uint64_t key = rnd_key(seed, S_RMAT);
    double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t u = 0, v = 0;
        for (int32_t l = 0; l < scale; ++l) {
            double r = unit_at(key, (uint64_t)e * (uint64_t)scale + (uint64_t)l);
            uint32_t bit = 1u << (scale - 1 - l);
            if (r < a) {
            } else if (r < ab) {
                v |= bit;
            } else if (r < abc) {
                u |= bit;
            } else {
                u |= bit;
                v |= bit;
            }
        }
        src[e] = (int32_t)u;
        dst[e] = (int32_t)v;
    }
}

/*
 * R-MAT edges on n nodes (n need not be a power of two): generated at scale
 * ceil(log2 n); an edge with an endpoint >= n is drawn again from the next
 * sub-stream (at most 64 times, then its endpoints are folded mod n).
 */
void synth_rmat_edges_n(int64_t n, int64_t m, double a, double b, double c, uint64_t seed,
                        int32_t* src, int32_t* dst) {
    int32_t scale = 0;
    while ((1ll << scale) < n) ++scale;
    if (scale == 0) scale = 1;
    double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t u = 0, v = 0;
        for (int attempt = 0; attempt < 64; ++attempt) {
            uint64_t key = rnd_key(seed, S_RMAT + 1000u * (uint64_t)attempt);
            u = 0;
            v = 0;
            for (int32_t l = 0; l < scale; ++l) {
                double r = unit_at(key, (uint64_t)e * (uint64_t)scale + (uint64_t)l);
                uint32_t bit = 1u << (scale - 1 - l);
                if (r < a) {
                } else if (r < ab) {
                    v |= bit;
                } else if (r < abc) {
                    u |= bit;
                } else {
                    u |= bit;
                    v |= bit;
                }
            }
            if ((int64_t)u < n && (int64_t)v < n) break;
        }
        src[e] = (int32_t)((int64_t)u % n);
        dst[e] = (int32_t)((int64_t)v % n);
    }
}

/* Seeded uniform random permutation of 0..n-1 (Fisher-Yates). */
void synth_permutation(int64_t n, uint64_t seed, int32_t* perm) {
    uint64_t key = rnd_key(seed, S_PERM);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)(rnd_at(key, (uint64_t)i) % (uint64_t)(i + 1));
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

/* Relabel both endpoints of m edges through perm (in place). */
void synth_relabel(int64_t m, const int32_t* perm, int32_t* src, int32_t* dst) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        src[e] = perm[src[e]];
        dst[e] = perm[dst[e]];
    }
}

/* m weights U(0,1] on the 2^-24 grid from the given stream. */
void synth_weights(int64_t m, uint64_t seed, uint64_t stream, float* w) {
    uint64_t key = rnd_key(seed, S_USER + stream);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) w[e] = weight_at(key, (uint64_t)e);
}

/* Appends the cycle i -> (i+1) mod n and the self-loop i -> i: 2n edges. */
void synth_cycle_selfloops(int64_t n, int32_t* src, int32_t* dst) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        src[2 * i] = (int32_t)i;
        dst[2 * i] = (int32_t)((i + 1) % n);
        src[2 * i + 1] = (int32_t)i;
        dst[2 * i + 1] = (int32_t)i;
    }
}

/*
 * Stable counting sort of an edge list by source into CSR. Within a row the
 * edges keep their order in the input list. w may be NULL (then wout is
 * ignored). Returns 0, or -1 if an endpoint is out of range.
 */
int synth_to_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                 const float* w, int64_t* row_ptr, int32_t* col, float* wout) {
    memset(row_ptr, 0, (size_t)(n + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -1;
        row_ptr[src[e] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
    int64_t* cur = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!cur) return -2;
    memcpy(cur, row_ptr, (size_t)n * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        int64_t p = cur[src[e]]++;
        col[p] = dst[e];
        if (w) wout[p] = w[e];
    }
    free(cur);
    return 0;
}

/*
 * One chain of the many-chain mix: n nodes, per-node out-degree
 * Poisson(delta) (inverse transform), targets drawn from a power law
 * P(rank r) proportional to 1/(r+1) over a seeded permutation of the nodes,
 * then the cycle and the self-loop. Node ids are local (0..n-1).
 * Returns the number of edges written (at most cap), or -1 if cap is short.
 */
int64_t synth_powerlaw_chain_edges(int64_t n, double delta, uint64_t seed,
                                   int32_t* src, int32_t* dst, int64_t cap) {
    uint64_t kp = rnd_key(seed, S_POIS), kt = rnd_key(seed, S_PL);
    int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    double* cdf = (double*)malloc((size_t)n * sizeof(double));
    if (!perm || !cdf) { free(perm); free(cdf); return -2; }
    synth_permutation(n, seed ^ 0x5bd1e995ULL, perm);
    double acc = 0.0;
    for (int64_t r = 0; r < n; ++r) { acc += 1.0 / (double)(r + 1); cdf[r] = acc; }
    int64_t m = 0;
    double emd = exp(-delta);
    for (int64_t i = 0; i < n; ++i) {
        /* Poisson(delta) by inverse transform on one uniform draw. */
        double u = unit_at(kp, (uint64_t)i), p = emd, s = p;
        int64_t d = 0;
        while (u > s && d < 10000) { ++d; p *= delta / (double)d; s += p; }
        for (int64_t k = 0; k < d; ++k) {
            if (m >= cap) { free(perm); free(cdf); return -1; }
            double x = unit_at(kt, (uint64_t)i * 4096u + (uint64_t)k) * acc;
            int64_t lo = 0, hi = n - 1;
            while (lo < hi) { int64_t mid = (lo + hi) / 2; if (cdf[mid] > x) hi = mid; else lo = mid + 1; }
            src[m] = (int32_t)i;
            dst[m] = perm[lo];
            ++m;
        }
        if (m + 2 > cap) { free(perm); free(cdf); return -1; }
        src[m] = (int32_t)i; dst[m] = (int32_t)((i + 1) % n); ++m;
        src[m] = (int32_t)i; dst[m] = (int32_t)i; ++m;
    }
    free(perm);
    free(cdf);
    return m;
}

/*
 * A batch of independent power-law chains written straight into one
 * block-diagonal CSR, in three passes so that the caller can size the
 * arrays: sizes (node_ptr), out-degrees (row_ptr), then targets (col).
 * Chain k has n_k = floor(exp(U(ln lo, ln hi))) nodes and mean out-degree
 * delta_k ~ U(dlo, dhi); node i draws Poisson(delta_k) targets from a power
 * law P(rank r) proportional to 1/(r+1) over a seeded permutation of the
 * chain, then gets the cycle edge and the self-loop. Node ids are global.
 */
static void batch_chain_params(uint64_t seed, int64_t k, double lo, double hi, double dlo,
                               double dhi, int64_t* n, double* delta) {
    double u = unit_at(rnd_key(seed, S_SIZE), (uint64_t)k);
    double v = unit_at(rnd_key(seed, S_DELTA), (uint64_t)k);
    *n = (int64_t)floor(exp(log(lo) + u * (log(hi) - log(lo))));
    if (*n < 2) *n = 2;
    *delta = dlo + v * (dhi - dlo);
}

static int64_t poisson_at(uint64_t key, uint64_t i, double delta) {
    double u = unit_at(key, i), p = exp(-delta), s = p;
    int64_t d = 0;
    while (u > s && d < 100000) { ++d; p *= delta / (double)d; s += p; }
    return d;
}

int64_t synth_batch_sizes(int64_t nchains, uint64_t seed, double lo, double hi, double dlo,
                          double dhi, int64_t* node_ptr) {
    node_ptr[0] = 0;
    for (int64_t k = 0; k < nchains; ++k) {
        int64_t n;
        double d;
        batch_chain_params(seed, k, lo, hi, dlo, dhi, &n, &d);
        node_ptr[k + 1] = node_ptr[k] + n;
    }
    return node_ptr[nchains];
}

int64_t synth_batch_degrees(int64_t nchains, uint64_t seed, double lo, double hi, double dlo,
                            double dhi, const int64_t* node_ptr, int64_t* row_ptr) {
    uint64_t kp = rnd_key(seed, S_POIS);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < nchains; ++k) {
        int64_t n;
        double delta;
        batch_chain_params(seed, k, lo, hi, dlo, dhi, &n, &delta);
        for (int64_t i = node_ptr[k]; i < node_ptr[k + 1]; ++i)
            row_ptr[i + 1] = poisson_at(kp, (uint64_t)i, delta) + 2;
    }
    row_ptr[0] = 0;
    int64_t N = node_ptr[nchains];
    for (int64_t i = 0; i < N; ++i) row_ptr[i + 1] += row_ptr[i];
    return row_ptr[N];
}

int synth_batch_fill(int64_t nchains, uint64_t seed, const int64_t* node_ptr,
                     const int64_t* row_ptr, int32_t* col) {
    uint64_t kt = rnd_key(seed, S_PL);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < nchains; ++k) {
        const int64_t base = node_ptr[k], n = node_ptr[k + 1] - base;
        int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        double* cdf = (double*)malloc((size_t)n * sizeof(double));
        if (!perm || !cdf) {
            free(perm);
            free(cdf);
#pragma omp atomic write
            err = 1;
            continue;
        }
        synth_permutation(n, seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(k + 1)), perm);
        double acc = 0.0;
        for (int64_t r = 0; r < n; ++r) { acc += 1.0 / (double)(r + 1); cdf[r] = acc; }
        for (int64_t i = 0; i < n; ++i) {
            const int64_t gi = base + i, a = row_ptr[gi], d = row_ptr[gi + 1] - a - 2;
            for (int64_t q = 0; q < d; ++q) {
                double x = unit_at(kt, (uint64_t)(a + q)) * acc;
                int64_t lo = 0, hi = n - 1;
                while (lo < hi) { int64_t mid = (lo + hi) / 2; if (cdf[mid] > x) hi = mid; else lo = mid + 1; }
                col[a + q] = (int32_t)(base + perm[lo]);
            }
            col[a + d] = (int32_t)(base + (i + 1) % n);
            col[a + d + 1] = (int32_t)gi;
        }
        free(perm);
        free(cdf);
    }
    return err ? -1 : 0;
}
