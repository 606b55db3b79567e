// bv_kmeans.cu -- K-means blocks on the GPU (Sec. 2.1; Algorithm 1 "Clustering").
//
// The paper names K-means without fixing its details; this library fixes them so the
// blocks are a deterministic function of (locations, k, seed, iterations), identical
// bit for bit to the plain definition:
//   * squared distance D2(x, c) = sum_k (x_k - c_k)^2, left to right, every -, * and +
//     rounded separately (no fused multiply-add);
//   * k-means++ seeding (Arthur and Vassilvitskii 2007): first centre = point
//     floor(r_0 n / 2^64); centre t is drawn with probability proportional to D2 to the
//     nearest chosen centre, on integer weights w_j = floor(D2_j 2^s) with s fixed from n
//     and the bounding box (sum w < 2^62): target = floor(r_t W / 2^64), the pick is the
//     first point whose inclusive prefix sum of w exceeds the target (W = 0: point
//     floor(r_t n / 2^64));
//   * Lloyd iterations: nearest centre with the lowest index on ties; centre = mean of its
//     members computed as ((double)S / count) 2^-q from the exact int64 sum S of
//     llrint(x 2^q); an empty cluster keeps its centre; a final assignment after the last
//     update gives the labels.
// r_t = SplitMix64 draw t of stream BV_STREAM_KPP(seed).
//
// GPU formulation.  The assignment scans all centres with FP32 arithmetic to find, per
// point, the smallest FP32 squared distance d32min; every centre whose FP32 distance is
// within a proven rounding margin of d32min is then re-scored with the exact FP64 rule.
// The margin bounds |d32 - D2| (coordinate rounding to FP32, the subtraction, the
// squares and the sum), so the exact minimiser is always among the re-scored centres.
// Centroid sums are exact integers (order-free atomics), so the update is bit-exact.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "bv_internal.h"

namespace {

// Exact squared distance, no contraction.
__device__ __forceinline__ double d2_exact(const double* x, const double* c, int d) {
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = __dsub_rn(x[k], c[k]);
        acc = __dadd_rn(acc, __dmul_rn(t, t));
    }
    return acc;
}

// Upper bound on |d32 - D2| for a squared distance whose FP32 value is about v, with
// coordinates bounded by amax in magnitude (derivation in the design notes: coordinate
// rounding eta = 1.01 u (|x|+|c|+|t|) <= 4.04 u amax per axis, error of the squares
// eta (2|t| + eta), FP32 sum rounding (d+1) u v; all doubled for safety).
__device__ __forceinline__ float fp32_margin(float v, float amax, int d) {
    const float u = 5.9604645e-8f;  // 2^-24
    const float eta = 4.04f * u * amax;
    const float D = sqrtf(fmaxf(v, 0.0f)) + 2.0f * eta;
    const float e = sqrtf((float)d) * eta * (2.0f * D + eta) + (float)(d + 2) * u * (v + 1e-30f);
    return 4.0f * e + 1e-30f;
}

constexpr int kTile = 256;  // centres per shared-memory tile

// Lloyd assignment.  x: SoA FP64 points [d][n_tot] (this dataset's slice at `off`),
// cent: row-major FP64 centres [k][d].  One thread per point.
__global__ void __launch_bounds__(256) k_assign(const double* __restrict__ locs, int64_t n_tot,
                                                int64_t off, int64_t n, int d,
                                                const double* __restrict__ cent, int64_t k,
                                                float amax, int32_t* __restrict__ label) {
    __shared__ float4 cf[kTile];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool live = i < n;
    double x[3] = {0.0, 0.0, 0.0};
    float xf[3] = {0.f, 0.f, 0.f};
    if (live)
        for (int q = 0; q < d; ++q) {
            x[q] = locs[(int64_t)q * n_tot + off + i];
            xf[q] = (float)x[q];
        }
    // pass 1: FP32 minimum
    float best32 = INFINITY;
    for (int64_t c0 = 0; c0 < k; c0 += kTile) {
        const int nt = (int)min((int64_t)kTile, k - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < nt; t += blockDim.x) {
            const double* cc = cent + (c0 + t) * d;
            cf[t] = make_float4((float)cc[0], d > 1 ? (float)cc[1] : 0.f, d > 2 ? (float)cc[2] : 0.f, 0.f);
        }
        __syncthreads();
        for (int t = 0; t < nt; ++t) {
            const float4 c = cf[t];
            const float a0 = xf[0] - c.x, a1 = xf[1] - c.y, a2 = xf[2] - c.z;
            const float v = fmaf(a2, a2, fmaf(a1, a1, a0 * a0));
            best32 = fminf(best32, v);
        }
    }
    const float thr = best32 + 2.0f * fp32_margin(best32 * 1.001f, amax, d);
    // pass 2: exact FP64 score of every centre inside the margin; strict < keeps the
    // lowest index among equal distances because centres are visited in index order
    double best = INFINITY;
    int32_t bi = 0;
    for (int64_t c0 = 0; c0 < k; c0 += kTile) {
        const int nt = (int)min((int64_t)kTile, k - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < nt; t += blockDim.x) {
            const double* cc = cent + (c0 + t) * d;
            cf[t] = make_float4((float)cc[0], d > 1 ? (float)cc[1] : 0.f, d > 2 ? (float)cc[2] : 0.f, 0.f);
        }
        __syncthreads();
        for (int t = 0; t < nt; ++t) {
            const float4 c = cf[t];
            const float a0 = xf[0] - c.x, a1 = xf[1] - c.y, a2 = xf[2] - c.z;
            const float v = fmaf(a2, a2, fmaf(a1, a1, a0 * a0));
            if (v <= thr) {
                const double e = d2_exact(x, cent + (c0 + t) * d, d);
                if (e < best) {
                    best = e;
                    bi = (int32_t)(c0 + t);
                }
            }
        }
    }
    if (live) label[i] = bi;
}

// Exact integer centroid sums.
__global__ void k_accum(const double* __restrict__ locs, int64_t n_tot, int64_t off, int64_t n,
                        int d, const int32_t* __restrict__ label, int q,
                        unsigned long long* __restrict__ S, unsigned long long* __restrict__ cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t c = label[i];
    atomicAdd(cnt + c, 1ull);
    for (int k = 0; k < d; ++k) {
        const long long v = llrint(ldexp(locs[(int64_t)k * n_tot + off + i], q));
        atomicAdd(S + c * d + k, (unsigned long long)v);
    }
}

__global__ void k_finalize(const unsigned long long* __restrict__ S,
                           const unsigned long long* __restrict__ cnt, int64_t k, int d, int q,
                           double* __restrict__ cent, int64_t* __restrict__ counts) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= k) return;
    const unsigned long long nc = cnt[c];
    if (counts) counts[c] = (int64_t)nc;
    if (nc == 0) return;
    for (int j = 0; j < d; ++j) {
        const long long s = (long long)S[c * d + j];
        cent[c * d + j] = ldexp(__ll2double_rn(s) / __ull2double_rn(nc), -q);
    }
}

// ---- k-means++ ---------------------------------------------------------------------
constexpr int kChunk = 1024;  // points per seeding chunk (one CTA)

// D2 <- min(D2, D2(x, c_new)) (or init), and exact per-chunk weight sums.
__global__ void __launch_bounds__(kChunk) k_kpp_update(const double* __restrict__ locs,
                                                       int64_t n_tot, int64_t off, int64_t n,
                                                       int d, const double* __restrict__ cnew,
                                                       int init, int s, double* __restrict__ D2,
                                                       unsigned long long* __restrict__ chunk_sum) {
    __shared__ unsigned long long red[kChunk / 32];
    const int64_t i = blockIdx.x * (int64_t)kChunk + threadIdx.x;
    unsigned long long w = 0;
    if (i < n) {
        double x[3];
        for (int q = 0; q < d; ++q) x[q] = locs[(int64_t)q * n_tot + off + i];
        const double v = d2_exact(x, cnew, d);
        double cur = init ? v : D2[i];
        if (!init && v < cur) cur = v;
        D2[i] = cur;
        w = (unsigned long long)ldexp(cur, s);
    }
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int j = 0; j < kChunk / 32; ++j) t += red[j];
        chunk_sum[blockIdx.x] = t;
    }
}

// Inclusive scan of one value per thread over a kChunk-thread block (exact integers).
__device__ __forceinline__ unsigned long long block_incl_scan(unsigned long long v,
                                                              unsigned long long* sh) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        unsigned long long x = lane < kChunk / 32 ? sh[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane < kChunk / 32) sh[lane] = x;
    }
    __syncthreads();
    const unsigned long long r = v + (w > 0 ? sh[w - 1] : 0ull);
    __syncthreads();
    return r;
}

// Pick centre t: the first point whose inclusive prefix weight exceeds the target.  One
// CTA: scan of the chunk sums (in pieces of kChunk) to find the chunk, then a scan of
// that chunk's weights.
__global__ void __launch_bounds__(kChunk) k_kpp_pick(const double* __restrict__ locs,
                                                     int64_t n_tot, int64_t off, int64_t n, int d,
                                                     const double* __restrict__ D2, int s,
                                                     const unsigned long long* __restrict__ chunk_sum,
                                                     int64_t nchunks, uint64_t stream, int64_t t,
                                                     double* __restrict__ cent_t) {
    __shared__ unsigned long long sh[kChunk / 32];
    __shared__ unsigned long long s_base, s_total;
    __shared__ long long s_chunk, s_pick;
    const int tid = threadIdx.x;
    // exact total weight
    unsigned long long part = 0;
    for (int64_t c = tid; c < nchunks; c += kChunk) part += chunk_sum[c];
    const unsigned long long tot = block_incl_scan(part, sh);
    if (tid == kChunk - 1) s_total = tot;
    if (tid == 0) {
        s_pick = -1;
        s_chunk = -1;
    }
    __syncthreads();
    const unsigned long long W = s_total;
    const uint64_t r = bv_sm64(stream, (uint64_t)t);
    if (W == 0) {
        if (tid == 0) s_pick = (long long)__umul64hi(r, (uint64_t)n);
        __syncthreads();
    } else {
        const unsigned long long target = __umul64hi(r, W);
        unsigned long long base = 0;
        for (int64_t c0 = 0; c0 < nchunks; c0 += kChunk) {
            const int64_t c = c0 + tid;
            const unsigned long long v = c < nchunks ? chunk_sum[c] : 0ull;
            const unsigned long long inc = block_incl_scan(v, sh) + base;
            const unsigned long long exc = inc - v;
            if (c < nchunks && inc > target && exc <= target) {
                s_chunk = c;
                s_base = exc;
            }
            __syncthreads();
            if (s_chunk >= 0) break;
            // base for the next piece: inclusive value of the last thread
            if (tid == kChunk - 1) s_base = inc;
            __syncthreads();
            base = s_base;
            __syncthreads();
        }
        // s_chunk is always found (target < W); the clamps only keep indices in range
        const long long ch = s_chunk >= 0 ? s_chunk : nchunks - 1;
        const unsigned long long rem = s_chunk >= 0 ? target - s_base : 0ull;
        const int64_t i = ch * kChunk + tid;
        const unsigned long long w = i < n ? (unsigned long long)ldexp(D2[i], s) : 0ull;
        const unsigned long long inc = block_incl_scan(w, sh);
        if (i < n && inc > rem && inc - w <= rem) s_pick = (long long)i;
        __syncthreads();
    }
    __syncthreads();
    const long long pick = (s_pick >= 0 && s_pick < n) ? s_pick : n - 1;
    if (tid < d) cent_t[tid] = locs[(int64_t)tid * n_tot + off + pick];
}

}  // namespace

static int ceil_log2_u64(uint64_t v) {
    int e = 0;
    while (e < 64 && ((uint64_t)1 << e) < v) ++e;
    return e;
}

int bv_kmeans_scales(const double* h, int64_t n, int d, int* s_out, int* q_out) {
    double lo[3], hi[3];
    for (int k = 0; k < d; ++k) lo[k] = hi[k] = h[k];
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < d; ++k) {
            const double v = h[i * d + k];
            lo[k] = std::min(lo[k], v);
            hi[k] = std::max(hi[k], v);
        }
    double d2max = 0.0, amax = 0.0;
    for (int k = 0; k < d; ++k) {
        const double e = hi[k] - lo[k];
        d2max += e * e;
        amax = std::max(amax, std::max(fabs(lo[k]), fabs(hi[k])));
    }
    int ed = 0, ea = 0;
    frexp(d2max, &ed);
    frexp(amax, &ea);
    const int ln = ceil_log2_u64((uint64_t)n);
    *s_out = 61 - ln - (ed + 1);
    *q_out = 61 - ln - (ea + 1);
    return BV_OK;
}

int bv_centroids_device(const double* d_locs, int64_t n_tot, int64_t off, int64_t n, int d,
                        const int32_t* d_label, int64_t k, int q, double* d_cent,
                        int64_t* d_counts, cudaStream_t s) {
    unsigned long long *S = nullptr, *cnt = nullptr;
    BV_CUDA(cudaMallocAsync(&S, sizeof(unsigned long long) * k * d, s));
    BV_CUDA(cudaMallocAsync(&cnt, sizeof(unsigned long long) * k, s));
    BV_CUDA(cudaMemsetAsync(S, 0, sizeof(unsigned long long) * k * d, s));
    BV_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * k, s));
    k_accum<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_locs, n_tot, off, n, d, d_label, q, S, cnt);
    BV_CUDA(cudaGetLastError());
    k_finalize<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(S, cnt, k, d, q, d_cent, d_counts);
    BV_CUDA(cudaGetLastError());
    BV_CUDA(cudaFreeAsync(S, s));
    BV_CUDA(cudaFreeAsync(cnt, s));
    return BV_OK;
}

// Full K-means of one dataset (points [off, off+n) of the SoA array): seeding, `iters`
// Lloyd iterations and the final assignment.  d_label[n] and d_cent[k x d] are outputs.
int bv_kmeans_device(const double* d_locs, int64_t n_tot, int64_t off, int64_t n, int d,
                     int64_t k, uint64_t seed, int iters, int32_t* d_label, double* d_cent,
                     cudaStream_t s) {
    // scales and the coordinate bound from a host copy of this slice
    std::vector<double> h((size_t)n * d);
    {
        std::vector<double> col((size_t)n);
        for (int q = 0; q < d; ++q) {
            BV_CUDA(cudaMemcpyAsync(col.data(), d_locs + (int64_t)q * n_tot + off, sizeof(double) * n,
                                    cudaMemcpyDeviceToHost, s));
            BV_CUDA(cudaStreamSynchronize(s));
            for (int64_t i = 0; i < n; ++i) h[(size_t)i * d + q] = col[(size_t)i];
        }
    }
    int sc = 0, q = 0;
    bv_kmeans_scales(h.data(), n, d, &sc, &q);
    double amax = 0.0;
    for (double v : h) amax = std::max(amax, fabs(v));

    const uint64_t stream = BV_STREAM_KPP(seed);
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    double* D2 = nullptr;
    unsigned long long* csum = nullptr;
    BV_CUDA(cudaMallocAsync(&D2, sizeof(double) * n, s));
    BV_CUDA(cudaMallocAsync(&csum, sizeof(unsigned long long) * nchunks, s));
    // first centre
    {
        const uint64_t r0 = bv_sm64(stream, 0);
        const int64_t first = (int64_t)(((unsigned __int128)r0 * (unsigned __int128)(uint64_t)n) >> 64);
        for (int q2 = 0; q2 < d; ++q2)
            BV_CUDA(cudaMemcpyAsync(d_cent + q2, d_locs + (int64_t)q2 * n_tot + off + first, sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
    }
    for (int64_t t = 1; t < k; ++t) {
        k_kpp_update<<<(unsigned)nchunks, kChunk, 0, s>>>(d_locs, n_tot, off, n, d, d_cent + (t - 1) * d,
                                                          t == 1, sc, D2, csum);
        BV_CUDA(cudaGetLastError());
        k_kpp_pick<<<1, kChunk, 0, s>>>(d_locs, n_tot, off, n, d, D2, sc, csum, nchunks, stream, t,
                                        d_cent + t * d);
        BV_CUDA(cudaGetLastError());
    }
    BV_CUDA(cudaFreeAsync(D2, s));
    BV_CUDA(cudaFreeAsync(csum, s));
    // Lloyd
    const unsigned gp = (unsigned)((n + 255) / 256);
    for (int it = 0; it < iters; ++it) {
        k_assign<<<gp, 256, 0, s>>>(d_locs, n_tot, off, n, d, d_cent, k, (float)amax, d_label);
        BV_CUDA(cudaGetLastError());
        BV_TRY(bv_centroids_device(d_locs, n_tot, off, n, d, d_label, k, q, d_cent, nullptr, s));
    }
    k_assign<<<gp, 256, 0, s>>>(d_locs, n_tot, off, n, d, d_cent, k, (float)amax, d_label);
    BV_CUDA(cudaGetLastError());
    return BV_OK;
}
