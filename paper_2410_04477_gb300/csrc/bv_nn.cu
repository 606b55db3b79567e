// bv_nn.cu -- block nearest neighbours on the GPU (Sec. 2.2; Algorithm 1 "Nearest
// neighbors").
//
// Definition (fixed by this library, identical to the plain brute-force rule): for the
// block at position i of the order, the candidates are all points of blocks 0..i-1 (for a
// prediction block, Algorithm 2: all observations); the
// query is the block centroid c_i; the key of candidate j is (D2(c_i, s_j), j), D2 being
// the squared distance summed left to right without fused multiply-add; the conditioning
// set is the m_i smallest keys, ascending.  Positive doubles order like their bit
// patterns, so keys compare as (uint64 bits, index).
//
// One CTA per query block.  The candidates are the prefix of the block-ordered point
// array, so they are read contiguously from an FP32 copy.  Selection:
//   pass 1/2: radix histograms of the FP32 squared distance's top 24 bits give a value T
//             at or above the m_i-th smallest FP32 distance;
//   pass 3:   every candidate with d32 <= T + 2 margin (margin bounds |d32 - D2|) gets its
//             exact FP64 key into a shared list -- a superset of the true m_i nearest;
//   sort:     bitonic sort of the list by (key, index); the first m_i are the answer.
// If more than kCap candidates fall under the threshold (massive exact ties), an exact
// radix selection over the full 96-bit key (8 bits per pass, FP64 keys) replaces pass 3.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "bv_internal.h"

namespace {

constexpr int kNT = 512;
constexpr int kCap = 4096;  // exact-key list capacity (also the largest m supported)

__device__ __forceinline__ double d2_exact3(double q0, double q1, double q2, double x0, double x1,
                                            double x2, int d) {
    double acc = 0.0;
    double t = __dsub_rn(q0, x0);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
    if (d > 1) {
        t = __dsub_rn(q1, x1);
        acc = __dadd_rn(acc, __dmul_rn(t, t));
    }
    if (d > 2) {
        t = __dsub_rn(q2, x2);
        acc = __dadd_rn(acc, __dmul_rn(t, t));
    }
    return acc;
}

__device__ __forceinline__ float fp32_margin(float v, float amax, int d) {
    const float u = 5.9604645e-8f;
    const float eta = 4.04f * u * amax;
    const float D = sqrtf(fmaxf(v, 0.0f)) + 2.0f * eta;
    const float e = sqrtf((float)d) * eta * (2.0f * D + eta) + (float)(d + 2) * u * (v + 1e-30f);
    return 4.0f * e + 1e-30f;
}

__device__ __forceinline__ bool key_less(unsigned long long ka, int ia, unsigned long long kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// Bitonic sort of n (power of two) (key, idx) pairs in shared memory.
__device__ void bitonic_sort(unsigned long long* key, int* idx, int n) {
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const bool sw = up ? key_less(key[hi], idx[hi], key[lo], idx[lo])
                                   : key_less(key[lo], idx[lo], key[hi], idx[hi]);
                if (sw) {
                    const unsigned long long tk = key[lo];
                    key[lo] = key[hi];
                    key[hi] = tk;
                    const int ti = idx[lo];
                    idx[lo] = idx[hi];
                    idx[hi] = ti;
                }
            }
            __syncthreads();
        }
    }
}

// Find the smallest bin b with cumulative count (over bins 0..b) >= need; returns b and the
// count of bins < b in *below.  hist has nb bins (multiple of kNT).
__device__ int find_bin(const unsigned int* hist, int nb, unsigned int need, unsigned int* s_scan,
                        unsigned int* below) {
    __shared__ int s_bin;
    __shared__ unsigned int s_below;
    const int per = nb / kNT;
    unsigned int loc = 0;
    for (int j = 0; j < per; ++j) loc += hist[threadIdx.x * per + j];
    s_scan[threadIdx.x] = loc;
    __syncthreads();
    for (int o = 1; o < kNT; o <<= 1) {
        const unsigned int v = threadIdx.x >= o ? s_scan[threadIdx.x - o] : 0u;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
    }
    const unsigned int incl = s_scan[threadIdx.x], excl = incl - loc;
    if (excl < need && incl >= need) {
        unsigned int c = excl;
        for (int j = 0; j < per; ++j) {
            const unsigned int h = hist[threadIdx.x * per + j];
            if (c + h >= need) {
                s_bin = threadIdx.x * per + j;
                s_below = c;
                break;
            }
            c += h;
        }
    }
    __syncthreads();
    *below = s_below;
    const int b = s_bin;
    __syncthreads();
    return b;
}

struct NNArgs {
    const float* xs32;    // [d][P_all] FP32 coordinates in block order, from `base`
    const double* xs64;   // [d][P_all] FP64 coordinates in block order, from `base`
    const int32_t* pord;  // point index in block order (slice); null: candidate p is point base + p
    int64_t P_all;
    int64_t fixed_P;      // >= 0: every query ranks the first fixed_P candidates (prediction)
    int d;
    const int64_t* bptr;  // global block ptr
    int64_t base;         // bptr[blk_begin]
    int64_t blk_begin;
    const double* cent;
    const int64_t* nptr;
    int32_t* nidx;
    float amax;
    int* overflow_count;
};

__global__ void __launch_bounds__(kNT) k_select(NNArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long* key = reinterpret_cast<unsigned long long*>(smraw);  // kCap
    int* idx = reinterpret_cast<int*>(key + kCap);                            // kCap
    unsigned int* hist = reinterpret_cast<unsigned int*>(idx + kCap);         // 4096
    unsigned int* scan = hist + 4096;                                         // kNT
    __shared__ int s_cnt;
    const int64_t blk = a.blk_begin + blockIdx.x;
    const int64_t P = a.fixed_P >= 0 ? a.fixed_P : a.bptr[blk] - a.base;
    auto gidx = [&](int64_t p) -> int { return a.pord ? a.pord[a.base + p] : (int)(a.base + p); };
    const int64_t out0 = a.nptr[blk];
    const int mi = (int)(a.nptr[blk + 1] - out0);
    if (mi == 0) return;
    const int d = a.d;
    const double q0 = a.cent[blk * d], q1 = d > 1 ? a.cent[blk * d + 1] : 0.0,
                 q2 = d > 2 ? a.cent[blk * d + 2] : 0.0;
    const float f0 = (float)q0, f1 = (float)q1, f2 = (float)q2;
    const float* X0 = a.xs32;
    const float* X1 = a.xs32 + a.P_all;
    const float* X2 = a.xs32 + 2 * a.P_all;
    const double* Y0 = a.xs64;
    const double* Y1 = a.xs64 + a.P_all;
    const double* Y2 = a.xs64 + 2 * a.P_all;
    auto d32 = [&](int64_t p) -> float {
        const float t0 = f0 - X0[p];
        float v = t0 * t0;
        if (d > 1) {
            const float t1 = f1 - X1[p];
            v = fmaf(t1, t1, v);
        }
        if (d > 2) {
            const float t2 = f2 - X2[p];
            v = fmaf(t2, t2, v);
        }
        return v;
    };
    auto k64 = [&](int64_t p) -> unsigned long long {
        const double v = d2_exact3(q0, q1, q2, Y0[p], d > 1 ? Y1[p] : 0.0, d > 2 ? Y2[p] : 0.0, d);
        return (unsigned long long)__double_as_longlong(v);
    };

    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int count = 0;
    if (P <= kCap) {
        for (int64_t p = threadIdx.x; p < P; p += kNT) {
            key[p] = k64(p);
            idx[p] = gidx(p);
        }
        count = (int)P;
    } else {
        // pass 1: top 11 value bits of the FP32 squared distance (sign bit is 0)
        for (int t = threadIdx.x; t < 4096; t += kNT) hist[t] = 0u;
        __syncthreads();
        for (int64_t p = threadIdx.x; p < P; p += kNT)
            atomicAdd(&hist[__float_as_uint(d32(p)) >> 20], 1u);
        __syncthreads();
        unsigned int below = 0;
        const int b1 = find_bin(hist, 2048, (unsigned)mi, scan, &below);
        // pass 2: next 12 bits inside bin b1
        for (int t = threadIdx.x; t < 4096; t += kNT) hist[t] = 0u;
        __syncthreads();
        for (int64_t p = threadIdx.x; p < P; p += kNT) {
            const unsigned int u = __float_as_uint(d32(p));
            if ((int)(u >> 20) == b1) atomicAdd(&hist[(u >> 8) & 4095u], 1u);
        }
        __syncthreads();
        unsigned int below2 = 0;
        const int b2 = find_bin(hist, 4096, (unsigned)mi - below, scan, &below2);
        const float T = __uint_as_float(((unsigned)b1 << 20) | ((unsigned)b2 << 8) | 0xFFu);
        const float thr = T + 2.0f * fp32_margin(T * 1.001f, a.amax, d);
        // pass 3: exact keys of everything under the threshold
        for (int64_t p = threadIdx.x; p < P; p += kNT) {
            if (d32(p) <= thr) {
                const int slot = atomicAdd(&s_cnt, 1);
                if (slot < kCap) {
                    key[slot] = k64(p);
                    idx[slot] = gidx(p);
                }
            }
        }
        __syncthreads();
        count = s_cnt;
        if (count > kCap) {
            // exact radix selection of the mi-th smallest (key, index) among candidates
            // under thr, 8 bits per pass over the 96-bit key (64 key bits, 32 index bits)
            if (threadIdx.x == 0) atomicAdd(a.overflow_count, 1);
            unsigned long long pk = 0ull, pmask = 0ull;
            unsigned int pidx = 0u, pimask = 0u;
            unsigned int need = (unsigned)mi;
            for (int pass = 0; pass < 12; ++pass) {
                for (int t = threadIdx.x; t < 4096; t += kNT) hist[t] = 0u;
                __syncthreads();
                for (int64_t p = threadIdx.x; p < P; p += kNT) {
                    if (!(d32(p) <= thr)) continue;
                    const unsigned long long kk = k64(p);
                    const unsigned int ii = (unsigned)gidx(p);
                    if ((kk & pmask) != pk || (ii & pimask) != pidx) continue;
                    const unsigned int digit = pass < 8 ? (unsigned)(kk >> (56 - 8 * pass)) & 255u
                                                        : (ii >> (24 - 8 * (pass - 8))) & 255u;
                    atomicAdd(&hist[digit * 16], 1u);  // spread bins (4096 / 256)
                }
                __syncthreads();
                unsigned int bl = 0;
                const int bin = find_bin(hist, 4096, need, scan, &bl);
                const unsigned int digit = (unsigned)bin >> 4;
                need -= bl;
                if (pass < 8) {
                    pk |= (unsigned long long)digit << (56 - 8 * pass);
                    pmask |= 255ull << (56 - 8 * pass);
                } else {
                    pidx |= digit << (24 - 8 * (pass - 8));
                    pimask |= 255u << (24 - 8 * (pass - 8));
                }
            }
            // (pk, pidx) is the mi-th smallest key: collect everything <= it (exactly mi)
            if (threadIdx.x == 0) s_cnt = 0;
            __syncthreads();
            for (int64_t p = threadIdx.x; p < P; p += kNT) {
                if (!(d32(p) <= thr)) continue;
                const unsigned long long kk = k64(p);
                const int ii = gidx(p);
                if (!key_less(pk, (int)pidx, kk, ii)) {
                    const int slot = atomicAdd(&s_cnt, 1);
                    if (slot < kCap) {
                        key[slot] = kk;
                        idx[slot] = ii;
                    }
                }
            }
            __syncthreads();
            count = min(s_cnt, kCap);
        }
    }
    __syncthreads();
    int n2 = 1;
    while (n2 < count) n2 <<= 1;
    for (int t = count + threadIdx.x; t < n2; t += kNT) {
        key[t] = ~0ull;
        idx[t] = 0x7fffffff;
    }
    __syncthreads();
    bitonic_sort(key, idx, n2);
    for (int t = threadIdx.x; t < mi; t += kNT) a.nidx[out0 + t] = idx[t];
}

__global__ void k_gather_order(const double* __restrict__ locs, int64_t n_tot, int d,
                               const int32_t* __restrict__ pidx, int64_t base, int64_t P_all,
                               float* __restrict__ xs32, double* __restrict__ xs64) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P_all) return;
    const int64_t g = pidx ? pidx[base + p] : base + p;
    for (int k = 0; k < d; ++k) {
        const double v = locs[(int64_t)k * n_tot + g];
        xs64[(int64_t)k * P_all + p] = v;
        xs32[(int64_t)k * P_all + p] = (float)v;
    }
}

}  // namespace

// Neighbour sets of blocks [blk_begin, blk_end) of one dataset.  h_nptr (host) and d_nptr
// (device) hold the output offsets (m_i already fixed); d_nidx receives the indices.
int bv_select_neighbors_device(const double* d_locs, int64_t n_tot, int d, const int64_t* d_bptr,
                               const int32_t* d_pidx, const double* d_cent, int64_t blk_begin,
                               int64_t blk_end, const int64_t* h_nptr, int64_t* d_nptr,
                               int32_t* d_nidx, double amax, cudaStream_t s) {
    (void)h_nptr;
    int64_t base = 0, top = 0;
    BV_CUDA(cudaMemcpyAsync(&base, d_bptr + blk_begin, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BV_CUDA(cudaMemcpyAsync(&top, d_bptr + blk_end, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BV_CUDA(cudaStreamSynchronize(s));
    const int64_t P_all = top - base;
    if (blk_end <= blk_begin || P_all <= 0) return BV_OK;
    float* xs32 = nullptr;
    double* xs64 = nullptr;
    int* ovf = nullptr;
    BV_CUDA(cudaMallocAsync(&xs32, sizeof(float) * P_all * 3, s));
    BV_CUDA(cudaMallocAsync(&xs64, sizeof(double) * P_all * 3, s));
    BV_CUDA(cudaMallocAsync(&ovf, sizeof(int), s));
    BV_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), s));
    BV_CUDA(cudaMemsetAsync(xs32, 0, sizeof(float) * P_all * 3, s));
    BV_CUDA(cudaMemsetAsync(xs64, 0, sizeof(double) * P_all * 3, s));
    k_gather_order<<<(unsigned)((P_all + 255) / 256), 256, 0, s>>>(d_locs, n_tot, d, d_pidx, base, P_all,
                                                                    xs32, xs64);
    BV_CUDA(cudaGetLastError());
    NNArgs a;
    a.xs32 = xs32;
    a.xs64 = xs64;
    a.pord = d_pidx;
    a.P_all = P_all;
    a.fixed_P = -1;
    a.d = d;
    a.bptr = d_bptr;
    a.base = base;
    a.blk_begin = blk_begin;
    a.cent = d_cent;
    a.nptr = d_nptr;
    a.nidx = d_nidx;
    a.amax = (float)amax;
    a.overflow_count = ovf;
    const size_t smem = sizeof(unsigned long long) * kCap + sizeof(int) * kCap +
                        sizeof(unsigned int) * (4096 + kNT);
    BV_CUDA(cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t nq = blk_end - blk_begin;
    k_select<<<(unsigned)nq, kNT, smem, s>>>(a);
    BV_CUDA(cudaGetLastError());
    BV_CUDA(cudaFreeAsync(xs32, s));
    BV_CUDA(cudaFreeAsync(xs64, s));
    BV_CUDA(cudaFreeAsync(ovf, s));
    return BV_OK;
}

// Prediction (Algorithm 2): the conditioning set of query q (centroid d_qcent[q]) is the
// m_q = d_nptr[q+1] - d_nptr[q] smallest keys among ALL n_tot observations.
int bv_select_pred_neighbors_device(const double* d_locs, int64_t n_tot, int d, const double* d_qcent, int64_t nq,
                                    const int64_t* d_nptr, int32_t* d_nidx, double amax, cudaStream_t s) {
    if (nq <= 0 || n_tot <= 0) return BV_OK;
    float* xs32 = nullptr;
    double* xs64 = nullptr;
    int* ovf = nullptr;
    BV_CUDA(cudaMallocAsync(&xs32, sizeof(float) * n_tot * 3, s));
    BV_CUDA(cudaMallocAsync(&xs64, sizeof(double) * n_tot * 3, s));
    BV_CUDA(cudaMallocAsync(&ovf, sizeof(int), s));
    BV_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), s));
    BV_CUDA(cudaMemsetAsync(xs32, 0, sizeof(float) * n_tot * 3, s));
    BV_CUDA(cudaMemsetAsync(xs64, 0, sizeof(double) * n_tot * 3, s));
    k_gather_order<<<(unsigned)((n_tot + 255) / 256), 256, 0, s>>>(d_locs, n_tot, d, nullptr, 0, n_tot, xs32, xs64);
    BV_CUDA(cudaGetLastError());
    NNArgs a;
    a.xs32 = xs32;
    a.xs64 = xs64;
    a.pord = nullptr;
    a.P_all = n_tot;
    a.fixed_P = n_tot;
    a.d = d;
    a.bptr = nullptr;
    a.base = 0;
    a.blk_begin = 0;
    a.cent = d_qcent;
    a.nptr = d_nptr;
    a.nidx = d_nidx;
    a.amax = (float)amax;
    a.overflow_count = ovf;
    const size_t smem = sizeof(unsigned long long) * kCap + sizeof(int) * kCap + sizeof(unsigned int) * (4096 + kNT);
    BV_CUDA(cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_select<<<(unsigned)nq, kNT, smem, s>>>(a);
    BV_CUDA(cudaGetLastError());
    BV_CUDA(cudaFreeAsync(xs32, s));
    BV_CUDA(cudaFreeAsync(xs64, s));
    BV_CUDA(cudaFreeAsync(ovf, s));
    return BV_OK;
}
