// bv_order.cu -- block orderings (Sec. 2.1: the random, maxmin, Morton, KD-tree and Hilbert
// permutations the paper compares in its KL study, Sec. 3.1).
//
// bv_order_blocks places the context's blocks in a new order chosen from their centroids;
// ties always go to the lower current position.
//   random   Fisher-Yates over the current positions (block-permutation stream of seed)
//   maxmin   first the centroid nearest to the mean centroid, then repeatedly the one
//            farthest (largest smallest squared distance) from those already placed
//            (Guinness 2018).  O(bc^2): one CTA on the GPU runs the greedy loop.
//   Morton   Z-order key of the centroid scaled to 21-bit integers over the bounding box
//   KD-tree  recursive median split cycling through the axes, left part first (Bentley 1975)
//   Hilbert  Hilbert index of the same 21-bit integers by Skilling's axes-to-transpose
//            transform (Skilling 2004)
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "bv_internal.h"

namespace {

// squared distance summed left to right, every operation rounded separately
__host__ __device__ inline double sqdist(const double* a, const double* b, int d) {
#ifdef __CUDA_ARCH__
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = __dsub_rn(a[k], b[k]);
        acc = __dadd_rn(acc, __dmul_rn(t, t));
    }
    return acc;
#else
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = a[k] - b[k];
        const double sq = t * t;
        acc = acc + sq;
    }
    return acc;
#endif
}

// Greedy farthest-point loop of the maxmin order in one CTA: per step every thread folds
// the newest centroid into its share of the running minima, then a block-wide arg-max
// over (minimum, -position) picks the next block.
constexpr int kMaxminNT = 1024;

__global__ void __launch_bounds__(kMaxminNT) k_maxmin(const double* __restrict__ cent, int64_t bc, int d,
                                                       int64_t first, double* __restrict__ dmin,
                                                       int64_t* __restrict__ perm) {
    __shared__ double s_v[kMaxminNT / 32];
    __shared__ int64_t s_p[kMaxminNT / 32];
    __shared__ int64_t s_pick;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t last = first;
    if (tid == 0) perm[0] = first;
    for (int64_t q = 1; q < bc; ++q) {
        double c[3];
        for (int k = 0; k < d; ++k) c[k] = cent[last * d + k];
        double bv = -2.0;
        int64_t bp = -1;
        for (int64_t p = tid; p < bc; p += kMaxminNT) {
            double v = dmin[p];
            if (v >= 0.0) {  // still unplaced
                const double t = sqdist(cent + p * d, c, d);
                if (q == 1 || t < v) v = t;
                if (p == last) v = -1.0;
                dmin[p] = v;
            }
            if (v > bv) {  // positions ascend per thread: ties keep the lower one
                bv = v;
                bp = p;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int64_t op = __shfl_xor_sync(0xffffffffu, bp, o);
            if (ov > bv || (ov == bv && op >= 0 && (bp < 0 || op < bp))) {
                bv = ov;
                bp = op;
            }
        }
        if (lane == 0) {
            s_v[warp] = bv;
            s_p[warp] = bp;
        }
        __syncthreads();
        if (tid == 0) {
            double v = s_v[0];
            int64_t p = s_p[0];
            for (int w = 1; w < kMaxminNT / 32; ++w)
                if (s_v[w] > v || (s_v[w] == v && s_p[w] >= 0 && (p < 0 || s_p[w] < p))) {
                    v = s_v[w];
                    p = s_p[w];
                }
            perm[q] = p;
            s_pick = p;
        }
        __syncthreads();
        last = s_pick;
        __syncthreads();
    }
}

void quantise21(const std::vector<double>& cent, int64_t bc, int d, std::vector<uint64_t>& q) {
    q.assign((size_t)bc * d, 0);
    for (int k = 0; k < d; ++k) {
        double lo = cent[k], hi = cent[k];
        for (int64_t p = 1; p < bc; ++p) {
            lo = std::min(lo, cent[(size_t)p * d + k]);
            hi = std::max(hi, cent[(size_t)p * d + k]);
        }
        if (!(hi > lo)) continue;
        const double span = hi - lo;
        for (int64_t p = 0; p < bc; ++p) {
            const double f = floor((cent[(size_t)p * d + k] - lo) / span * 2097152.0);
            q[(size_t)p * d + k] = f >= 2097151.0 ? 2097151ull : (uint64_t)f;
        }
    }
}

uint64_t morton21(const uint64_t* x, int d) {
    uint64_t key = 0;
    for (int b = 0; b < 21; ++b)
        for (int a = 0; a < d; ++a) key |= ((x[a] >> b) & 1ull) << (b * d + a);
    return key;
}

// Skilling's transform of 21-bit axes to the transposed Hilbert index, then the bits read
// level by level (most significant first), axis 0 first within a level.
uint64_t hilbert21(const uint64_t* x, int d) {
    uint64_t v[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) v[a] = x[a];
    for (uint64_t bit = 1ull << 20; bit > 1; bit >>= 1) {
        const uint64_t low = bit - 1;
        for (int a = 0; a < d; ++a) {
            if (v[a] & bit) {
                v[0] ^= low;
            } else {
                const uint64_t sw = (v[0] ^ v[a]) & low;
                v[0] ^= sw;
                v[a] ^= sw;
            }
        }
    }
    for (int a = 1; a < d; ++a) v[a] ^= v[a - 1];
    uint64_t flip = 0;
    for (uint64_t bit = 1ull << 20; bit > 1; bit >>= 1)
        if (v[d - 1] & bit) flip ^= bit - 1;
    for (int a = 0; a < d; ++a) v[a] ^= flip;
    uint64_t key = 0;
    for (int lev = 20; lev >= 0; --lev)
        for (int a = 0; a < d; ++a) key = (key << 1) | ((v[a] >> lev) & 1ull);
    return key;
}

void kd_order(const std::vector<double>& cent, int d, int64_t* idx, int64_t n, int depth) {
    if (n <= 1) return;
    const int ax = depth % d;
    std::sort(idx, idx + n, [&](int64_t a, int64_t b) {
        const double va = cent[(size_t)a * d + ax], vb = cent[(size_t)b * d + ax];
        return va < vb || (va == vb && a < b);
    });
    const int64_t h = n / 2;
    kd_order(cent, d, idx, h, depth + 1);
    kd_order(cent, d, idx + h, n - h, depth + 1);
}

}  // namespace

// Places block perm[q] (current position) at new position q, re-uploading the structure.
int bv_apply_block_order(bv_ctx* c, const std::vector<int64_t>& perm, const std::vector<double>& cent);

extern "C" int bv_order_blocks(bv_ctx* c, int32_t order, uint64_t seed, int64_t* block_ptr, int32_t* point_idx) {
    if (!c || order < BV_ORDER_RANDOM || order > BV_ORDER_HILBERT) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    if (!c->have_blocks) return BV_ESTATE;
    BV_CUDA(cudaSetDevice(c->device));
    const int64_t bc = c->nblk;
    const int d = c->d;
    std::vector<double> cent((size_t)bc * d);
    BV_CUDA(cudaMemcpy(cent.data(), c->d_cent, sizeof(double) * bc * d, cudaMemcpyDeviceToHost));
    std::vector<int64_t> perm(bc);
    std::iota(perm.begin(), perm.end(), (int64_t)0);
    if (order == BV_ORDER_RANDOM) {
        const uint64_t zs = BV_STREAM_ZETA(seed);
        for (int64_t i = bc - 1; i >= 1; --i) {
            const uint64_t r = bv_sm64(zs, (uint64_t)i);
            const int64_t j = (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(i + 1)) >> 64);
            std::swap(perm[i], perm[j]);
        }
    } else if (order == BV_ORDER_MAXMIN) {
        double mean[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < d; ++k) {
            double sacc = 0.0;
            for (int64_t p = 0; p < bc; ++p) sacc = sacc + cent[(size_t)p * d + k];
            mean[k] = sacc / (double)bc;
        }
        int64_t first = 0;
        double best = INFINITY;
        for (int64_t p = 0; p < bc; ++p) {
            const double v = sqdist(&cent[(size_t)p * d], mean, d);
            if (v < best) {
                best = v;
                first = p;
            }
        }
        if (bc > 1) {
            double *d_dmin = nullptr, *d_c = nullptr;
            int64_t* d_perm = nullptr;
            BV_CUDA(cudaMalloc(&d_dmin, sizeof(double) * bc));
            BV_CUDA(cudaMalloc(&d_c, sizeof(double) * bc * d));
            BV_CUDA(cudaMalloc(&d_perm, sizeof(int64_t) * bc));
            BV_CUDA(cudaMemsetAsync(d_dmin, 0, sizeof(double) * bc, c->stream));
            BV_CUDA(cudaMemcpyAsync(d_c, cent.data(), sizeof(double) * bc * d, cudaMemcpyHostToDevice, c->stream));
            k_maxmin<<<1, kMaxminNT, 0, c->stream>>>(d_c, bc, d, first, d_dmin, d_perm);
            BV_CUDA(cudaGetLastError());
            BV_CUDA(cudaMemcpyAsync(perm.data(), d_perm, sizeof(int64_t) * bc, cudaMemcpyDeviceToHost, c->stream));
            BV_CUDA(cudaStreamSynchronize(c->stream));
            cudaFree(d_dmin);
            cudaFree(d_c);
            cudaFree(d_perm);
        }
    } else if (order == BV_ORDER_MORTON || order == BV_ORDER_HILBERT) {
        std::vector<uint64_t> q;
        quantise21(cent, bc, d, q);
        std::vector<uint64_t> key(bc);
        for (int64_t p = 0; p < bc; ++p)
            key[p] = order == BV_ORDER_MORTON ? morton21(&q[(size_t)p * d], d) : hilbert21(&q[(size_t)p * d], d);
        std::sort(perm.begin(), perm.end(),
                  [&](int64_t a, int64_t b) { return key[a] < key[b] || (key[a] == key[b] && a < b); });
    } else {
        kd_order(cent, d, perm.data(), bc, 0);
    }
    std::vector<double> ncent((size_t)bc * d);
    for (int64_t q = 0; q < bc; ++q)
        for (int k = 0; k < d; ++k) ncent[(size_t)q * d + k] = cent[(size_t)perm[q] * d + k];
    BV_TRY(bv_apply_block_order(c, perm, ncent));
    if (block_ptr) memcpy(block_ptr, c->h_bptr.data(), sizeof(int64_t) * (bc + 1));
    if (point_idx) memcpy(point_idx, c->h_pidx.data(), sizeof(int32_t) * c->n_tot);
    return BV_OK;
}

// Points of [off, off + n) (row-major host coordinates) in the order of the Hilbert index
// of their coordinates scaled to 21-bit integers over the range's bounding box (ties by
// index).  order receives the global point indices.
void bv_hilbert_order(const double* locs, int64_t off, int64_t n, int d, std::vector<int32_t>& order) {
    std::vector<double> pts((size_t)n * d);
    for (int64_t i = 0; i < n * d; ++i) pts[(size_t)i] = locs[(size_t)off * d + i];
    std::vector<uint64_t> q;
    quantise21(pts, n, d, q);
    std::vector<uint64_t> key(n);
    for (int64_t i = 0; i < n; ++i) key[i] = hilbert21(&q[(size_t)i * d], d);
    order.resize(n);
    std::iota(order.begin(), order.end(), (int32_t)0);
    std::sort(order.begin(), order.end(),
              [&](int32_t a, int32_t b) { return key[a] < key[b] || (key[a] == key[b] && a < b); });
    for (auto& v : order) v = (int32_t)(v + off);
}
