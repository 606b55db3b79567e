// bv_exact.cu -- the exact Gaussian log-likelihood (Eq. 1) by a dense tiled Cholesky
// factorisation on the GPU, and the KL divergence of the block-Vecchia approximation
// (Eq. 7 of Sec. 3.1: KL = ell_0(theta; 0) - ell_a(theta; 0)).
//
// The (n+1) x (n+1) augmented matrix [[Sigma, .], [y^T, .]] is padded to a multiple of
// the tile size T with an identity block and stored as packed lower T x T tiles (tile
// (i, j), j <= i, at (i(i+1)/2 + j) T^2, row-major inside).  Right-looking tiled
// Cholesky, three launches per tile column k:
//   k_potrf   the diagonal tile (one CTA, shared memory)
//   k_trsm    L_ik = A_ik L_kk^-T for every tile below it (one CTA per tile)
//   k_update  A_ij -= L_ik L_jk^T for every trailing tile (one CTA per tile, 4 x 4 outputs
//             per thread from shared-memory operands)
// The factor's row n is z = L^-1 y, so y^T Sigma^-1 y = |z|^2 and log|Sigma| = 2 sum log
// L_ii.  The pivot of row n itself is not part of Sigma and is set to 1.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "bv_device.cuh"
#include "bv_internal.h"

namespace {

constexpr int T = 64;          // tile edge
constexpr int TT = T * T;
constexpr int kUpdNT = 256;    // 16 x 16 threads, 4 x 4 outputs each

__device__ __forceinline__ int64_t tile_off(int64_t i, int64_t j) { return ((i * (i + 1)) / 2 + j) * TT; }

__device__ __forceinline__ double matern_exact(const DevTheta& th, double x) {
    if (th.nu_code == NU_GENERAL) return th.sigma2 * matern_gen_corr(th, x);
    const double e = exp(-x);
    if (th.nu_code == NU_HALF) return th.sigma2 * e;
    if (th.nu_code == NU_3HALF) return th.sigma2 * ((1.0 + x) * e);
    return th.sigma2 * ((1.0 + x * (1.0 + x * (1.0 / 3.0))) * e);
}

struct FillArgs {
    const double* locs;  // SoA d x n
    const double* y;     // null: y = 0
    int64_t n;
    int d;
    int64_t nt;
    DevTheta th;
    double* A;
};

// One CTA per lower tile (blockIdx.x = packed tile index).
__global__ void __launch_bounds__(256) k_fill(FillArgs a) {
    const int64_t f = blockIdx.x;
    int64_t ti = (int64_t)((sqrt(8.0 * (double)f + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= f) ++ti;
    while (ti * (ti + 1) / 2 > f) --ti;
    const int64_t tj = f - ti * (ti + 1) / 2;
    double* out = a.A + f * TT;
    for (int e = threadIdx.x; e < TT; e += 256) {
        const int64_t r = ti * T + e / T, c = tj * T + e % T;
        double v = 0.0;
        if (c > r) {
            v = 0.0;
        } else if (r < a.n) {
            double acc = 0.0;
            for (int k = 0; k < a.d; ++k) {
                const double t = (a.locs[k * a.n + r] - a.locs[k * a.n + c]) * inv_range_k(a.th, k);
                acc = fma(t, t, acc);
            }
            v = matern_exact(a.th, sqrt(acc));
            if (r == c) v += a.th.nugget;
        } else if (r == a.n) {
            v = c < a.n ? (a.y ? a.y[c] : 0.0) : 1.0;
        } else {
            v = (r == c) ? 1.0 : 0.0;
        }
        out[e] = v;
    }
}

// Unblocked right-looking Cholesky of diagonal tile k in shared memory.  Row `yrow` (the
// data row, global index n) gets pivot 1; a non-positive pivot elsewhere sets *fail.
__global__ void __launch_bounds__(256) k_potrf(double* A, int64_t k, int64_t yrow, unsigned long long* fail) {
    __shared__ double s[TT];
    double* t = A + tile_off(k, k);
    for (int e = threadIdx.x; e < TT; e += 256) s[e] = t[e];
    __syncthreads();
    for (int c = 0; c < T; ++c) {
        const int64_t g = k * T + c;
        if (threadIdx.x == 0) {
            double p = s[c * T + c];
            if (g == yrow) {
                p = 1.0;
            } else if (!(p > 0.0)) {
                atomicMin(fail, (unsigned long long)g);
                p = 1.0;
            } else {
                p = sqrt(p);
            }
            s[c * T + c] = p;
        }
        __syncthreads();
        const double rl = 1.0 / s[c * T + c];
        for (int r = c + 1 + threadIdx.x; r < T; r += 256) s[r * T + c] *= rl;
        __syncthreads();
        for (int e = threadIdx.x; e < TT; e += 256) {
            const int r = e / T, q = e % T;
            if (q > c && q <= r) s[e] = fma(-s[r * T + c], s[q * T + c], s[e]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < TT; e += 256) t[e] = s[e];
}

// L_ik = A_ik L_kk^-T for i = k+1 .. nt-1 (blockIdx.x = i - k - 1): row r of L_ik solves
// x L_kk^T = a, column by column; 64 threads, one row each.
constexpr size_t kTrsmSmem = sizeof(double) * (TT + T * (T + 1));
constexpr size_t kUpdSmem = sizeof(double) * 2 * TT;

__global__ void __launch_bounds__(64) k_trsm(double* A, int64_t k) {
    extern __shared__ __align__(32) double sm[];
    double* L = sm;
    double* X = sm + TT;
    const int64_t i = k + 1 + blockIdx.x;
    const double* lk = A + tile_off(k, k);
    double* ai = A + tile_off(i, k);
    for (int e = threadIdx.x; e < TT; e += 64) {
        L[e] = lk[e];
        X[(e / T) * (T + 1) + e % T] = ai[e];
    }
    __syncthreads();
    const int r = threadIdx.x;
    double* x = X + r * (T + 1);
    for (int c = 0; c < T; ++c) {
        double v = x[c];
        for (int l = 0; l < c; ++l) v = fma(-x[l], L[c * T + l], v);
        x[c] = v / L[c * T + c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TT; e += 64) ai[e] = X[(e / T) * (T + 1) + e % T];
}

// A_ij -= L_ik L_jk^T for the trailing tiles k < j <= i < nt, blockIdx.x = packed index
// of (i - k - 1, j - k - 1).  Operands staged transposed in shared memory so that each
// thread reads its 4 rows and 4 columns of every inner step as two 32-byte loads.
__global__ void __launch_bounds__(kUpdNT) k_update(double* A, int64_t k) {
    extern __shared__ __align__(32) double sm[];
    double* Ls = sm;        // Ls[l * T + r] = L_ik[r][l]
    double* Rs = sm + TT;   // Rs[l * T + c] = L_jk[c][l]
    const int64_t f = blockIdx.x;
    int64_t a = (int64_t)((sqrt(8.0 * (double)f + 1.0) - 1.0) * 0.5);
    while ((a + 1) * (a + 2) / 2 <= f) ++a;
    while (a * (a + 1) / 2 > f) --a;
    const int64_t b = f - a * (a + 1) / 2;
    const int64_t i = k + 1 + a, j = k + 1 + b;
    const double* li = A + tile_off(i, k);
    const double* lj = A + tile_off(j, k);
    for (int e = threadIdx.x; e < TT; e += kUpdNT) {
        const int r = e / T, l = e % T;
        Ls[l * T + r] = li[e];
        Rs[l * T + r] = lj[e];
    }
    __syncthreads();
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
    double acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;
#pragma unroll 4
    for (int l = 0; l < T; ++l) {
        const double4_32a x = *reinterpret_cast<const double4_32a*>(&Ls[l * T + 4 * tr]);
        const double4_32a w = *reinterpret_cast<const double4_32a*>(&Rs[l * T + 4 * tc]);
        const double xv[4] = {x.x, x.y, x.z, x.w}, wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] = fma(xv[p], wv[q], acc[p][q]);
    }
    double* out = A + tile_off(i, j);
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = 4 * tr + p, c = 4 * tc + q;
            if (i != j || c <= r) out[r * T + c] -= acc[p][q];
        }
}

// log-det and quadratic form from the factor: one CTA, fixed-order sums.
__global__ void __launch_bounds__(256) k_exact_terms(const double* A, int64_t n, double* out) {
    __shared__ double s1[256], s2[256];
    double ld = 0.0, q = 0.0;
    const int64_t yt = n / T, yr = n % T;
    for (int64_t g = threadIdx.x; g < n; g += 256) {
        const int64_t t = g / T, r = g % T;
        ld += log(A[tile_off(t, t) + r * T + r]);
        const double z = A[tile_off(yt, t) + yr * T + r];
        q = fma(z, z, q);
    }
    s1[threadIdx.x] = ld;
    s2[threadIdx.x] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int t = 0; t < 256; ++t) {
            a += s1[t];
            b += s2[t];
        }
        out[0] = 2.0 * a;
        out[1] = b;
    }
}

}  // namespace

extern "C" int bv_exact_loglik(bv_ctx* c, const bv_theta* theta, int32_t use_y, double* out_loglik,
                               double* out_quad, double* out_logdet) {
    if (!c || !theta) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    if (use_y && !c->have_y) return BV_ESTATE;
    const int64_t n = c->n_tot;
    if (n <= 0 || n > 65536) return BV_EINVAL;
    DevTheta th;
    BV_TRY(bv_theta_to_dev(theta, c->d, &th));
    BV_CUDA(cudaSetDevice(c->device));
    const int64_t nt = (n + 1 + T - 1) / T;
    const int64_t ntiles = nt * (nt + 1) / 2;
    double* A = nullptr;
    double* terms = nullptr;
    unsigned long long* fail = nullptr;
    BV_CUDA(cudaMallocAsync(&A, sizeof(double) * ntiles * TT, c->stream));
    BV_CUDA(cudaMallocAsync(&terms, sizeof(double) * 2, c->stream));
    BV_CUDA(cudaMallocAsync(&fail, sizeof(unsigned long long), c->stream));
    BV_CUDA(cudaMemsetAsync(fail, 0xff, sizeof(unsigned long long), c->stream));
    BV_CUDA(cudaFuncSetAttribute(k_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrsmSmem));
    BV_CUDA(cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpdSmem));
    FillArgs fa{c->d_locs, use_y ? c->d_y : nullptr, n, c->d, nt, th, A};
    k_fill<<<(unsigned)ntiles, 256, 0, c->stream>>>(fa);
    BV_CUDA(cudaGetLastError());
    for (int64_t k = 0; k < nt; ++k) {
        k_potrf<<<1, 256, 0, c->stream>>>(A, k, n, fail);
        const int64_t m = nt - k - 1;
        if (m > 0) {
            k_trsm<<<(unsigned)m, 64, kTrsmSmem, c->stream>>>(A, k);
            k_update<<<(unsigned)(m * (m + 1) / 2), kUpdNT, kUpdSmem, c->stream>>>(A, k);
        }
    }
    BV_CUDA(cudaGetLastError());
    k_exact_terms<<<1, 256, 0, c->stream>>>(A, n, terms);
    BV_CUDA(cudaGetLastError());
    double h[2] = {0.0, 0.0};
    unsigned long long hf = 0;
    BV_CUDA(cudaMemcpyAsync(h, terms, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaMemcpyAsync(&hf, fail, sizeof(hf), cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaFreeAsync(A, c->stream));
    BV_CUDA(cudaFreeAsync(terms, c->stream));
    BV_CUDA(cudaFreeAsync(fail, c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    if (hf != ~0ull) {
        if (out_loglik) *out_loglik = -INFINITY;
        return BV_ENOTPD;
    }
    const double logdet = h[0], quad = h[1];
    if (out_logdet) *out_logdet = logdet;
    if (out_quad) *out_quad = quad;
    if (out_loglik) *out_loglik = -0.5 * (quad + logdet + (double)n * 1.8378770664093454835606594728112);
    return BV_OK;
}

extern "C" int bv_exact_flops(int64_t n, double* flops) {
    if (n <= 0 || !flops) return BV_EINVAL;
    const double N = (double)(n + 1);
    *flops = N * N * N / 3.0 + N * N;  // Cholesky of the augmented matrix, leading terms
    return BV_OK;
}

extern "C" int bv_kl_divergence(bv_ctx* c, const bv_theta* theta, int32_t precision, double* out_kl,
                                double* out_logdet_exact, double* out_logdet_approx) {
    if (!c || !theta || !out_kl) return BV_EINVAL;
    if (!c->have_nn) return BV_ESTATE;
    // log-determinants do not depend on y: any observations (zeros if none) serve
    if (!c->have_y) {
        std::vector<double> zero(c->n_tot, 0.0);
        BV_TRY(bv_set_observations(c, zero.data(), 0));
    }
    double d0 = 0.0, da = 0.0, la = 0.0;
    BV_TRY(bv_exact_loglik(c, theta, 0, nullptr, nullptr, &d0));
    BV_TRY(bv_loglik_terms(c, theta, precision, &la, nullptr, &da));
    if (out_logdet_exact) *out_logdet_exact = d0;
    if (out_logdet_approx) *out_logdet_approx = da;
    // Eq. 7 with tr(Sigma_a^-1 Sigma_0) = n for Vecchia-type approximations:
    // KL = ell_0(theta; 0) - ell_a(theta; 0) = (log|Sigma_a| - log|Sigma_0|) / 2
    *out_kl = 0.5 * (da - d0);
    return BV_OK;
}
