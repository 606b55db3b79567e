// bv_sim.cu -- block-Vecchia sampler: Eq. 4 read generatively.
//
// The block-Vecchia model draws block i (in the block order) as
//     y_{B_i} = W_i^T y_{NN_i} + L'_i z_{B_i},   W_i = (Sigma^con_i)^{-1} Sigma^cross_i,
//     L'_i = chol(Sigma^lk_i - Sigma^cross_i^T W_i),
// the conditional mean and the factor of the conditional covariance of Algorithm 1.
// W_i and L'_i do not depend on y, so they are computed for all blocks in parallel
// (phase 1: the augmented Cholesky of [[Sigma^con, Sigma^cross], [., Sigma^lk]] gives L,
// V^T and L'; a back substitution gives W = L^{-T} V).  Only the cheap apply step is
// sequential: blocks are grouped into levels (a block's level is one more than the
// highest level among the blocks owning its conditioning points), and one launch per
// level draws all its blocks (phase 2).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "bv_device.cuh"
#include "bv_internal.h"

namespace {

__device__ __forceinline__ int64_t pk64(int64_t r, int64_t c) { return ((r * (r + 1)) >> 1) + c; }


__device__ __forceinline__ double matern64s(const DevTheta& th, double x) {
    if (th.nu_code == NU_GENERAL) return th.sigma2 * matern_gen_corr(th, x);
    const double e = exp(-x);
    if (th.nu_code == NU_HALF) return th.sigma2 * e;
    if (th.nu_code == NU_3HALF) return th.sigma2 * ((1.0 + x) * e);
    return th.sigma2 * ((1.0 + x * (1.0 + x * (1.0 / 3.0))) * e);
}

struct SimArgs {
    const double* locs;
    int64_t n_tot;
    int d;
    const int64_t* bptr;
    const int32_t* pidx;
    const int64_t* nptr;
    const int32_t* nidx;
    DevTheta th;
    const int64_t* woff;   // offset of block i's W (m_i x b_i, row-major) in wbuf
    const int64_t* loff;   // offset of block i's L' (packed b_i x b_i) in lbuf
    double* wbuf;
    double* lbuf;
    double* ws;
    int64_t ws_stride;
    int64_t nblk;
    unsigned long long* fail;
};

// Phase 1: one CTA per block (grid-stride), packed factor in a global workspace slot.
__global__ void __launch_bounds__(256) k_sim_factor(SimArgs a) {
    const int NT = 256;
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* A = a.ws + (int64_t)blockIdx.x * a.ws_stride;
    for (int64_t blk = blockIdx.x; blk < a.nblk; blk += gridDim.x) {
        const int64_t b0 = a.bptr[blk], n0 = a.nptr[blk];
        const int b = (int)(a.bptr[blk + 1] - b0), m = (int)(a.nptr[blk + 1] - n0);
        const int N = m + b;
        double* px = A + pk64(N, 0) + 8;   // after the packed N x N triangle
        double* col = px + 3 * N;          // scratch column
        for (int t = tid; t < N; t += NT) {
            const int g = t < m ? a.nidx[n0 + t] : a.pidx[b0 + (t - m)];
            for (int k = 0; k < a.d; ++k) px[k * N + t] = a.locs[(int64_t)k * a.n_tot + g];
        }
        if (tid == 0) s_fail = 0;
        __syncthreads();
        for (int r = warp; r < N; r += NT / 32)
            for (int c = lane; c <= r; c += 32) {
                double acc = 0.0;
                for (int k = 0; k < a.d; ++k) {
                    const double t = (px[k * N + r] - px[k * N + c]) * inv_range_k(a.th, k);
                    acc = fma(t, t, acc);
                }
                double v = matern64s(a.th, sqrt(acc));
                if (r == c) v += a.th.nugget;
                A[pk64(r, c)] = v;
            }
        __syncthreads();
        // right-looking Cholesky, one column per step
        for (int k = 0; k < N; ++k) {
            if (warp == 0) {
                const double p = A[pk64(k, k)];
                if (bad_pivot(p) && lane == 0) s_fail = 1;
                const double l = sqrt(p), rl = 1.0 / l;
                if (lane == 0) A[pk64(k, k)] = l;
                for (int j = k + 1 + lane; j < N; j += 32) A[pk64(j, k)] *= rl;
            }
            __syncthreads();
            for (int j = k + 1 + warp; j < N; j += NT / 32) {
                const double cj = A[pk64(j, k)];
                for (int i = k + 1 + lane; i <= j; i += 32) A[pk64(j, i)] = fma(-cj, A[pk64(i, k)], A[pk64(j, i)]);
            }
            __syncthreads();
        }
        // W = L^{-T} V: column c of V is A[m + c][0..m); back substitution with L^T
        double* W = a.wbuf + a.woff[blk];
        for (int c = warp; c < b; c += NT / 32) {
            // solve L^T w = v, v_t = A[m+c][t]; lanes stride over rows
            double* w = col + (int64_t)warp * N;  // per-warp scratch (N doubles)
            for (int t = lane; t < m; t += 32) w[t] = A[pk64(m + c, t)];
            __syncwarp();
            for (int t = m - 1; t >= 0; --t) {
                const double wt = w[t] / A[pk64(t, t)];
                __syncwarp();
                if (lane == 0) w[t] = wt;
                for (int r = lane; r < t; r += 32) w[r] = fma(-A[pk64(t, r)], wt, w[r]);
                __syncwarp();
            }
            for (int t = lane; t < m; t += 32) W[(int64_t)t * b + c] = w[t];
            __syncwarp();
        }
        // L' = trailing b x b factor
        double* Lp = a.lbuf + a.loff[blk];
        for (int f = tid; f < (b * (b + 1)) / 2; f += NT) {
            int r = (int)((sqrtf(8.0f * f + 1.0f) - 1.0f) * 0.5f);
            if (((r + 1) * (r + 2)) / 2 <= f) ++r;
            if ((r * (r + 1)) / 2 > f) --r;
            const int c = f - (r * (r + 1)) / 2;
            Lp[f] = A[pk64(m + r, m + c)];
        }
        if (tid == 0 && s_fail) atomicMin(a.fail, (unsigned long long)blk);
        __syncthreads();
    }
}

// Phase 2: one warp per block of the level.
__global__ void k_sim_apply(SimArgs a, const int32_t* __restrict__ blocks, int64_t nb,
                            const double* __restrict__ z, double* __restrict__ y) {
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= nb) return;
    const int64_t blk = blocks[wg];
    const int64_t b0 = a.bptr[blk], n0 = a.nptr[blk];
    const int b = (int)(a.bptr[blk + 1] - b0), m = (int)(a.nptr[blk + 1] - n0);
    const double* W = a.wbuf + a.woff[blk];
    const double* Lp = a.lbuf + a.loff[blk];
    for (int j = lane; j < b; j += 32) {
        double mu = 0.0;
        for (int t = 0; t < m; ++t) mu = fma(W[(int64_t)t * b + j], y[a.nidx[n0 + t]], mu);
        double v = mu;
        for (int t = 0; t <= j; ++t) v = fma(Lp[(j * (j + 1)) / 2 + t], z[a.pidx[b0 + t]], v);
        y[a.pidx[b0 + j]] = v;
    }
}

}  // namespace

int bv_simulate_device(bv_ctx* c, const DevTheta& th, const double* d_z, double* d_y) {
    const int64_t nb = c->ds_blk_off[1] - c->ds_blk_off[0];
    // offsets of W and L' per block, levels, workspace
    std::vector<int64_t> woff(nb + 1, 0), loff(nb + 1, 0);
    int64_t maxN = 1;
    for (int64_t i = 0; i < nb; ++i) {
        const int64_t b = c->h_bptr[i + 1] - c->h_bptr[i], m = c->h_nptr[i + 1] - c->h_nptr[i];
        woff[i + 1] = woff[i] + m * b;
        loff[i + 1] = loff[i] + (b * (b + 1)) / 2;
        maxN = std::max(maxN, m + b);
    }
    if (maxN > BV_LARGE_MAX_N) return BV_EINVAL;
    std::vector<int32_t> nidx(std::max<int64_t>(c->h_nptr[nb], 1));
    if (c->h_nptr[nb] > 0)
        BV_CUDA(cudaMemcpy(nidx.data(), c->d_nidx, sizeof(int32_t) * c->h_nptr[nb], cudaMemcpyDeviceToHost));
    std::vector<int32_t> blk_of(c->n_tot, -1);
    for (int64_t i = 0; i < nb; ++i)
        for (int64_t p = c->h_bptr[i]; p < c->h_bptr[i + 1]; ++p) blk_of[c->h_pidx[p]] = (int32_t)i;
    std::vector<int32_t> level(nb, 0);
    int32_t nlev = 0;
    for (int64_t i = 0; i < nb; ++i) {
        int32_t lv = 0;
        for (int64_t p = c->h_nptr[i]; p < c->h_nptr[i + 1]; ++p) {
            const int32_t bj = blk_of[nidx[p]];
            if (bj < 0 || bj >= i) return BV_EINVAL;  // conditioning points must precede the block
            lv = std::max(lv, level[bj] + 1);
        }
        level[i] = lv;
        nlev = std::max(nlev, lv + 1);
    }
    std::vector<int64_t> lcount(nlev + 1, 0);
    for (int64_t i = 0; i < nb; ++i) lcount[level[i] + 1]++;
    for (int l = 0; l < nlev; ++l) lcount[l + 1] += lcount[l];
    std::vector<int32_t> order(nb);
    {
        std::vector<int64_t> fill(lcount.begin(), lcount.end() - 1);
        for (int64_t i = 0; i < nb; ++i) order[fill[level[i]]++] = (int32_t)i;
    }
    const int64_t stride = (maxN * (maxN + 1)) / 2 + 8 + 3 * maxN + 8 * maxN + 8;
    int slots = (int)std::min<int64_t>(nb, 2 * (int64_t)c->num_sms);
    while (slots > 1 && (double)slots * stride * 8.0 > 8e9) --slots;
    double *ws = nullptr, *wbuf = nullptr, *lbuf = nullptr;
    int64_t *d_woff = nullptr, *d_loff = nullptr;
    int32_t* d_order = nullptr;
    BV_CUDA(cudaMalloc(&ws, sizeof(double) * stride * slots));
    BV_CUDA(cudaMalloc(&wbuf, sizeof(double) * std::max<int64_t>(woff[nb], 1)));
    BV_CUDA(cudaMalloc(&lbuf, sizeof(double) * std::max<int64_t>(loff[nb], 1)));
    BV_CUDA(cudaMalloc(&d_woff, sizeof(int64_t) * (nb + 1)));
    BV_CUDA(cudaMalloc(&d_loff, sizeof(int64_t) * (nb + 1)));
    BV_CUDA(cudaMalloc(&d_order, sizeof(int32_t) * nb));
    BV_CUDA(cudaMemcpyAsync(d_woff, woff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, c->stream));
    BV_CUDA(cudaMemcpyAsync(d_loff, loff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, c->stream));
    BV_CUDA(cudaMemcpyAsync(d_order, order.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, c->stream));
    SimArgs a;
    a.locs = c->d_locs;
    a.n_tot = c->n_tot;
    a.d = c->d;
    a.bptr = c->d_bptr;
    a.pidx = c->d_pidx;
    a.nptr = c->d_nptr;
    a.nidx = c->d_nidx;
    a.th = th;
    a.woff = d_woff;
    a.loff = d_loff;
    a.wbuf = wbuf;
    a.lbuf = lbuf;
    a.ws = ws;
    a.ws_stride = stride;
    a.nblk = nb;
    a.fail = c->d_fail;
    BV_CUDA(bv_launch_fail_reset(c->d_fail, c->stream));
    k_sim_factor<<<slots, 256, 0, c->stream>>>(a);
    BV_CUDA(cudaGetLastError());
    for (int l = 0; l < nlev; ++l) {
        const int64_t cnt = lcount[l + 1] - lcount[l];
        const unsigned grid = (unsigned)((cnt * 32 + 255) / 256);
        k_sim_apply<<<grid, 256, 0, c->stream>>>(a, d_order + lcount[l], cnt, d_z, d_y);
        BV_CUDA(cudaGetLastError());
    }
    BV_CUDA(cudaMemcpyAsync(c->h_fail, c->d_fail, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    cudaFree(ws);
    cudaFree(wbuf);
    cudaFree(lbuf);
    cudaFree(d_woff);
    cudaFree(d_loff);
    cudaFree(d_order);
    return *c->h_fail != ~0ull ? BV_ENOTPD : BV_OK;
}

extern "C" int bv_simulate(bv_ctx* c, const bv_theta* theta, const double* z, double* y_out) {
    if (!c || !theta || !z) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    if (!c->have_nn) return BV_ESTATE;
    DevTheta th;
    BV_TRY(bv_theta_to_dev(theta, c->d, &th));
    BV_CUDA(cudaSetDevice(c->device));
    double* d_z = nullptr;
    BV_CUDA(cudaMalloc(&d_z, sizeof(double) * c->n_tot));
    BV_CUDA(cudaMemcpyAsync(d_z, z, sizeof(double) * c->n_tot, cudaMemcpyHostToDevice, c->stream));
    BV_CUDA(cudaMemsetAsync(c->d_y, 0, sizeof(double) * c->n_tot, c->stream));
    int st = bv_simulate_device(c, th, d_z, c->d_y);
    if (st == BV_OK) st = bv_refresh_layout_y(c);
    cudaFree(d_z);
    if (st != BV_OK) return st;
    c->have_y = true;
    if (y_out) BV_CUDA(cudaMemcpy(y_out, c->d_y, sizeof(double) * c->n_tot, cudaMemcpyDeviceToHost));
    return BV_OK;
}
