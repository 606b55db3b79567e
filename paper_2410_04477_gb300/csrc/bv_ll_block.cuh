// bv_ll_block.cuh -- helpers shared by the per-block log-likelihood kernels (the FP64 and
// FP32 SIMT kernels in bv_loglik.cu and the tensor-core kernel in bv_mixed_tc.cu): work
// distribution of a persistent launch, the FP32 Matern closed forms, the warp sum of a
// block's terms and the per-block result with its failure handling.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bv_device.cuh"
#include "bv_internal.h"

namespace {

constexpr double kLog2Pi = 1.8378770664093454835606594728112;

// e^{-x} for x >= 0 in FP32 by Tang's table-driven method (ACM TOMS 15(2), 1989) with 32
// table steps: x = n ln2/32 + r (Cody-Waite split of ln2/32, |r| <= ln2/64), n = 32 q + j,
// e^{-x} = 2^{-q} (T_j + (T_j p + T'_j)) with T_j + T'_j = 2^{-j/32} held as two floats
// and p = e^{-r} - 1 from its degree-4 Taylor polynomial (truncation below 1.2e-12).  Every
// step before the last addition errs by a few hundredths of an ulp, so the result is the
// exact value rounded once: an error of at most about half an ulp, without the one-sided
// bias a shared exponential would put into every covariance entry.  t: the 64 floats of
// the table in shared memory; underflows to 0 beyond x = 87.
__device__ __forceinline__ float exp_neg32(float x, const float* t, float K, float L1, float L2) {
    if (!(x < 87.0f)) return 0.0f;
    const float nf = rintf(x * K);
    const int n = (int)nf;
    const float r = fmaf(-nf, L2, fmaf(-nf, L1, x));
    const float p = r * fmaf(r, fmaf(r, fmaf(r, 1.0f / 24.0f, -1.0f / 6.0f), 0.5f), -1.0f);
    const int j = n & 31, q = n >> 5;
    const float th = t[j];
    const float v = th + fmaf(th, p, t[32 + j]);
    return v * __int_as_float((127 - q) << 23);
}

// The closed-form Matern correlations times sigma^2 in FP32; t32: the table of exp_neg32
// in shared memory.  (CUDA's expf errs high on average, by 0.09 ulp over [0, 20] and
// 0.16 ulp over [0.2, 1] as measured on this GPU: a bias shared by every covariance entry
// that the mixed path's error check would see as a trend of the errors with conditioning.)
__device__ __forceinline__ float matern32(int nu, float sigma2, float x, const float* t32, const ExpConsts& ex) {
    const float e = exp_neg32(x, t32, ex.k32, ex.l1_32, ex.l2_32);
    if (nu == NU_HALF) return sigma2 * e;
    if (nu == NU_3HALF) return sigma2 * ((1.0f + x) * e);
    return sigma2 * ((1.0f + x * (1.0f + x * (1.0f / 3.0f))) * e);
}

// Sums of the block columns' terms z_k^2 + log L_kk (Algorithm 1's quadratic form and
// log-determinant) and of z_k^2 alone, k = m..N-1, taken by the 32 lanes of one warp
// (a block has few columns, b = N - m); the totals are valid in lane 0.
template <typename ZF, typename LF>
__device__ __forceinline__ double2 warp_terms(int m, int N, int lane, ZF zk, LF logk) {
    double part = 0.0, partu = 0.0;
    for (int k = m + lane; k < N; k += 32) {
        const double z = zk(k);
        partu += z * z;
        part += z * z + logk(k);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        part += __shfl_xor_sync(0xffffffffu, part, o);
        partu += __shfl_xor_sync(0xffffffffu, partu, o);
    }
    return make_double2(part, partu);
}

// The conditioning indicator of a block factored in FP32: sum over all N pivots of
// (sigma^2 + tau^2) / p_k, the ratio of each point's variance to its conditional variance
// given the points before it.  The FP32 error of the block's ell_i grows with it.  One
// warp; the sum is valid in lane 0.
template <typename PF>
__device__ __forceinline__ float warp_indicator(int N, int lane, float diag, PF pivk) {
    float s = 0.0f;
    for (int k = lane; k < N; k += 32) s += diag / pivk(k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__device__ __forceinline__ void record_fail(unsigned long long* fail, int blk) {
    atomicMin(fail, (unsigned long long)blk);
}

// Work distribution of one launch.  With a counter, each CTA (or warp) takes its next
// work item from the launch's atomic counter, asked for one item ahead so that the
// atomic's latency hides behind the current block; a CTA that starts late (its SM held
// by a concurrent bin of the same evaluation) then takes fewer items instead of a fixed
// share.  Without a counter: the fixed grid stride `stride_next`.
__device__ __forceinline__ int take_work(int* ctr, int stride_next) {
    return ctr ? atomicAdd(ctr, 1) : stride_next;
}

// Work items of one launch: the host's count, or fewer when the list is filled on the
// device during the evaluation (the mixed path's FP64 redo lists).
__device__ __forceinline__ int work_count(const LLArgs& a) {
    return a.nwork_dev ? min(*a.nwork_dev, a.nwork) : a.nwork;
}

// A block whose FP32 factorisation breaks down (non-positive pivot) is queued for the FP64
// fallback pass instead of failing the evaluation.
// With the mixed path's check, the block's error weight: its conditioning indicator
// (written by the same thread before) times 1 + u_i / b_i, since the quadratic form's
// rounding error grows with the form itself; 0 for a block recomputed in FP64.
__device__ __forceinline__ void finish_block(const LLArgs& a, int blk, int b, double s, double su, int failed) {
    double ell = -0.5 * (s + (double)b * kLog2Pi);
    if (failed || !(ell == ell)) {
        ell = -INFINITY;
        if (a.fb) a.fb[1 + atomicAdd(a.fb, 1)] = blk;
        else record_fail(a.fail, blk);
        if (a.ind_blk) a.ind_blk[blk] = 0.0f;  // recomputed in FP64: exact for the check
    } else if (a.ind_blk) {
        a.ind_blk[blk] = (float)((double)a.ind_blk[blk] * (1.0 + su / (double)(b > 0 ? b : 1)));
    }
    a.ell_blk[blk] = ell;
    a.u_blk[blk] = su;
}

}  // namespace
