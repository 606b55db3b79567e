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

__device__ __forceinline__ float matern32(int nu, float sigma2, float x) {
    const float e = expf(-x);
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
