// bv_device.cuh -- device helpers shared by the FP64 block kernels (log-likelihood and
// prediction): packed-triangle indexing, the table-driven exponential and the Matern
// covariance at half-integer smoothness (Eq. 5).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bv_internal.h"

namespace {

// Row-major packed lower triangle: element (r, c), c <= r, at r(r+1)/2 + c.
__device__ __forceinline__ int pk(int r, int c) { return (r * (r + 1) >> 1) + c; }

// Inverse of pk over a full triangle: flat index f -> (r, c).
__device__ __forceinline__ void tri_rc(int f, int& r, int& c) {
    int rr = (int)((sqrtf(8.0f * (float)f + 1.0f) - 1.0f) * 0.5f);
    if (((rr + 1) * (rr + 2) >> 1) <= f) ++rr;
    if ((rr * (rr + 1) >> 1) > f) --rr;
    r = rr;
    c = f - (rr * (rr + 1) >> 1);
}

// e^{-x} for x >= 0 by Tang's table-driven method (see ExpConsts): reduction to
// |r| <= ln2/64, e^r - 1 by its Taylor polynomial through r^6 (truncation < 4e-18), one
// table multiply and an exponent-field scaling.  11 FP64 operations.  Results below
// e^{-700} are flushed to zero (a covariance entry that small is irrelevant next to the
// diagonal).  Accuracy: within 2 ulp of e^{-x} (checked against libm in the tests).
__device__ __forceinline__ double exp_neg(double x, const double* __restrict__ tab, double K, double L1,
                                          double L2) {
    const double shift = 6755399441055744.0;  // 1.5 * 2^52: adding it rounds to an integer
    const double s = fma(x, -K, shift);
    const int n = __double2loint(s);
    const double nd = s - shift;               // round(-x K), exact
    double r = fma(nd, -L1, -x);
    r = fma(nd, -L2, r);
    double q = fma(1.0 / 720.0, r, 1.0 / 120.0);
    q = fma(q, r, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    const double p = fma(q * r, r, r);         // e^r - 1
    const double t = tab[n & 31];
    const double v = fma(t, p, t);             // 2^{j/32} e^r in [0.98, 2)
    const int hi = __double2hiint(v) + ((n >> 5) << 20);
    const double res = __hiloint2double(hi, __double2loint(v));
    return x > 700.0 ? 0.0 : res;
}

// Matern correlation times sigma^2 at scaled distance x (Eq. 5, half-integer closed forms).
__device__ __forceinline__ double matern64t(int nu, double sigma2, double x, const double* tab, double K,
                                            double L1, double L2) {
    const double e = exp_neg(x, tab, K, L1, L2);
    if (nu == NU_HALF) return sigma2 * e;
    if (nu == NU_3HALF) return sigma2 * ((1.0 + x) * e);
    return sigma2 * ((1.0 + x * (1.0 + x * (1.0 / 3.0))) * e);
}

}  // namespace
