// bv_device.cuh -- device helpers shared by the FP64 block kernels (log-likelihood and
// prediction): packed-triangle indexing, the table-driven exponential and the Matern
// covariance at half-integer smoothness (Eq. 5).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bv_internal.h"

namespace {

constexpr double kPiD = 3.141592653589793238462643383279502884;

// Row-major packed lower triangle: element (r, c), c <= r, at r(r+1)/2 + c.
__device__ __forceinline__ int pk(int r, int c) { return (r * (r + 1) >> 1) + c; }

// Inverse range of coordinate k (k < 3) read without a dynamically indexed array, which
// would make the compiler copy the whole parameter struct to local memory.
__device__ __forceinline__ double inv_range_k(const DevTheta& th, int k) {
    return k == 0 ? th.inv_range[0] : (k == 1 ? th.inv_range[1] : th.inv_range[2]);
}

// A Cholesky pivot that is not a positive, finite, (nearly) normal number -- zero, negative,
// infinite or NaN -- tested on the high word with integer operations (off the FP64 pipe).
__device__ __forceinline__ bool bad_pivot(double p) {
    return (unsigned)(__double2hiint(p) - 1) >= 0x7FEFFFFFu;
}

// Inverse of pk over a full triangle: flat index f -> (r, c).
__device__ __forceinline__ void tri_rc(int f, int& r, int& c) {
    int rr = (int)((sqrtf(8.0f * (float)f + 1.0f) - 1.0f) * 0.5f);
    if (((rr + 1) * (rr + 2) >> 1) <= f) ++rr;
    if ((rr * (rr + 1) >> 1) > f) --rr;
    r = rr;
    c = f - (rr * (rr + 1) >> 1);
}

// e^{-x} for x >= 0 by Tang's table-driven method (see ExpConsts): reduction to
// |r| <= ln2/512, e^r - 1 by its Taylor polynomial through r^4 (truncation below 4e-17
// relative), one table multiply and an exponent-field scaling.  9 FP64 operations.
// Results below about e^{-700} are flushed to zero (a covariance entry that small is
// irrelevant next to the diagonal); the test is an integer compare of the high word
// (x >= 0, so its bit pattern orders like the value), off the FP64 pipe.  Accuracy: within 2 ulp of e^{-x} (checked against libm in the
// tests).
__device__ __forceinline__ double exp_neg(double x, const double* __restrict__ tab, double K, double L1,
                                          double L2) {
    const double shift = 6755399441055744.0;  // 1.5 * 2^52: adding it rounds to an integer
    const double s = fma(x, -K, shift);
    const int n = __double2loint(s);
    const double nd = s - shift;               // round(-x K), exact
    double r = fma(nd, -L1, -x);
    r = fma(nd, -L2, r);
    double q = fma(1.0 / 24.0, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    const double p = fma(q * r, r, r);         // e^r - 1
    const double t = tab[n & (BV_EXP_TAB - 1)];
    const double v = fma(t, p, t);             // 2^{j/256} e^r in [0.99, 2)
    const int hi = __double2hiint(v) + ((n >> 8) << 20);
    const double res = __hiloint2double(hi, __double2loint(v));
    return __double2hiint(x) > 0x4085E000 ? 0.0 : res;  // high word of 700.0
}

// Matern correlation rho(x) = 2^{1-nu}/G(nu) x^nu K_nu(x) of Eq. 5 for any nu > 0.
// K_mu and K_{mu+1} at |mu| <= 1/2 come from Temme's series for x <= 2 (N. M. Temme,
// "On the numerical evaluation of the modified Bessel function of the third kind",
// J. Comput. Phys. 19, 1975) and from Steed's evaluation of Temme's continued fraction
// for x > 2 (Thompson and Barnett, J. Comput. Phys. 64, 1986); the upward recurrence
// K_{a+1} = K_{a-1} + (2a/x) K_a (stable for K) reaches nu = nrec + mu.  The product with
// x^nu is formed in logarithms: the routine returns log rho(x) for x > 0.
__device__ __noinline__ double matern_gen_logcorr(const DevTheta& th, double x) {
    const double mu = th.mu, eps = 1e-17;
    double kmu, kmu1;
    if (x <= 2.0) {
        const double half = 0.5 * x;
        const double lnh = -log(half);           // log(2 / x)
        const double pimu = kPiD * mu;
        const double fpi = fabs(pimu) < 1e-12 ? 1.0 : pimu / sin(pimu);
        const double sg = mu * lnh;
        const double fs = fabs(sg) < 1e-12 ? 1.0 : sinh(sg) / sg;
        double f = fpi * (th.gam1 * cosh(sg) + th.gam2 * fs * lnh);  // f_0
        const double es = exp(sg);                                   // (x/2)^{-mu}
        double p = 0.5 * es / th.gampl;                              // (x/2)^{-mu} G(1+mu) / 2
        double q = 0.5 / (es * th.gammi);                            // (x/2)^{mu} G(1-mu) / 2
        double c = 1.0;
        const double h2 = half * half;
        double sum = f, sum1 = p;
        for (int k = 1; k < 500; ++k) {
            const double dk = (double)k;
            f = (dk * f + p + q) / (dk * dk - mu * mu);
            c *= h2 / dk;
            p /= dk - mu;
            q /= dk + mu;
            const double t = c * f;
            sum += t;
            sum1 += c * (p - dk * f);
            if (fabs(t) < fabs(sum) * eps) break;
        }
        kmu = sum;
        kmu1 = sum1 * (2.0 / x);
    } else {
        // continued fraction for the ratio, with Steed's simultaneous sum for the scale
        double b = 2.0 * (1.0 + x);
        double dd = 1.0 / b;
        double h = dd, dh = dd;
        double q1 = 0.0, q2 = 1.0;
        const double a1 = 0.25 - mu * mu;
        double q = a1, c = a1, a = -a1;
        double s = 1.0 + q * dh;
        for (int i = 2; i < 2000; ++i) {
            a -= 2.0 * (double)(i - 1);
            c = -a * c / (double)i;
            const double qn = (q1 - b * q2) / a;
            q1 = q2;
            q2 = qn;
            q += c * qn;
            b += 2.0;
            dd = 1.0 / (b + a * dd);
            dh = (b * dd - 1.0) * dh;
            h += dh;
            const double ds = q * dh;
            s += ds;
            if (fabs(ds) < fabs(s) * eps) break;
        }
        h *= a1;
        // K_mu = sqrt(pi / (2x)) e^{-x} / s, formed in logarithms below
        kmu = sqrt(kPiD / (2.0 * x)) / s;           // times e^{-x}
        kmu1 = kmu * (mu + x + 0.5 - h) / x;
    }
    // upward recurrence in the order: K_{mu+1}, ..., K_{mu+nrec}
    double km = kmu, kc = kmu1;
    double knu = th.nrec == 0 ? kmu : kmu1;
    for (int i = 1; i < th.nrec; ++i) {
        const double kn = km + (2.0 * (mu + (double)i) / x) * kc;
        km = kc;
        kc = kn;
        knu = kn;
    }
    const double lk = log(knu) - (x > 2.0 ? x : 0.0);
    return th.lognorm + th.nu * log(x) + lk;
}

__device__ __forceinline__ double matern_gen_corr(const DevTheta& th, double x) {
    if (!(x > 0.0)) return 1.0;
    if (x > 745.0) return 0.0;
    return exp(matern_gen_logcorr(th, x));
}

// Per-evaluation table of a general-nu Matern (built by k_gtab_build for every dataset):
// on each octave [2^e, 2^{e+1}), e = GTAB_E0 .. GTAB_E0 + GTAB_NOCT - 1, the Chebyshev
// expansion of degree GTAB_DEG - 1 of L(x) = x + log rho(x) in t = 2 x / 2^e - 3.  L has
// its only singularity at x = 0, so each octave converges at the same geometric rate,
// and rho = exp(-(x - L)) keeps the relative accuracy over the whole range (about 1e-13
// for nu <= 20).  Distances outside the tabulated octaves use K_nu directly.
#define GTAB_E0 (-40)
#define GTAB_NOCT 49
#define GTAB_DEG 19
#define GTAB_SIZE (GTAB_NOCT * GTAB_DEG)

__device__ __forceinline__ double matern_gen_tab(const double* __restrict__ tab, const DevTheta* __restrict__ g,
                                                 double x, const double* etab, double K, double L1, double L2) {
    const long long ux = __double_as_longlong(x);
    const int ex = (int)((ux >> 52) & 0x7ff) - 1023;
    const int o = ex - GTAB_E0;
    if (x == 0.0) return 1.0;
    if (o < 0 || o >= GTAB_NOCT) return matern_gen_corr(*g, x);
    const double m = __longlong_as_double((ux & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);  // [1, 2)
    const double t = 2.0 * m - 3.0;
    const double* c = tab + o * GTAB_DEG;
    double b1 = 0.0, b2 = 0.0;
#pragma unroll
    for (int k = GTAB_DEG - 1; k >= 1; --k) {
        const double b0 = fma(2.0 * t, b1, c[k] - b2);
        b2 = b1;
        b1 = b0;
    }
    const double L = fma(t, b1, c[0] - b2);
    return exp_neg(fmax(x - L, 0.0), etab, K, L1, L2);
}

// Matern covariance sigma^2 rho(x) at scaled distance x (Eq. 5, half-integer closed forms
// through the table-driven exponential).
__device__ __forceinline__ double matern64t(int nu, double sigma2, double x, const double* tab, double K,
                                            double L1, double L2) {
    const double se = sigma2 * exp_neg(x, tab, K, L1, L2);
    if (nu == NU_HALF) return se;
    if (nu == NU_3HALF) return fma(x, se, se);                       // sigma^2 (1 + x) e^{-x}
    return fma(x * fma(x, 1.0 / 3.0, 1.0), se, se);                  // sigma^2 (1 + x + x^2/3) e^{-x}
}

// Scaled distance sqrt(acc) for acc >= 0 through the reciprocal square root (within
// 2 ulp); acc == 0 (and subnormal acc) gives 0, tested on the high word off the FP64 pipe.
__device__ __forceinline__ double dist_of(double acc) {
    return __double2hiint(acc) > 0 ? acc * rsqrt(acc) : 0.0;
}

// FP32 evaluation of the same table (mixed precision: covariance entries are FP32).
__device__ __forceinline__ float matern_gen_tab32(const double* __restrict__ tab, const DevTheta* __restrict__ g,
                                                  float x) {
    const int ux = __float_as_int(x);
    const int ex = ((ux >> 23) & 0xff) - 127;
    const int o = ex - GTAB_E0;
    if (x == 0.0f) return 1.0f;
    if (o < 0 || o >= GTAB_NOCT) return (float)matern_gen_corr(*g, (double)x);
    const float m = __int_as_float((ux & 0x007FFFFF) | 0x3F800000);  // [1, 2)
    const float t = 2.0f * m - 3.0f;
    const double* c = tab + o * GTAB_DEG;
    float b1 = 0.0f, b2 = 0.0f;
#pragma unroll
    for (int k = GTAB_DEG - 1; k >= 1; --k) {
        const float b0 = fmaf(2.0f * t, b1, (float)c[k] - b2);
        b2 = b1;
        b1 = b0;
    }
    const float L = fmaf(t, b1, (float)c[0] - b2);
    return expf(-fmaxf(x - L, 0.0f));
}

// Any nu: closed forms for the half-integers, the dataset's table otherwise.  `g` points
// at the theta in global memory (read only off the table's range).
__device__ __forceinline__ double matern64g(const double* __restrict__ gtab, const DevTheta* __restrict__ g, int nu,
                                            double sigma2, double x, const double* tab, double K, double L1,
                                            double L2) {
    if (nu == NU_GENERAL) return sigma2 * matern_gen_tab(gtab, g, x, tab, K, L1, L2);
    return matern64t(nu, sigma2, x, tab, K, L1, L2);
}

}  // namespace
