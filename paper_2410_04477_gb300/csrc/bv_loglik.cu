// bv_loglik.cu -- fused block-Vecchia log-likelihood kernels (Eq. 4, Algorithm 1).
//
// Per block i with m conditioning points and b block points, Algorithm 1 factors
// Sigma^con, solves for Sigma'^cross and y', forms Sigma^new = Sigma^lk - V^T V and
// mu = V^T y', factors Sigma^new and solves for v.  All of those are the steps of ONE
// Cholesky factorisation of the augmented (N+1) x (N+1) matrix (N = m + b)
//
//        [ Sigma^con     Sigma^cross   y_NN ]
//        [ Sigma^crossT  Sigma^lk      y_B  ]
//        [ y_NN^T        y_B^T         *    ]
//
// by block-Cholesky algebra: its leading m x m factor is L = chol(Sigma^con), the rows
// below it hold V^T = (L^{-1} Sigma^cross)^T and y'^T, the trailing b x b factor is
// L' = chol(Sigma^new), and the last row's entries under the block columns are
// v = L'^{-1}(y_B - mu).  So u = sum_{k>=m} z_k^2 and d = sum_{k>=m} log p_k, with z the
// last row of the factor and p_k the pivots (squared diagonal of the factor), and
//        ell_i = -(u + d + b log 2 pi) / 2.
// The kernels generate the matrix (Matern, Eq. 5) straight into shared memory, factor it
// in place (right-looking, one or two columns per step in FP64, 4-column tile panels in
// mixed precision) and reduce ell_i, so nothing but the
// locations, y and the index lists is read from HBM and one double per block is written.
//
// Paths:
//   k_ll_fp64<NT>   FP64 packed lower triangle in shared memory (N up to 233 for d=3; 231 with two-column steps)
//   k_ll_mixed<NT>  FP32 covariance (block-local coordinates), FP32 updates; pivots,
//                   log-determinant and quadratic form accumulated in FP64
//   k_ll_large<NT>  FP64, packed triangle in a global-memory workspace slot (any N)
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "bv_device.cuh"
#include "bv_internal.h"
#include "bv_ll_block.cuh"

namespace {

// ---------------------------------------------------------------------------------
// FP64, shared memory.  Layout (doubles): A packed (N+1)(N+2)/2 | col[2 or 4][N+1] | pts[d][N]
// ---------------------------------------------------------------------------------

// Column c of the factor, by one warp: its entries in rows c..N have been updated with
// every column before it except those in `prev` (np of them, each a finished column held
// contiguously by row, applied here in order); then the pivot and the scaling, the scaled
// column written to A and to out.  Raises *fail on a bad pivot.
template <int NP>
__device__ __forceinline__ void fp64_column(double* A, int c, int N, int lane, const double* const (&prev)[NP], int np,
                                            double* out, int* fail) {
    for (int j = c + lane; j <= N; j += 32) {
        double v = A[pk(j, c)];
#pragma unroll
        for (int q = 0; q < NP; ++q)
            if (q < np) v = fma(-prev[q][j], prev[q][c], v);
        A[pk(j, c)] = v;
    }
    __syncwarp();
    const double p = A[pk(c, c)];
    if (bad_pivot(p) && lane == 0) *fail = 1;
    const double rs = rsqrt(p);
    for (int j = c + 1 + lane; j <= N; j += 32) {
        const double v = A[pk(j, c)] * rs;
        A[pk(j, c)] = v;
        out[j] = v;
    }
    __syncwarp();
}

// W2 selects the step width of the factorisation: one column per barrier (two column
// buffers) or two (four buffers); both give the same results bit for bit, and the planner
// times both per size bin (one column wins on small blocks, where the panel warp's pivot
// chain is the critical path, two on large ones, where the trailing update is).
template <int NT, bool GEN, bool W2>
__global__ void __launch_bounds__(NT) k_ll_fp64(LLArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double* sm = reinterpret_cast<double*>(smraw);
    __shared__ double etab[BV_EXP_TAB];
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < BV_EXP_TAB; i += NT) etab[i] = a.ex.tab[i];
    const double eK = a.ex.k, eL1 = a.ex.l1, eL2 = a.ex.l2;

    __shared__ int s_w;
    const int nwork = work_count(a);
    if (tid == 0) s_w = take_work(a.ctr, blockIdx.x);
    __syncthreads();
    for (int w = s_w; w < nwork; w = s_w) {
        const int nx = tid == 0 ? take_work(a.ctr, w + gridDim.x) : 0;
        const int blk = a.work[w];
        const int64_t b0 = a.bptr[blk], n0 = a.nptr[blk];
        const int b = (int)(a.bptr[blk + 1] - b0), m = (int)(a.nptr[blk + 1] - n0);
        const int N = m + b, R = N + 1;
        const DevTheta th = a.theta[a.bds[blk]];
        double* A = sm;
        double* colbuf = A + ((R * (R + 1)) >> 1);  // column buffers of R doubles
        double* px = colbuf + (W2 ? 4 : 2) * R;
        const int d = a.d;

        // gather: conditioning points first, then the block (Algorithm 1 order)
        for (int t = tid; t < N; t += NT) {
            const int g = t < m ? a.nidx[n0 + t] : a.pidx[b0 + (t - m)];
            for (int k = 0; k < d; ++k) px[k * N + t] = a.locs[(int64_t)k * a.n_tot + g] * inv_range_k(th, k);
            A[pk(N, t)] = a.y[g];
            A[pk(t, t)] = th.sigma2 + th.nugget;  // diagonal of Eq. 5 + nugget: rho(0) = 1
        }
        if (tid == 0) {
            A[pk(N, N)] = 0.0;
            s_fail = 0;
        }
        __syncthreads();

        // covariance (Eq. 5), strictly lower triangle of rows 1..N-1: flat index f over that
        // triangle maps to (r' + 1, c) with (r', c) = tri_rc(f), packed index f + r' + 1
        const int T = (N * (N - 1)) >> 1;
        for (int f = tid; f < T; f += NT) {
            int r, c;
            tri_rc(f, r, c);
            ++r;
            double acc = 0.0;
            for (int k = 0; k < d; ++k) {
                const double t = px[k * N + r] - px[k * N + c];
                acc = fma(t, t, acc);
            }
            // x = acc / sqrt(acc) through the reciprocal square root (within 2 ulp)
            const double x = dist_of(acc);
            const double v = GEN ? matern64g(a.gtab + (int64_t)a.bds[blk] * GTAB_SIZE, a.theta + a.bds[blk],
                                             th.nu_code, th.sigma2, x, etab, eK, eL1, eL2)
                                 : matern64t(th.nu_code, th.sigma2, x, etab, eK, eL1, eL2);
            A[f + r] = v;
        }
        __syncthreads();

        if constexpr (!W2) {
            // column 0 (warp 0)
            if (warp == 0) {
                const double* none[1] = {nullptr};
                fp64_column<1>(A, 0, N, lane, none, 0, colbuf, &s_fail);
            }
            __syncthreads();

            // right-looking steps: warp 0 finishes column k+1 (update, pivot, scale) while
            // the other warps apply column k to the rest of the trailing triangle; one
            // barrier per step
            for (int k = 0; k + 1 < N; ++k) {
                const double* cur = colbuf + (k & 1) * R;
                double* nxt = colbuf + ((k & 1) ^ 1) * R;
                const int kk = k + 1;
                if (warp == 0) {
                    const double* p1[1] = {cur};
                    fp64_column<1>(A, kk, N, lane, p1, 1, nxt, &s_fail);
                } else {
                    // rows kk+1..N, columns kk+1..row, two independent elements per iteration
                    const int S = N - kk;
                    const int TS = (S * (S + 1)) >> 1;
                    constexpr int NU = NT - 32;
                    for (int f = tid - 32; f < TS; f += 2 * NU) {
                        int r1, c1, r2, c2;
                        tri_rc(f, r1, c1);
                        const bool two = f + NU < TS;
                        tri_rc(two ? f + NU : f, r2, c2);
                        const int j1 = kk + 1 + r1, i1 = kk + 1 + c1, j2 = kk + 1 + r2, i2 = kk + 1 + c2;
                        const double a1 = A[pk(j1, i1)], x1 = cur[j1], y1 = cur[i1];
                        const double a2 = A[pk(j2, i2)], x2 = cur[j2], y2 = cur[i2];
                        A[pk(j1, i1)] = fma(-x1, y1, a1);
                        if (two) A[pk(j2, i2)] = fma(-x2, y2, a2);
                    }
                }
                __syncthreads();
            }
        } else {
            // columns 0 and 1 (warp 0)
            if (warp == 0) {
                const double* none[1] = {nullptr};
                fp64_column<1>(A, 0, N, lane, none, 0, colbuf, &s_fail);
                if (N > 1) {
                    const double* p0[1] = {colbuf};
                    fp64_column<1>(A, 1, N, lane, p0, 1, colbuf + R, &s_fail);
                }
            }
            __syncthreads();

            // right-looking steps of two columns: with columns k and k+1 finished (buffers
            // c0, c1), warp 0 finishes columns k+2 and k+3 (their updates by k and k+1, then
            // k+3's by k+2; pivots; scaling) while the other warps apply columns k and k+1 to
            // the trailing triangle from row and column k+4; one barrier per two columns.
            // Every entry receives its updates in column order, as in a one-column-per-step
            // factorisation, so the results are the same bit for bit.
            for (int k = 0; k + 2 < N; k += 2) {
                const int sel = (k >> 1) & 1;
                const double* c0 = colbuf + (2 * sel) * R;
                const double* c1 = c0 + R;
                double* n0b = colbuf + (2 * (sel ^ 1)) * R;
                double* n1b = n0b + R;
                if (warp == 0) {
                    const double* p2[2] = {c0, c1};
                    fp64_column<2>(A, k + 2, N, lane, p2, 2, n0b, &s_fail);
                    if (k + 3 < N) {
                        const double* p3[3] = {c0, c1, n0b};
                        fp64_column<3>(A, k + 3, N, lane, p3, 3, n1b, &s_fail);
                    }
                } else {
                    const int kk = k + 4;  // trailing triangle: rows kk..N, columns kk..row
                    const int S = N - kk + 1;
                    if (S > 0) {
                        const int TS = (S * (S + 1)) >> 1;
                        constexpr int NU = NT - 32;
                        for (int f = tid - 32; f < TS; f += NU) {
                            int r, c;
                            tri_rc(f, r, c);
                            const int j = kk + r, i = kk + c;
                            const double v = fma(-c0[j], c0[i], A[pk(j, i)]);
                            A[pk(j, i)] = fma(-c1[j], c1[i], v);
                        }
                    }
                }
                __syncthreads();
            }
        }

        // u + d over the block columns (warp 0)
        if (warp == 0) {
            const double2 s2 = warp_terms(m, N, lane, [&](int k) { return A[pk(N, k)]; },
                                          [&](int k) { return log(A[pk(k, k)]); });
            const double s = s2.x, su = s2.y;
            if (lane == 0) {
                double ell = -0.5 * (s + (double)b * kLog2Pi);
                if (s_fail || !(ell == ell)) {
                    ell = -INFINITY;
                    record_fail(a.fail, blk);
                }
                a.ell_blk[blk] = ell;
                a.u_blk[blk] = su;
                s_w = nx;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------
// Mixed: FP32 covariance and updates, FP64 log-determinant and quadratic form.
// The augmented matrix is held as 4x4 tiles (lower tile triangle; tile q = I(I+1)/2 + J
// starts at 16 q floats; row r of a tile, 16 bytes, is stored at row slot r ^ ((q >> 1) & 3),
// so that the same row of eight consecutive tiles falls on eight distinct 16-byte bank
// groups without padding), factored by 4-column panels:
//   panel p:  every thread solves its rows of tile column p against the factored 4x4
//             diagonal tile (read from `dfac`) and stores them, contiguous and swizzled
//             the same way, in `pbuf` (in place only for the tile holding row N, whose
//             z entries are read at the end; one barrier);
//   update:   every trailing tile (I,J), p < J <= I, is updated by one thread,
//             A_IJ -= P_I P_J^T with 128-bit shared-memory accesses, P_I and P_J read
//             from `pbuf` (consecutive threads take consecutive J: conflict-free); the
//             thread that updates the next diagonal tile (always thread 0) factors it at
//             once into `dfac` (look-ahead), so the pivots never sit on every thread's path.
// Coordinates are taken relative to the block centroid in FP64 and rounded to FP32, so
// FP32 differences keep their relative accuracy for nearby points.
// ---------------------------------------------------------------------------------
constexpr int kTS = 16;  // floats per stored 4x4 tile

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ int tile_index(int I, int J) { return ((I * (I + 1)) >> 1) + J; }
// Row r (4 floats, 16-byte aligned) of tile q in a swizzled tile array.
__device__ __forceinline__ float* tile_row(float* t, int q, int r) { return t + q * kTS + 4 * (r ^ ((q >> 1) & 3)); }
__device__ __forceinline__ const float* tile_row(const float* t, int q, int r) {
    return t + q * kTS + 4 * (r ^ ((q >> 1) & 3));
}

// Factor the 4x4 diagonal tile q of `tiles` (pivot columns c < nc) into dfac:
// dfac[0..15] = L (strictly lower part), dfac[16..19] = 1/sqrt(pivot), dfac[20..23] = pivot.
// Every pivot gets dlo, the part of the matrix diagonal its FP32 value misses (a diagonal
// entry enters the factorisation only as its column's pivot).  Writes the pivots of global
// columns k0.. to piv, row N's entries (if row N lies in this tile) to ydiag, and raises
// *fail on a non-positive pivot.
__device__ __forceinline__ void factor_diag(const float* tiles, int qd, int nc, int k0, int N, float* dfac,
                                            float* piv, float* ydiag, int* fail, float dlo) {
    float D[16];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float4 q = ld4(tile_row(tiles, qd, r));
        D[4 * r] = q.x;
        D[4 * r + 1] = q.y;
        D[4 * r + 2] = q.z;
        D[4 * r + 3] = q.w;
    }
    float rs[4], pv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        pv[c] = D[5 * c] + dlo;
        // correctly rounded 1/sqrt: the approximate reciprocal square root errs to one
        // side, and that shared bias of every column scaling turns into a bias of the
        // Schur complements that grows with the block's conditioning
        rs[c] = c < nc ? __frsqrt_rn(pv[c]) : 0.0f;
#pragma unroll
        for (int r = c + 1; r < 4; ++r) D[4 * r + c] *= rs[c];
#pragma unroll
        for (int r = c + 1; r < 4; ++r)
#pragma unroll
            for (int q = c + 1; q <= r; ++q) D[4 * r + q] = fmaf(-D[4 * r + c], D[4 * q + c], D[4 * r + q]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) st4(dfac + 4 * r, make_float4(D[4 * r], D[4 * r + 1], D[4 * r + 2], D[4 * r + 3]));
    st4(dfac + 16, make_float4(rs[0], rs[1], rs[2], rs[3]));
    st4(dfac + 20, make_float4(pv[0], pv[1], pv[2], pv[3]));
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (c < nc) {
            piv[k0 + c] = pv[c];
            if (!(pv[c] > 0.0f)) *fail = 1;
        }
    const int ra = N - k0;  // row N inside this tile?
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (r == ra) {
#pragma unroll
            for (int c = 0; c < 4; ++c) ydiag[c] = (c < nc && c < r) ? D[4 * r + c] : 0.0f;
        }
}

// Group synchronisation: a whole CTA, or one warp that owns its block.
template <bool WARP>
__device__ __forceinline__ void gsync() {
    if (WARP) __syncwarp();
    else __syncthreads();
}

// Floats of shared memory one mixed-precision block of augmented size <= nmax needs.
// Layout: tiles (T(T+1)/2 x 16) | pbuf (T x 16) | px (3 N) | y (N) | pivots (N) | dfac (28).
__host__ __device__ __forceinline__ int mixed_floats(int nmax) {
    const int T = (nmax + 1 + 3) >> 2;
    return ((((T * (T + 1)) >> 1) * kTS + T * kTS + 5 * nmax + 28) + 3) & ~3;
}

// One block, mixed precision, by a group of NG threads (tid in [0, NG)).  sm: the
// group's shared region (mixed_floats(N) floats, 16-byte aligned).  Returns (sum of
// z^2 + log pivot, sum of z^2) over the block columns, valid in thread 0, and sets *fail.
template <int NG, bool WARP, bool GEN>
__device__ __forceinline__ double2 mixed_block(const LLArgs& a, int blk, float* sm, int tid, int* fail,
                                               const float* t32) {
    const int64_t b0 = a.bptr[blk], n0 = a.nptr[blk];
    const int b = (int)(a.bptr[blk + 1] - b0), m = (int)(a.nptr[blk + 1] - n0);
    const int N = m + b, R = N + 1, T = (R + 3) >> 2;
    const DevTheta th = a.theta[a.bds[blk]];
    float* tiles = sm;
    float* pbuf = tiles + ((T * (T + 1)) >> 1) * kTS;
    float* px = pbuf + T * kTS;
    float* yv = px + 3 * N;
    float* piv = yv + N;
    float* dfac = sm + ((((((T * (T + 1)) >> 1) * kTS + T * kTS + 5 * N) + 3) & ~3));  // 16-byte aligned
    float* ydiag = dfac + 24;
    const int d = a.d;
    const float s2 = th.sigma2_f, tau2 = th.nugget_f;
    // offsets from the block centroid in FP64 (exact enough to keep the block-local
    // coordinates accurate), rounded to FP32 and scaled by 1/beta in FP32: the FP64 pipe,
    // 1/64 of the FP32 rate on this part, does only the subtraction and the conversion
    const float ir0 = th.inv_range_f[0], ir1 = th.inv_range_f[1], ir2 = th.inv_range_f[2];

    for (int t = tid; t < N; t += NG) {
        const int g = t < m ? a.nidx[n0 + t] : a.pidx[b0 + (t - m)];
        const double* cb = a.cent + (int64_t)blk * d;
        px[t] = (float)(a.locs[g] - cb[0]) * ir0;
        px[N + t] = d > 1 ? (float)(a.locs[a.n_tot + g] - cb[1]) * ir1 : 0.0f;
        px[2 * N + t] = d > 2 ? (float)(a.locs[2 * a.n_tot + g] - cb[2]) * ir2 : 0.0f;
        yv[t] = (float)a.y[g];
    }
    gsync<WARP>();

    // fill: one 4x4 tile per thread (padding rows/columns and the strictly upper part of
    // diagonal tiles get 0; row N is y)
    const int NTL = (T * (T + 1)) >> 1;
    for (int q = tid; q < NTL; q += NG) {
        int I, J;
        tri_rc(q, I, J);
        float cx[4], cy[4], cz[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = (J << 2) + e;
            const bool ok = c < N;
            cx[e] = ok ? px[c] : 0.0f;
            cy[e] = ok ? px[N + c] : 0.0f;
            cz[e] = ok ? px[2 * N + c] : 0.0f;
        }
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int r = (I << 2) + rr;
            float o[4];
            if (r < N) {
                const float rx = px[r], ry = px[N + r], rz = px[2 * N + r];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = (J << 2) + e;
                    const float t0 = rx - cx[e], t1 = ry - cy[e], t2 = rz - cz[e];
                    const float xf = sqrtf(fmaf(t2, t2, fmaf(t1, t1, t0 * t0)));
                    float v = (GEN && th.nu_code == NU_GENERAL)
                                  ? s2 * matern_gen_tab32(a.gtab + (int64_t)a.bds[blk] * GTAB_SIZE,
                                                          a.theta + a.bds[blk], xf)
                                  : matern32(th.nu_code, s2, xf, t32, a.ex);
                    if (r == c) v += tau2;
                    o[e] = c <= r ? v : 0.0f;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = (J << 2) + e;
                    o[e] = (r == N && c < N) ? yv[c] : 0.0f;
                }
            }
            st4(tile_row(tiles, q, rr), make_float4(o[0], o[1], o[2], o[3]));
        }
    }
    gsync<WARP>();
    if (tid == 0) factor_diag(tiles, 0, min(4, N), 0, N, dfac, piv, ydiag, fail, th.diag_lo_f);
    gsync<WARP>();

    for (int p = 0; (p << 2) < N; ++p) {
        const int k0 = p << 2, nc = min(4, N - k0);
        // rows of tile column p below the diagonal tile
        {
            float L[16], rs[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float4 q = ld4(dfac + 4 * r);
                L[4 * r] = q.x;
                L[4 * r + 1] = q.y;
                L[4 * r + 2] = q.z;
                L[4 * r + 3] = q.w;
            }
            {
                const float4 q = ld4(dfac + 16);
                rs[0] = q.x;
                rs[1] = q.y;
                rs[2] = q.z;
                rs[3] = q.w;
            }
            for (int r = k0 + 4 + tid; r < (T << 2); r += NG) {
                float* rowp = tile_row(tiles, tile_index(r >> 2, p), r & 3);
                const float4 q = ld4(rowp);
                float x[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float v = x[c];
#pragma unroll
                    for (int q2 = 0; q2 < c; ++q2) v = fmaf(-x[q2], L[4 * c + q2], v);
                    x[c] = c < nc ? v * rs[c] : 0.0f;
                }
                // the trailing update reads the solved column from pbuf; of tile column p
                // only the tile holding row N (its z entries) is read again in place
                if ((r >> 2) == (N >> 2)) st4(rowp, make_float4(x[0], x[1], x[2], x[3]));
                st4(tile_row(pbuf, (r >> 2) - p - 1, r & 3), make_float4(x[0], x[1], x[2], x[3]));
            }
        }
        gsync<WARP>();
        // trailing tiles; thread 0 starts with the next diagonal tile and factors it
        const int S = T - p - 1;
        const int cnt = (S * (S + 1)) >> 1;
        for (int q = tid; q < cnt; q += NG) {
            int ii, jj;
            tri_rc(q, ii, jj);
            const int I = p + 1 + ii, J = p + 1 + jj, qa = tile_index(I, J);
            float pi[16], pj[16];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float4 u = ld4(tile_row(pbuf, ii, r)), v = ld4(tile_row(pbuf, jj, r));
                pi[4 * r] = u.x; pi[4 * r + 1] = u.y; pi[4 * r + 2] = u.z; pi[4 * r + 3] = u.w;
                pj[4 * r] = v.x; pj[4 * r + 1] = v.y; pj[4 * r + 2] = v.z; pj[4 * r + 3] = v.w;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float* at = tile_row(tiles, qa, r);
                const float4 acc = ld4(at);
                float o[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int k = 0; k < 4; ++k) o[c] = fmaf(-pi[4 * r + k], pj[4 * c + k], o[c]);
                st4(at, make_float4(o[0], o[1], o[2], o[3]));
            }
            if (q == 0 && ((p + 1) << 2) < N)
                factor_diag(tiles, qa, min(4, N - ((p + 1) << 2)), (p + 1) << 2, N, dfac, piv, ydiag, fail, th.diag_lo_f);
        }
        gsync<WARP>();
    }

    // quadratic form and log-determinant terms of the block columns, accumulated in FP64,
    // the logarithm of each pivot taken in FP64; by the first warp only, the totals are
    // valid in thread 0
    if (tid >= 32) return make_double2(0.0, 0.0);
    if (a.ind_blk) {
        const float ind = warp_indicator(N, tid, s2 + tau2, [&](int k) { return piv[k]; });
        if (tid == 0) a.ind_blk[blk] = ind;
    }
    return warp_terms(
        m, N, tid,
        [&](int k) {
            return (k >> 2) == (N >> 2) ? (double)ydiag[k & 3]
                                        : (double)tile_row(tiles, tile_index(N >> 2, k >> 2), N & 3)[k & 3];
        },
        [&](int k) { return log((double)piv[k]); });
}

// CTA per block.
template <int NT, bool GEN>
__global__ void __launch_bounds__(NT) k_ll_mixed(LLArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float* sm = reinterpret_cast<float*>(smraw);
    __shared__ int s_fail;
    __shared__ int s_w;
    __shared__ float t32[64];
    const int tid = threadIdx.x;
    for (int i = tid; i < 64; i += NT) t32[i] = a.ex.t32[i];
    if (tid == 0) s_w = take_work(a.ctr, blockIdx.x);
    __syncthreads();
    for (int w = s_w; w < a.nwork; w = s_w) {
        const int nx = tid == 0 ? take_work(a.ctr, w + gridDim.x) : 0;
        const int blk = a.work[w];
        if (tid == 0) s_fail = 0;
        __syncthreads();
        const double2 sr = mixed_block<NT, false, GEN>(a, blk, sm, tid, &s_fail, t32);
        if (tid == 0) {
            finish_block(a, blk, (int)(a.bptr[blk + 1] - a.bptr[blk]), sr.x, sr.y, s_fail);
            s_w = nx;
        }
        __syncthreads();
    }
}

// Warp per block: each of the NT/32 warps of a CTA factors its own blocks with warp
// synchronisation only (small blocks, where CTA-wide barriers dominate).
template <int NT, bool GEN>
__global__ void __launch_bounds__(NT) k_ll_mixed_w(LLArgs a, int region_floats) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int WPB = NT / 32;
    __shared__ int s_fail[WPB];
    __shared__ float t32[64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 64; i += NT) t32[i] = a.ex.t32[i];
    __syncthreads();
    float* sm = reinterpret_cast<float*>(smraw) + (size_t)warp * region_floats;
    int w = __shfl_sync(0xffffffffu, lane == 0 ? take_work(a.ctr, blockIdx.x * WPB + warp) : 0, 0);
    while (w < a.nwork) {
        const int nx = lane == 0 ? take_work(a.ctr, w + gridDim.x * WPB) : 0;
        const int blk = a.work[w];
        if (lane == 0) s_fail[warp] = 0;
        __syncwarp();
        const double2 part = mixed_block<32, true, GEN>(a, blk, sm, lane, &s_fail[warp], t32);
        __syncwarp();
        if (lane == 0) finish_block(a, blk, (int)(a.bptr[blk + 1] - a.bptr[blk]), part.x, part.y, s_fail[warp]);
        __syncwarp();
        w = __shfl_sync(0xffffffffu, nx, 0);
    }
}

// ---------------------------------------------------------------------------------
// FP64, one warp per block (several blocks per CTA): for small blocks, where a CTA's
// barriers and partly filled update warps cost more than the work.  Same arithmetic as
// k_ll_fp64 (gather with the diagonal, strictly-lower covariance, right-looking Cholesky
// of the augmented matrix, Algorithm 1 order); every column's pivot, scaling and trailing
// update by the warp's 32 lanes with warp synchronisation only.  Layout per warp
// (doubles, region_doubles each): A packed (N+1)(N+2)/2 | col[N+1] | pts[d][N].
// ---------------------------------------------------------------------------------
template <int NT, bool GEN>
__global__ void __launch_bounds__(NT) k_ll_fp64_w(LLArgs a, int region_doubles) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int WPB = NT / 32;
    __shared__ double etab[BV_EXP_TAB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < BV_EXP_TAB; i += NT) etab[i] = a.ex.tab[i];
    __syncthreads();
    const double eK = a.ex.k, eL1 = a.ex.l1, eL2 = a.ex.l2;
    double* A = reinterpret_cast<double*>(smraw) + (size_t)warp * region_doubles;
    const int nwork = work_count(a);
    int w = __shfl_sync(0xffffffffu, lane == 0 ? take_work(a.ctr, blockIdx.x * WPB + warp) : 0, 0);
    while (w < nwork) {
        const int nx = lane == 0 ? take_work(a.ctr, w + gridDim.x * WPB) : 0;
        const int blk = a.work[w];
        const int64_t b0 = a.bptr[blk], n0 = a.nptr[blk];
        const int b = (int)(a.bptr[blk + 1] - b0), m = (int)(a.nptr[blk + 1] - n0);
        const int N = m + b, R = N + 1;
        const DevTheta th = a.theta[a.bds[blk]];
        double* col = A + ((R * (R + 1)) >> 1);
        double* px = col + R;
        const int d = a.d;

        for (int t = lane; t < N; t += 32) {
            const int g = t < m ? a.nidx[n0 + t] : a.pidx[b0 + (t - m)];
            for (int k = 0; k < d; ++k) px[k * N + t] = a.locs[(int64_t)k * a.n_tot + g] * inv_range_k(th, k);
            A[pk(N, t)] = a.y[g];
            A[pk(t, t)] = th.sigma2 + th.nugget;
        }
        if (lane == 0) A[pk(N, N)] = 0.0;
        __syncwarp();
        const int T = (N * (N - 1)) >> 1;
        for (int f = lane; f < T; f += 32) {
            int r, c;
            tri_rc(f, r, c);
            ++r;
            double acc = 0.0;
            for (int k = 0; k < d; ++k) {
                const double t = px[k * N + r] - px[k * N + c];
                acc = fma(t, t, acc);
            }
            const double x = dist_of(acc);
            A[f + r] = GEN ? matern64g(a.gtab + (int64_t)a.bds[blk] * GTAB_SIZE, a.theta + a.bds[blk], th.nu_code,
                                       th.sigma2, x, etab, eK, eL1, eL2)
                           : matern64t(th.nu_code, th.sigma2, x, etab, eK, eL1, eL2);
        }
        __syncwarp();

        bool bad = false;  // the same pivot in every lane: warp-uniform
        for (int k = 0; k < N; ++k) {
            const double p = A[pk(k, k)];
            bad = bad || bad_pivot(p);
            const double rs = rsqrt(p);
            for (int j = k + 1 + lane; j <= N; j += 32) {
                const double v = A[pk(j, k)] * rs;
                A[pk(j, k)] = v;
                col[j] = v;
            }
            __syncwarp();
            // trailing triangle, rows and columns k+1..N (row N: the forward solve of y)
            const int S = N - k;
            const int TS = (S * (S + 1)) >> 1;
            for (int f = lane; f < TS; f += 32) {
                int r, c;
                tri_rc(f, r, c);
                const int j = k + 1 + r, i = k + 1 + c;
                A[pk(j, i)] = fma(-col[j], col[i], A[pk(j, i)]);
            }
            __syncwarp();
        }
        const double2 s2 = warp_terms(m, N, lane, [&](int k) { return A[pk(N, k)]; },
                                      [&](int k) { return log(A[pk(k, k)]); });
        if (lane == 0) {
            double ell = -0.5 * (s2.x + (double)b * kLog2Pi);
            if (bad || !(ell == ell)) {
                ell = -INFINITY;
                record_fail(a.fail, blk);
            }
            a.ell_blk[blk] = ell;
            a.u_blk[blk] = s2.y;
        }
        __syncwarp();
        w = __shfl_sync(0xffffffffu, nx, 0);
    }
}

// ---------------------------------------------------------------------------------
// Large blocks: same algorithm in FP64 with the packed triangle in a global workspace
// slot (one slot per CTA; the grid never exceeds the number of slots).
// ---------------------------------------------------------------------------------
template <int NT, bool GEN>
__global__ void __launch_bounds__(NT) k_ll_large(LLArgs a) {
    __shared__ double etab[BV_EXP_TAB];
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* slot = a.ws + (int64_t)blockIdx.x * a.ws_stride;
    for (int i = tid; i < BV_EXP_TAB; i += NT) etab[i] = a.ex.tab[i];
    const double eK = a.ex.k, eL1 = a.ex.l1, eL2 = a.ex.l2;
    const int nwork = a.dyn ? *a.fb : work_count(a);
    const int* work = a.dyn ? a.fb + 1 : a.work;

    __shared__ int s_w;
    if (tid == 0) s_w = take_work(a.ctr, blockIdx.x);
    __syncthreads();
    for (int w = s_w; w < nwork; w = s_w) {
        const int nx = tid == 0 ? take_work(a.ctr, w + gridDim.x) : 0;
        const int blk = work[w];
        const int64_t b0 = a.bptr[blk], n0 = a.nptr[blk];
        const int b = (int)(a.bptr[blk + 1] - b0), m = (int)(a.nptr[blk + 1] - n0);
        const int N = m + b, R = N + 1;
        const DevTheta th = a.theta[a.bds[blk]];
        const int d = a.d;
        double* A = slot;
        double* col0 = A + (((int64_t)R * (R + 1)) >> 1);
        double* col1 = col0 + R;
        double* px = col1 + R;

        for (int t = tid; t < N; t += NT) {
            const int g = t < m ? a.nidx[n0 + t] : a.pidx[b0 + (t - m)];
            for (int k = 0; k < d; ++k) px[k * N + t] = a.locs[(int64_t)k * a.n_tot + g] * inv_range_k(th, k);
            A[pk(N, t)] = a.y[g];
        }
        if (tid == 0) {
            A[pk(N, N)] = 0.0;
            s_fail = 0;
        }
        __syncthreads();
        // covariance row by row (one warp per row, lanes along the contiguous columns)
        for (int r = warp; r < N; r += NT / 32) {
            double* row = A + pk(r, 0);
            for (int c = lane; c <= r; c += 32) {
                double acc = 0.0;
                for (int k = 0; k < d; ++k) {
                    const double t = px[k * N + r] - px[k * N + c];
                    acc = fma(t, t, acc);
                }
                double v = GEN ? matern64g(a.gtab + (int64_t)a.bds[blk] * GTAB_SIZE, a.theta + a.bds[blk], th.nu_code,
                                           th.sigma2, sqrt(acc), etab, eK, eL1, eL2)
                               : matern64t(th.nu_code, th.sigma2, sqrt(acc), etab, eK, eL1, eL2);
                if (r == c) v += th.nugget;
                row[c] = v;
            }
        }
        __syncthreads();
        if (warp == 0) {
            const double p = A[0];
            if (bad_pivot(p) && lane == 0) s_fail = 1;
            const double rs = rsqrt(p);
            for (int j = 1 + lane; j <= N; j += 32) {
                const double v = A[pk(j, 0)] * rs;
                A[pk(j, 0)] = v;
                col0[j] = v;
            }
        }
        __syncthreads();
        for (int k = 0; k + 1 < N; ++k) {
            const double* cur = (k & 1) ? col1 : col0;
            double* nxt = (k & 1) ? col0 : col1;
            const int kk = k + 1;
            if (warp == 0) {
                const double ck = cur[kk];
                for (int j = kk + lane; j <= N; j += 32) A[pk(j, kk)] = fma(-cur[j], ck, A[pk(j, kk)]);
                __syncwarp();
                const double p = A[pk(kk, kk)];
                if (bad_pivot(p) && lane == 0) s_fail = 1;
                const double rs = rsqrt(p);
                for (int j = kk + 1 + lane; j <= N; j += 32) {
                    const double v = A[pk(j, kk)] * rs;
                    A[pk(j, kk)] = v;
                    nxt[j] = v;
                }
            }
            // rows kk+1..N: iterate row-wise (contiguous columns) for coalescing
            for (int j = kk + 1 + warp; j <= N; j += NT / 32) {
                const double cj = cur[j];
                double* row = A + pk(j, 0);
                for (int i = kk + 1 + lane; i <= j; i += 32) row[i] = fma(-cj, cur[i], row[i]);
            }
            __syncthreads();
        }
        if (warp == 0) {
            const double2 s2 = warp_terms(m, N, lane, [&](int k) { return A[pk(N, k)]; },
                                          [&](int k) { return log(A[pk(k, k)]); });
            const double s = s2.x, su = s2.y;
            if (lane == 0) {
                double ell = -0.5 * (s + (double)b * kLog2Pi);
                if (s_fail || !(ell == ell)) {
                    ell = -INFINITY;
                    record_fail(a.fail, blk);
                }
                a.ell_blk[blk] = ell;
                a.u_blk[blk] = su;
                s_w = nx;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------
// Deterministic per-dataset sum of the per-block terms (fixed thread->block map, Neumaier
// compensation per thread, fixed-order combination).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

// Deterministic two-stage compensated sums of the per-block ell_i and u_i of every
// dataset (the order depends only on the block order, never on the launch plan).
// Stage 1: CTA (x, ds) sums blocks [lo + x C, lo + (x+1) C) of dataset ds, C = kRedChunk:
// each thread a Neumaier sum over its strided elements, then a fixed binary tree of
// (sum, compensation) pairs.  Stage 2: one thread per dataset adds its chunks in order.
// Spreading stage 1 over many SMs matters on this part, whose FP64 rate per SM is low.
constexpr int kRedChunk = 1024;

__device__ __forceinline__ void pair_add(double& S, double& C, double s, double c) {
    neumaier_add(S, C, s);
    C += c;
}

__global__ void __launch_bounds__(256) k_reduce_part(const double* __restrict__ ell_blk,
                                                     const double* __restrict__ u_blk, const int64_t* ds_off,
                                                     int maxchunks, double4_16a* part) {
    __shared__ double4_16a sh[256];
    const int ds = blockIdx.y, tid = threadIdx.x;
    const int64_t end = ds_off[ds + 1];
    const int64_t lo = ds_off[ds] + (int64_t)blockIdx.x * kRedChunk;
    if (lo >= end) return;
    const int64_t hi = min(end, lo + (int64_t)kRedChunk);
    double s1 = 0.0, c1 = 0.0, s2 = 0.0, c2 = 0.0;
    for (int64_t i = lo + tid; i < hi; i += 256) {
        neumaier_add(s1, c1, ell_blk[i]);
        neumaier_add(s2, c2, u_blk[i]);
    }
    sh[tid].x = s1;
    sh[tid].y = c1;
    sh[tid].z = s2;
    sh[tid].w = c2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) {
            double4_16a a = sh[tid];
            const double4_16a b = sh[tid + w];
            pair_add(a.x, a.y, b.x, b.y);
            pair_add(a.z, a.w, b.z, b.w);
            sh[tid] = a;
        }
        __syncthreads();
    }
    if (tid == 0) part[(int64_t)ds * maxchunks + blockIdx.x] = sh[0];
}

__global__ void k_reduce_final(const double4_16a* __restrict__ part, const int64_t* ds_off, int ndata, int maxchunks,
                               double* out, double* out_quad) {
    const int ds = blockIdx.x * blockDim.x + threadIdx.x;
    if (ds >= ndata) return;
    const int64_t nb = ds_off[ds + 1] - ds_off[ds];
    const int nch = (int)((nb + kRedChunk - 1) / kRedChunk);
    double S1 = 0.0, C1 = 0.0, S2 = 0.0, C2 = 0.0;
    for (int ch = 0; ch < nch; ++ch) {
        const double4_16a p = part[(int64_t)ds * maxchunks + ch];
        pair_add(S1, C1, p.x, p.y);
        pair_add(S2, C2, p.z, p.w);
    }
    const double l = S1 + C1;
    out[ds] = (l == l) ? l : -INFINITY;
    out_quad[ds] = S2 + C2;
}

// ---------------------------------------------------------------------------------
// Mixed precision's error check.  Model: the FP32 error of block i's term is
// delta_i = r_i eps w_i, eps = 2^-24 and w_i the block's error weight (its conditioning
// indicator, the sum over its pivots of variance / conditional variance, times
// 1 + u_i / b_i), with r_i independent, zero mean and of a scale rho that depends on the
// dataset.  Per dataset (one CTA):
//   1. on the fixed sample of blocks (evenly spaced positions in the random block order),
//      recomputed in FP64: rho^2 = mean r_i^2, the mean of r_i and its z-score; the
//      sampled blocks take their FP64 terms;
//   2. the dataset's log-likelihood L is the sum of all its terms (FP32 and sampled FP64;
//      its own error is the quantity bounded, far below |L|);
//   3. the bound on the dataset's error is 3 (2.5 rho) eps sqrt(sum w_i^2) over the blocks
//      still in FP32: 3 standard deviations of their summed noise, with a margin of 2.5 on
//      the sampled rho.  The margin covers the sampling error of rho (64 or more samples
//      of a heavy-tailed r) and a small mean of r that moves with w (a few per cent of
//      rho, from FP32 roundings shared by many blocks): it cancels over a whole dataset,
//      so the z-test below does not see it, but not over the well-conditioned blocks that
//      step 4 keeps in FP32 (measured: up to 1.7 times the 1.5-margin bound without it);
//   4. if a bias shows (|z| > 4) every block is recomputed in FP64 (flag 2); else if the
//      bound exceeds tol |L|, the blocks with the largest w_i are recomputed in FP64 until
//      it does not: the largest threshold w* (bisection on log2 w*, 16 steps) with the bound
//      over {w_i <= w*} within tol |L| (flag 1, thr = w*).
// Fixed-order sums throughout: the decision is deterministic.  Blocks that the FP32-failure
// fallback already recomputed carry w_i = 0 and count as exact.
// ---------------------------------------------------------------------------------
constexpr int kChkThreads = 256;
constexpr float kEps32 = 5.9604644775390625e-8f;  // 2^-24

// Whether local block j of a dataset with B blocks is one of its s sampled blocks
// (positions floor(q B / s), q = 0 .. s-1).
__device__ __forceinline__ bool is_sampled(int64_t j, int64_t B, int64_t s) {
    if (s >= B) return true;
    const int64_t q = (j * s + B - 1) / B;  // smallest q with q B / s >= j
    return q < s && (q * B) / s == j;
}

__device__ __forceinline__ double cta_sum(double v, double* sh, int tid) {
    sh[tid] = v;
    __syncthreads();
    for (int w = kChkThreads / 2; w > 0; w >>= 1) {
        if (tid < w) sh[tid] += sh[tid + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// The bound on the error of the dataset's FP32 blocks with w_i <= thr, in units of eps:
// 3 rho' sqrt(sum w_i^2), three standard deviations of their summed noise.
__device__ __forceinline__ double kept_bound(const float* ind, int64_t lo, int64_t B, int64_t s, float thr,
                                             double rho, double* sh, int tid) {
    double a2 = 0.0;
    for (int64_t j = tid; j < B; j += kChkThreads) {
        const float b = ind[lo + j];
        if (b > 0.0f && b <= thr && !is_sampled(j, B, s)) a2 += (double)b * (double)b;
    }
    a2 = cta_sum(a2, sh, tid);
    return 3.0 * rho * sqrt(a2);
}

__global__ void __launch_bounds__(kChkThreads) k_mixed_check(double* ell_blk, double* u_blk, const double* ell64,
                                                             const double* u64, const float* ind,
                                                             const int32_t* samp, const int64_t* samp_ptr,
                                                             const int64_t* ds_off, double tol, int32_t* flag,
                                                             float* thr, double* est) {
    __shared__ double sh[kChkThreads];
    const int ds = blockIdx.x, tid = threadIdx.x;
    const int64_t s0 = samp_ptr[ds], s1 = samp_ptr[ds + 1], lo = ds_off[ds];
    const int64_t B = ds_off[ds + 1] - lo, s = s1 - s0;
    double r1 = 0.0, r2 = 0.0, cnt = 0.0, bad = 0.0;
    for (int64_t j = s0 + tid; j < s1; j += kChkThreads) {
        const int blk = samp[j];
        const double x64 = ell64[blk], x32 = ell_blk[blk];
        const float b = ind[blk];
        if (!(x64 > -INFINITY) || !(x64 < INFINITY)) bad += 1.0;
        if (b > 0.0f && b < INFINITY) {
            const double r = (x32 - x64) / ((double)kEps32 * (double)b);
            r1 += r;
            r2 += r * r;
            cnt += 1.0;
        }
        ell_blk[blk] = x64;
        u_blk[blk] = u64[blk];
    }
    r1 = cta_sum(r1, sh, tid);
    r2 = cta_sum(r2, sh, tid);
    cnt = cta_sum(cnt, sh, tid);
    bad = cta_sum(bad, sh, tid);
    double e = 0.0;  // the dataset's ell (after the sampled blocks took their FP64 terms)
    for (int64_t j = tid; j < B; j += kChkThreads) e += ell_blk[lo + j];
    e = cta_sum(e, sh, tid);
    int f = 0;
    float t = INFINITY;
    double bound = 0.0;
    if (bad > 0.0) {
        bound = INFINITY;  // a block fails in FP64 too: the dataset's ell is -inf either way
    } else if (s < B && cnt < 2.0) {
        f = 2;  // too few FP32 blocks in the sample to calibrate rho: all to FP64
        bound = INFINITY;
    } else if (s < B) {
        const double rho = 2.5 * sqrt(r2 / cnt), mu = r1 / cnt;  // margin on the sampled scale (step 3)
        const double sd_mu = sqrt(fmax(r2 / cnt - mu * mu, 0.0) / cnt);
        const double L = fabs(e);
        const double k = (double)kEps32 / L;  // bound = k kept_bound
        if (!(fabs(mu) <= 4.0 * sd_mu + 1e-300) || !(L > 0.0)) {
            f = 2;
            bound = INFINITY;
        } else {
            bound = k * kept_bound(ind, lo, B, s, INFINITY, rho, sh, tid);
            if (!(bound <= tol)) {
                // largest log2 threshold in [0, 48] whose kept blocks meet the bound
                float a = 0.0f, c = 48.0f;
                for (int it = 0; it < 16; ++it) {
                    const float mid = 0.5f * (a + c);
                    if (k * kept_bound(ind, lo, B, s, exp2f(mid), rho, sh, tid) <= tol) a = mid;
                    else c = mid;
                }
                f = 1;
                t = exp2f(a);
                bound = k * kept_bound(ind, lo, B, s, t, rho, sh, tid);
            }
        }
    }
    if (tid == 0) {
        flag[ds] = f;
        thr[ds] = t;
        est[ds] = bound;
    }
}

// Queue on the FP64 redo list of its bin every block the check sends back: all blocks of a
// dataset with flag 2, those with B_i above the dataset's threshold with flag 1.
__global__ void k_mixed_redo_list(const int32_t* __restrict__ bds, int64_t nblk, const int32_t* __restrict__ flag,
                                  const float* __restrict__ thr, const float* __restrict__ ind,
                                  const int64_t* __restrict__ samp_ptr, const int64_t* __restrict__ ds_off,
                                  const int32_t* __restrict__ blk_bin, const int64_t* __restrict__ roff,
                                  int32_t* __restrict__ redo, int* cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nblk) return;
    const int ds = bds[i];
    const int f = flag[ds];
    if (f == 0 || (f == 1 && !(ind[i] > thr[ds]))) return;
    const int64_t lo = ds_off[ds];
    if (is_sampled(i - lo, ds_off[ds + 1] - lo, samp_ptr[ds + 1] - samp_ptr[ds])) return;  // FP64 already
    const int b = blk_bin[i];
    const int pos = atomicAdd(cnt + b, 1);
    redo[roff[b] + pos] = (int32_t)i;
}

__global__ void k_fail_reset(unsigned long long* f) { *f = ~0ull; }

__global__ void k_eval_reset(unsigned long long* f, int* ctr, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) ctr[i] = 0;
    if (threadIdx.x == 0) *f = ~0ull;
}

__global__ void k_exp_check(const double* x, double* out, int64_t n, ExpConsts ex) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = exp_neg(x[i], ex.tab, ex.k, ex.l1, ex.l2);
}

// One CTA per dataset: L(x) = x + log rho(x) at the Chebyshev nodes of every octave, then
// the coefficients c_k = (2 / D) sum_j L_j cos(pi k (j + 1/2) / D), c_0 halved.
__global__ void __launch_bounds__(1024) k_gtab_build(const DevTheta* theta, double* gtab) {
    __shared__ double node[GTAB_SIZE];
    const DevTheta* g = theta + blockIdx.x;
    if (g->nu_code != NU_GENERAL) return;
    double* out = gtab + (int64_t)blockIdx.x * GTAB_SIZE;
    for (int f = threadIdx.x; f < GTAB_SIZE; f += blockDim.x) {
        const int o = f / GTAB_DEG, j = f % GTAB_DEG;
        const double a = ldexp(1.0, o + GTAB_E0);
        const double x = a * (1.5 + 0.5 * cospi((j + 0.5) / GTAB_DEG));
        node[f] = x + matern_gen_logcorr(*g, x);
    }
    __syncthreads();
    for (int f = threadIdx.x; f < GTAB_SIZE; f += blockDim.x) {
        const int o = f / GTAB_DEG, k = f % GTAB_DEG;
        double s = 0.0;
        for (int j = 0; j < GTAB_DEG; ++j) s = fma(node[o * GTAB_DEG + j], cospi(k * (j + 0.5) / GTAB_DEG), s);
        s *= 2.0 / GTAB_DEG;
        out[f] = k == 0 ? 0.5 * s : s;
    }
}

__global__ void k_matern_check(const double* x, double* out, int64_t n, const DevTheta* th, const double* gtab,
                               int tabulated, ExpConsts ex) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (th->nu_code == NU_GENERAL && !tabulated) out[i] = matern_gen_corr(*th, x[i]);
    else out[i] = matern64g(gtab, th, th->nu_code, 1.0, x[i], ex.tab, ex.k, ex.l1, ex.l2);
}

// Dynamic shared-memory cap of the shared-memory kernels.  Every size bin launches the
// same instantiation with its own footprint, so the per-function maximum is set once to
// this cap and never lowered (a launch captured in a graph with a larger footprint must
// stay valid when a smaller bin is launched later).
constexpr int kSmemCap = 227 * 1024 - 3072;

// NT = 1024 (one panel warp and 31 update warps) exists for the FP64 CTA kernels only:
// their large blocks run one CTA per SM, where more update warps hide more latency.
template <int NT, bool GEN>
cudaError_t set_smem_cap_g() {
    cudaError_t e = cudaFuncSetAttribute(k_ll_fp64<NT, GEN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ll_fp64<NT, GEN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
    if constexpr (NT == 1024) return e;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ll_mixed<NT, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ll_mixed_w<NT, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ll_fp64_w<NT, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
    return e;
}

template <int NT>
cudaError_t set_smem_cap() {
    cudaError_t e = set_smem_cap_g<NT, false>();
    return e == cudaSuccess ? set_smem_cap_g<NT, true>() : e;
}

// GEN: the instantiation that also evaluates K_nu for a general smoothness (chosen when
// any dataset's nu is not 1/2, 3/2 or 5/2); the others carry no call in their inner loops.
template <int NT, bool GEN>
cudaError_t launch_kind_g(int kind, int grid, size_t smem, const LLArgs& a, cudaStream_t s) {
    if (kind == 0) k_ll_fp64<NT, GEN, false><<<grid, NT, smem, s>>>(a);
    else if (kind == 6) k_ll_fp64<NT, GEN, true><<<grid, NT, smem, s>>>(a);
    else if constexpr (NT == 1024) return cudaErrorInvalidValue;
    else if (kind == 1) k_ll_mixed<NT, GEN><<<grid, NT, smem, s>>>(a);
    else if (kind == 3) k_ll_mixed_w<NT, GEN><<<grid, NT, smem, s>>>(a, (int)(smem / sizeof(float) / (NT / 32)));
    else if (kind == 4) k_ll_fp64_w<NT, GEN><<<grid, NT, smem, s>>>(a, (int)(smem / sizeof(double) / (NT / 32)));
    else k_ll_large<NT, GEN><<<grid, NT, 0, s>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_kind(int kind, int grid, size_t smem, const LLArgs& a, cudaStream_t s) {
    if (kind != 2) {  // per device and function; idempotent and cheap
        cudaError_t e = set_smem_cap<NT>();
        if (e != cudaSuccess) return e;
    }
    return a.gen ? launch_kind_g<NT, true>(kind, grid, smem, a, s) : launch_kind_g<NT, false>(kind, grid, smem, a, s);
}

}  // namespace

// Shared-memory footprint of one CTA for augmented size N.
size_t bv_smem_bytes(int kind, int nmax, int d, int threads) {
    (void)threads;
    const size_t R = (size_t)nmax + 1;
    const size_t el = kind == 1 ? sizeof(float) : sizeof(double);
    if (kind == 2) return 0;
    if (kind == 5) return bv_tc_smem_bytes(nmax);
    if (kind == 1) return sizeof(float) * (size_t)mixed_floats(nmax);
    if (kind == 3) return sizeof(float) * (size_t)mixed_floats(nmax) * (size_t)(threads / 32);
    if (kind == 4) {  // one region per warp, each a multiple of 16 bytes
        const size_t region = (R * (R + 1) / 2 + R + (size_t)d * nmax + 1) & ~(size_t)1;
        return sizeof(double) * region * (size_t)(threads / 32);
    }
    size_t bytes = el * (R * (R + 1) / 2 + (kind == 6 ? 4 : 2) * R + (size_t)d * nmax);
    return (bytes + 15) & ~(size_t)15;
}

// Largest N the shared-memory kernels take (227 KB opt-in per CTA, minus static smem).
int bv_smem_max_n(int kind, int d) {
    const size_t cap = kSmemCap;
    int n = 8;
    while (bv_smem_bytes(kind, n + 1, d, 0) <= cap) ++n;
    return n;
}

int bv_max_threads_for(int kind) { return kind == 2 ? 256 : 544; }

cudaError_t bv_launch_bin(const BinPlan& bp, const LLArgs& a0, cudaStream_t s) {
    if (bp.nwork == 0) return cudaSuccess;
    LLArgs a = a0;
    a.work = bp.d_work;
    a.nwork = bp.nwork;
    a.ctr = bp.d_ctr;
    if (bp.kind == 5) return bv_tc_launch(bp.threads, bp.grid, bp.smem, a, s);
    switch (bp.threads) {
        case 64: return launch_kind<64>(bp.kind, bp.grid, bp.smem, a, s);
        case 128: return launch_kind<128>(bp.kind, bp.grid, bp.smem, a, s);
        case 96: return launch_kind<96>(bp.kind, bp.grid, bp.smem, a, s);
        case 160: return launch_kind<160>(bp.kind, bp.grid, bp.smem, a, s);
        case 288: return launch_kind<288>(bp.kind, bp.grid, bp.smem, a, s);
        case 544: return launch_kind<544>(bp.kind, bp.grid, bp.smem, a, s);
        case 256: return launch_kind<256>(bp.kind, bp.grid, bp.smem, a, s);
        case 1024: return launch_kind<1024>(bp.kind, bp.grid, bp.smem, a, s);
        default: return cudaErrorInvalidValue;
    }
}

int bv_reduce_chunks(int64_t max_blocks_per_dataset) {
    return (int)std::max<int64_t>(1, (max_blocks_per_dataset + kRedChunk - 1) / kRedChunk);
}

cudaError_t bv_launch_reduce(const double* ell_blk, const double* u_blk, const int64_t* ds_blk_off,
                             int32_t ndata, int32_t maxchunks, void* part, double* out, double* out_quad,
                             cudaStream_t s) {
    k_reduce_part<<<dim3(maxchunks, ndata), 256, 0, s>>>(ell_blk, u_blk, ds_blk_off, maxchunks,
                                                         static_cast<double4_16a*>(part));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<(ndata + 127) / 128, 128, 0, s>>>(static_cast<const double4_16a*>(part), ds_blk_off, ndata,
                                                       maxchunks, out, out_quad);
    return cudaGetLastError();
}

cudaError_t bv_launch_gtab(const DevTheta* theta, int32_t ndata, double* gtab, cudaStream_t s) {
    k_gtab_build<<<ndata, 1024, 0, s>>>(theta, gtab);
    return cudaGetLastError();
}

cudaError_t bv_launch_fallback(const LLArgs& a0, int grid, cudaStream_t s) {
    LLArgs a = a0;
    a.dyn = 1;
    a.fb = a0.fb;
    a.ctr = nullptr;
    return a.gen ? launch_kind_g<256, true>(2, grid, 0, a, s) : launch_kind_g<256, false>(2, grid, 0, a, s);
}

cudaError_t bv_launch_mixed_check(double* ell_blk, double* u_blk, const double* ell64, const double* u64,
                                  const float* ind, const int32_t* samp, const int64_t* samp_ptr,
                                  const int64_t* ds_blk_off, int32_t ndata, double tol, int32_t* flag, float* thr,
                                  double* est, cudaStream_t s) {
    k_mixed_check<<<ndata, kChkThreads, 0, s>>>(ell_blk, u_blk, ell64, u64, ind, samp, samp_ptr, ds_blk_off, tol,
                                               flag, thr, est);
    return cudaGetLastError();
}

cudaError_t bv_launch_mixed_redo_list(const int32_t* bds, int64_t nblk, const int32_t* flag, const float* thr,
                                      const float* ind, const int64_t* samp_ptr, const int64_t* ds_blk_off,
                                      const int32_t* blk_bin, const int64_t* roff, int32_t* redo, int* cnt,
                                      cudaStream_t s) {
    k_mixed_redo_list<<<(unsigned)((nblk + 255) / 256), 256, 0, s>>>(bds, nblk, flag, thr, ind, samp_ptr, ds_blk_off,
                                                                     blk_bin, roff, redo, cnt);
    return cudaGetLastError();
}

cudaError_t bv_launch_fail_reset(unsigned long long* fail, cudaStream_t s) {
    k_fail_reset<<<1, 1, 0, s>>>(fail);
    return cudaGetLastError();
}

cudaError_t bv_launch_eval_reset(unsigned long long* fail, int* ctr, int n, cudaStream_t s) {
    k_eval_reset<<<1, 64, 0, s>>>(fail, ctr, n);
    return cudaGetLastError();
}

// Occupancy helper for the planner.
int bv_occupancy(int kind, int threads, size_t smem) {
    if (kind == 5) return bv_tc_occupancy(threads, smem);
    int nb = 0;
    cudaError_t e = cudaSuccess;
#define BV_OCC(NT)                                                                            \
    if (threads == NT) {                                                                      \
        if (kind != 2) e = set_smem_cap<NT>();                                                \
        if (e == cudaSuccess) {                                                               \
            if (kind == 0)                                                                    \
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ll_fp64<NT, false, false>, NT, smem); \
            else if (kind == 6)                                                               \
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ll_fp64<NT, false, true>, NT, smem); \
            else if (kind == 1)                                                               \
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ll_mixed<NT, false>, NT, smem); \
            else if (kind == 3)                                                               \
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ll_mixed_w<NT, false>, NT, smem); \
            else if (kind == 4)                                                               \
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ll_fp64_w<NT, false>, NT, smem); \
            else                                                                              \
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ll_large<NT, false>, NT, 0);    \
        }                                                                                     \
    }
    BV_OCC(64) BV_OCC(128) BV_OCC(96) BV_OCC(160) BV_OCC(288) BV_OCC(544) BV_OCC(256)
#undef BV_OCC
    if (threads == 1024 && (kind == 0 || kind == 6)) {
        e = set_smem_cap<1024>();
        if (e == cudaSuccess)
            e = kind == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ll_fp64<1024, false, false>, 1024, smem)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ll_fp64<1024, false, true>, 1024, smem);
    }
    if (e != cudaSuccess) return 0;
    return nb;
}

static void fill_exp_consts(ExpConsts* o) {
    const long double ln2 = 0.693147180559945309417232121458176568L;
    for (int j = 0; j < BV_EXP_TAB; ++j) o->tab[j] = (double)exp2l((long double)j / (long double)BV_EXP_TAB);
    const long double L = ln2 / (long double)BV_EXP_TAB;
    double l1 = (double)L;
    unsigned long long bits;
    memcpy(&bits, &l1, sizeof(bits));
    bits &= ~((1ull << 21) - 1ull);
    memcpy(&l1, &bits, sizeof(bits));
    o->l1 = l1;
    o->l2 = (double)(L - (long double)l1);
    o->k = (double)((long double)BV_EXP_TAB / ln2);
    for (int j = 0; j < 32; ++j) {
        const long double t = exp2l(-(long double)j / 32.0L);
        o->t32[j] = (float)t;
        o->t32[32 + j] = (float)(t - (long double)o->t32[j]);
    }
    const long double L32 = ln2 / 32.0L;
    float f1 = (float)L32;
    unsigned int fb;
    memcpy(&fb, &f1, sizeof(fb));
    fb &= ~((1u << 12) - 1u);
    memcpy(&f1, &fb, sizeof(fb));
    o->l1_32 = f1;
    o->l2_32 = (float)(L32 - (long double)f1);
    o->k32 = (float)(32.0L / ln2);
}

// The table is computed once per process (long double is a software type on some hosts,
// which makes 256 exp2l calls cost a fraction of a millisecond).
void bv_exp_consts(ExpConsts* o) {
    static const ExpConsts cached = [] {
        ExpConsts e;
        fill_exp_consts(&e);
        return e;
    }();
    *o = cached;
}

__global__ void k_exp32_check(const float* x, float* own, float* lib, int64_t n, ExpConsts ex) {
    __shared__ float t[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) t[i] = ex.t32[i];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        own[i] = exp_neg32(x[i], t, ex.k32, ex.l1_32, ex.l2_32);
        lib[i] = expf(-x[i]);
    }
}

// Diagnostic: the mixed kernels' FP32 exp(-x) (own) and CUDA's expf(-x) (lib) on the
// device for host inputs x[n] >= 0.
extern "C" int bv_exp_neg32_check(int64_t n, const float* x, float* own, float* lib) {
    if (n <= 0 || !x || !own || !lib) return BV_EINVAL;
    ExpConsts ex;
    bv_exp_consts(&ex);
    float *dx = nullptr, *d1 = nullptr, *d2 = nullptr;
    BV_CUDA(cudaMalloc(&dx, sizeof(float) * n));
    BV_CUDA(cudaMalloc(&d1, sizeof(float) * n));
    BV_CUDA(cudaMalloc(&d2, sizeof(float) * n));
    BV_CUDA(cudaMemcpy(dx, x, sizeof(float) * n, cudaMemcpyHostToDevice));
    k_exp32_check<<<(unsigned)((n + 255) / 256), 256>>>(dx, d1, d2, n, ex);
    BV_CUDA(cudaGetLastError());
    BV_CUDA(cudaMemcpy(own, d1, sizeof(float) * n, cudaMemcpyDeviceToHost));
    BV_CUDA(cudaMemcpy(lib, d2, sizeof(float) * n, cudaMemcpyDeviceToHost));
    cudaFree(dx);
    cudaFree(d1);
    cudaFree(d2);
    return BV_OK;
}

// Diagnostic: the library's FP64 exp(-x) on the device for host inputs x[n].
extern "C" int bv_exp_neg_check(int64_t n, const double* x, double* out) {
    if (n <= 0 || !x || !out) return BV_EINVAL;
    ExpConsts ex;
    bv_exp_consts(&ex);
    double *dx = nullptr, *dy = nullptr;
    BV_CUDA(cudaMalloc(&dx, sizeof(double) * n));
    BV_CUDA(cudaMalloc(&dy, sizeof(double) * n));
    BV_CUDA(cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice));
    k_exp_check<<<(unsigned)((n + 255) / 256), 256>>>(dx, dy, n, ex);
    BV_CUDA(cudaGetLastError());
    BV_CUDA(cudaMemcpy(out, dy, sizeof(double) * n, cudaMemcpyDeviceToHost));
    cudaFree(dx);
    cudaFree(dy);
    return BV_OK;
}

extern "C" int bv_matern_check(double nu, int32_t tabulated, int64_t n, const double* x, double* out) {
    if (n <= 0 || !x || !out) return BV_EINVAL;
    bv_theta t{};
    t.sigma2 = 1.0;
    t.range[0] = 1.0;
    t.nu = nu;
    DevTheta th;
    BV_TRY(bv_theta_to_dev(&t, 1, &th));
    ExpConsts ex;
    bv_exp_consts(&ex);
    double *dx = nullptr, *dy = nullptr, *dtab = nullptr;
    DevTheta* dth = nullptr;
    BV_CUDA(cudaMalloc(&dx, sizeof(double) * n));
    BV_CUDA(cudaMalloc(&dy, sizeof(double) * n));
    BV_CUDA(cudaMalloc(&dth, sizeof(DevTheta)));
    BV_CUDA(cudaMalloc(&dtab, sizeof(double) * GTAB_SIZE));
    BV_CUDA(cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice));
    BV_CUDA(cudaMemcpy(dth, &th, sizeof(DevTheta), cudaMemcpyHostToDevice));
    k_gtab_build<<<1, 1024>>>(dth, dtab);
    BV_CUDA(cudaGetLastError());
    k_matern_check<<<(unsigned)((n + 255) / 256), 256>>>(dx, dy, n, dth, dtab, tabulated, ex);
    BV_CUDA(cudaGetLastError());
    BV_CUDA(cudaMemcpy(out, dy, sizeof(double) * n, cudaMemcpyDeviceToHost));
    cudaFree(dx);
    cudaFree(dy);
    cudaFree(dth);
    cudaFree(dtab);
    return BV_OK;
}
