// bv_mixed_tc.cu -- mixed-precision block kernel with the Schur-complement updates of the
// augmented Cholesky factorisation on the tensor cores (large blocks).
//
// The per-block computation is the same as the FP32 SIMT kernel's (bv_loglik.cu): one
// Cholesky factorisation of the augmented (N+1) x (N+1) matrix
//     [[Sigma^con, Sigma^cross, y_NN], [., Sigma^lk, y_B], [., ., *]]
// whose trailing pivots and last row give Algorithm 1's log-determinant and quadratic form
// of the block (Eq. 4).  Here the factorisation is blocked by 16 columns:
//   diagonal tile   one warp factors the 16 x 16 diagonal tile in FP32, one row per lane
//                   (the tile's rows below its pivot columns, e.g. the observation row,
//                   are solved in the same pass);
//   panel (TRSM)    every thread solves one row of the tile column below against it
//                   (V = L^{-1} Sigma^cross and y' for the conditioning columns);
//   update (SYRK)   each warp updates 16 x 16 tiles of the trailing triangle,
//                   A_IJ -= P_I P_J^T, with mma.sync m16n8k16 on BF16 operands: every FP32
//                   operand is split exactly into three BF16 parts x = x0 + x1 + x2 and the
//                   six products x_i y_j with i + j <= 2 are accumulated in FP32, smallest
//                   first, so the product keeps FP32 accuracy (the dropped terms are below
//                   2^-24 of it).
// Look-ahead: while the other warps apply panel p to the trailing triangle, warp 0 factors
// the diagonal tile of panel p+1 (its column was updated first), so the pivot chain
// overlaps the tensor-core work.  Pivots, log-determinant and quadratic form are
// accumulated in FP64 as in the SIMT kernel, and a non-positive pivot sends the block to
// the FP64 fallback pass.
//
// Storage: the lower triangle of 16 x 16 FP32 tiles, tile (I, J) at I(I+1)/2 + J, each
// row-major with the column's 4-float group permuted by bits 1 and 2 of the row (see
// toff), which keeps the fragment loads of the MMAs (8-byte, half-warp) and the panel
// solve's row loads (16-byte, quarter-warp) free of bank conflicts.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bv_device.cuh"
#include "bv_internal.h"
#include "bv_ll_block.cuh"

namespace {

constexpr int kE = 16;         // tile edge
constexpr int kTF = kE * kE;   // floats per tile

__device__ __forceinline__ int tc_tile(int I, int J) { return ((I * (I + 1)) >> 1) + J; }
// Offset of element (r, c) inside a tile.
__device__ __forceinline__ int toff(int r, int c) {
    return (r << 4) + (c ^ ((((r >> 1) & 1) << 3) | (((r >> 2) & 1) << 2)));
}

// Floats of shared memory for one block of augmented size N (R = N + 1 rows):
// tiles | Lp (16 x 16, the current diagonal factor, plain row-major) | rs (16) |
// px, py, pz (N each) | yv (N) | piv (N)
__host__ __device__ __forceinline__ int tc_floats(int nmax) {
    const int T = (nmax + 1 + kE - 1) / kE;
    return ((T * (T + 1)) >> 1) * kTF + kTF + kE + 5 * nmax + 4;
}

// x = x0 + x1 + x2 exactly, each part a BF16 (8 significant bits; 24 in all).
__device__ __forceinline__ void split3(float x, float& x0, float& x1, float& x2) {
    x0 = __bfloat162float(__float2bfloat16_rn(x));
    const float r1 = x - x0;  // exact
    x1 = __bfloat162float(__float2bfloat16_rn(r1));
    x2 = r1 - x1;             // exact, at most 8 significant bits
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
    return *reinterpret_cast<uint32_t*>(&v);
}

// D += A B with A 16x16 (row), B 16x8 (col), BF16 operands, FP32 accumulation.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The A operand of C -= X_I X_J^T, split once for every tile of row I a warp updates: the
// rows g, g+8 and columns 2t, 2t+1, 2t+8, 2t+9 of X_I, negated (so that the MMAs
// subtract) and split into three BF16 parts, packed in pairs.
struct AFrag {
    uint32_t q[3][4];
};

__device__ __forceinline__ void load_a(const float* XI, int lane, AFrag& A) {
    const int g = lane >> 2, t = lane & 3;
    float v[8];
    const float2 p0 = *reinterpret_cast<const float2*>(XI + toff(g, 2 * t));
    const float2 p1 = *reinterpret_cast<const float2*>(XI + toff(g + 8, 2 * t));
    const float2 p2 = *reinterpret_cast<const float2*>(XI + toff(g, 2 * t + 8));
    const float2 p3 = *reinterpret_cast<const float2*>(XI + toff(g + 8, 2 * t + 8));
    v[0] = -p0.x; v[1] = -p0.y; v[2] = -p1.x; v[3] = -p1.y;
    v[4] = -p2.x; v[5] = -p2.y; v[6] = -p3.x; v[7] = -p3.y;
    float s[3][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) split3(v[e], s[0][e], s[1][e], s[2][e]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        A.q[q][0] = pack_bf16(s[q][0], s[q][1]);
        A.q[q][1] = pack_bf16(s[q][2], s[q][3]);
        A.q[q][2] = pack_bf16(s[q][4], s[q][5]);
        A.q[q][3] = pack_bf16(s[q][6], s[q][7]);
    }
}

// C -= X_I X_J^T for one 16 x 16 tile C (tile pointers into the tile array), by one warp,
// with X_I's fragments in A.  B fragments: rows h*8 + g of X_J, columns 2t, 2t+1 and
// 2t+8, 2t+9, split the same way.
__device__ __forceinline__ void tile_update_a(float* C, const AFrag& A, const float* XJ, int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t B[3][2];
        {
            const int rj = h * 8 + g;
            const float2 q0 = *reinterpret_cast<const float2*>(XJ + toff(rj, 2 * t));
            const float2 q1 = *reinterpret_cast<const float2*>(XJ + toff(rj, 2 * t + 8));
            float s[3][4];
            split3(q0.x, s[0][0], s[1][0], s[2][0]);
            split3(q0.y, s[0][1], s[1][1], s[2][1]);
            split3(q1.x, s[0][2], s[1][2], s[2][2]);
            split3(q1.y, s[0][3], s[1][3], s[2][3]);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                B[q][0] = pack_bf16(s[q][0], s[q][1]);
                B[q][1] = pack_bf16(s[q][2], s[q][3]);
            }
        }
        float2* c01 = reinterpret_cast<float2*>(C + toff(g, h * 8 + 2 * t));
        float2* c23 = reinterpret_cast<float2*>(C + toff(g + 8, h * 8 + 2 * t));
        // the product is accumulated from zero, smallest terms first, and added to C in
        // FP32 afterwards: the tensor core's accumulation does not round C to nearest, so C
        // itself never enters it
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        mma_bf16(d, A.q[2], B[0][0], B[0][1]);
        mma_bf16(d, A.q[1], B[1][0], B[1][1]);
        mma_bf16(d, A.q[0], B[2][0], B[2][1]);
        mma_bf16(d, A.q[1], B[0][0], B[0][1]);
        mma_bf16(d, A.q[0], B[1][0], B[1][1]);
        mma_bf16(d, A.q[0], B[0][0], B[0][1]);
        const float2 u = *c01, w = *c23;
        *c01 = make_float2(u.x + d[0], u.y + d[1]);
        *c23 = make_float2(w.x + d[2], w.y + d[3]);
    }
}

__device__ __forceinline__ void tile_update(float* C, const float* XI, const float* XJ, int lane) {
    AFrag A;
    load_a(XI, lane, A);
    tile_update_a(C, A, XJ, lane);
}

// Factor the diagonal tile of panel p (warp 0, FP32, lane r < 16 holds row r): pivot
// columns c < nc; every row of the tile below a pivot column is scaled and updated, so
// rows past the last pivot column (the observation row, padding) come out solved.
// Writes the factor back to the tile and to Lp (plain row-major), 1/sqrt(pivot) to rs,
// the pivots to piv and raises *fail on a non-positive pivot.  Every pivot gets dlo, the
// part of the matrix diagonal its FP32 value misses.
__device__ __forceinline__ void diag_factor(float* tile, float* Lp, float* rs, float* piv, int k0, int nc, int lane,
                                            int* fail, float dlo) {
    const int r = lane & 15;
    float a[kE];
#pragma unroll
    for (int c = 0; c < kE; ++c) a[c] = tile[toff(r, c)];
    // Column c's update uses the unscaled column: a_ri -= (a_rc / p_c) a_ic, so the
    // broadcasts of a_ic do not wait for the pivot's reciprocal square root; the column is
    // scaled by 1/sqrt(p_c) afterwards, off the chain from one pivot to the next.
#pragma unroll
    for (int c = 0; c < kE; ++c) {
        if (c < nc) {  // warp-uniform
            float col[kE];
#pragma unroll
            for (int i = c + 1; i < kE; ++i) col[i] = __shfl_sync(0xffffffffu, a[c], i);
            const float pc = __shfl_sync(0xffffffffu, a[c], c) + dlo;
            const float t = a[c] * __frcp_rn(pc);
#pragma unroll
            for (int i = c + 1; i < kE; ++i)
                if (r >= i) a[i] = fmaf(-t, col[i], a[i]);
            const float rc = __frsqrt_rn(pc);  // correctly rounded: no one-sided bias
            if (lane == c) {
                piv[k0 + c] = pc;
                rs[c] = rc;
                if (!(pc > 0.0f) || !(pc < INFINITY)) *fail = 1;
            }
            if (r > c) a[c] *= rc;
        }
    }
    if (lane < kE) {
#pragma unroll
        for (int c = 0; c < kE; ++c) {
            tile[toff(r, c)] = a[c];
            Lp[r * kE + c] = a[c];
        }
    }
}

// Solve one row of the tile column below a factored diagonal tile: x_c = (a_c - sum_{j<c}
// x_j L_cj) / L_cc for the pivot columns c < nc (right-looking inside the row, so the
// inner updates are independent).
__device__ __forceinline__ void panel_row(float* row_tile, int r, const float* Lp, const float* rs, int nc) {
    float x[kE];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 v = *reinterpret_cast<const float4*>(row_tile + toff(r, 4 * q));
        x[4 * q] = v.x;
        x[4 * q + 1] = v.y;
        x[4 * q + 2] = v.z;
        x[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int j = 0; j < kE; ++j) {
        if (j < nc) {
            x[j] *= rs[j];
#pragma unroll
            for (int c = j + 1; c < kE; ++c) x[c] = fmaf(-x[j], Lp[c * kE + j], x[c]);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(row_tile + toff(r, 4 * q)) =
            make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
}

template <int NT, bool GEN>
__global__ void __launch_bounds__(NT) k_ll_mixed_tc(LLArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float* sm = reinterpret_cast<float*>(smraw);
    __shared__ int s_fail;
    __shared__ int s_w;
    __shared__ float t32[64];
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 64; i += NT) t32[i] = a.ex.t32[i];
    const int nwork = work_count(a);
    if (tid == 0) s_w = take_work(a.ctr, blockIdx.x);
    __syncthreads();
    for (int w = s_w; w < nwork; w = s_w) {
        const int nx = tid == 0 ? take_work(a.ctr, w + gridDim.x) : 0;
        const int blk = a.work[w];
        const int64_t b0 = a.bptr[blk], n0 = a.nptr[blk];
        const int b = (int)(a.bptr[blk + 1] - b0), m = (int)(a.nptr[blk + 1] - n0);
        const int N = m + b, R = N + 1, T = (R + kE - 1) / kE;
        const DevTheta th = a.theta[a.bds[blk]];
        float* tiles = sm;
        float* Lp = tiles + ((T * (T + 1)) >> 1) * kTF;
        float* rs = Lp + kTF;
        float* px = rs + kE;
        float* py = px + N;
        float* pz = py + N;
        float* yv = pz + N;
        float* piv = yv + N;
        const int d = a.d;
        const float s2 = th.sigma2_f, tau2 = th.nugget_f;
        const float ir0 = th.inv_range_f[0], ir1 = th.inv_range_f[1], ir2 = th.inv_range_f[2];
        if (tid == 0) s_fail = 0;

        // gather: offsets from the block centroid in FP64, rounded to FP32 and scaled
        for (int t = tid; t < N; t += NT) {
            const int gi = t < m ? a.nidx[n0 + t] : a.pidx[b0 + (t - m)];
            const double* cb = a.cent + (int64_t)blk * d;
            px[t] = (float)(a.locs[gi] - cb[0]) * ir0;
            py[t] = d > 1 ? (float)(a.locs[a.n_tot + gi] - cb[1]) * ir1 : 0.0f;
            pz[t] = d > 2 ? (float)(a.locs[2 * a.n_tot + gi] - cb[2]) * ir2 : 0.0f;
            yv[t] = (float)a.y[gi];
        }
        __syncthreads();

        // fill: one tile per warp at a time, two rows per pass (lane -> row 2i + lane/16)
        const int ntile = (T * (T + 1)) >> 1;
        for (int q = warp; q < ntile; q += NW) {
            int I, J;
            tri_rc(q, I, J);
            float* tl = tiles + q * kTF;
            const int c = lane & 15, gc = J * kE + c;
            const float cx = gc < N ? px[gc] : 0.0f, cy = gc < N ? py[gc] : 0.0f, cz = gc < N ? pz[gc] : 0.0f;
#pragma unroll 2
            for (int rr = lane >> 4; rr < kE; rr += 2) {
                const int gr = I * kE + rr;
                float v = 0.0f;
                if (gr < N && gc <= gr) {
                    const float t0 = px[gr] - cx, t1 = py[gr] - cy, t2 = pz[gr] - cz;
                    const float xf = sqrtf(fmaf(t2, t2, fmaf(t1, t1, t0 * t0)));
                    v = (GEN && th.nu_code == NU_GENERAL)
                            ? s2 * matern_gen_tab32(a.gtab + (int64_t)a.bds[blk] * GTAB_SIZE, a.theta + a.bds[blk], xf)
                            : matern32(th.nu_code, s2, xf, t32, a.ex);
                    if (gr == gc) v += tau2;
                } else if (gr == N && gc < N) {
                    v = yv[gc];
                }
                tl[toff(rr, c)] = v;
            }
        }
        __syncthreads();

        // panel 0: diagonal tile, then the tile column below it
        if (warp == 0) diag_factor(tiles, Lp, rs, piv, 0, min(kE, N), lane, &s_fail, th.diag_lo_f);
        __syncthreads();
        for (int r = kE + tid; r < T * kE; r += NT) {
            float* rt = tiles + tc_tile(r >> 4, 0) * kTF;
            panel_row(rt, r & 15, Lp, rs, min(kE, N));
        }
        __syncthreads();

        for (int p = 0; p + 1 < T; ++p) {
            const int p1 = p + 1;
            // column p+1 first (the look-ahead's input): tiles (I, p+1), I >= p+1
            for (int I = p1 + warp; I < T; I += NW)
                tile_update(tiles + tc_tile(I, p1) * kTF, tiles + tc_tile(I, p) * kTF, tiles + tc_tile(p1, p) * kTF,
                            lane);
            __syncthreads();
            // warp 0 factors the next diagonal tile; the other warps update the rest of the
            // trailing triangle, columns p+2.., with panel p
            const int k1 = p1 * kE, nc1 = min(kE, N - k1);
            if (warp == 0) {
                if (nc1 > 0) diag_factor(tiles + tc_tile(p1, p1) * kTF, Lp, rs, piv, k1, nc1, lane, &s_fail, th.diag_lo_f);
            } else {
                // trailing tile rows p+2 .. T-1, each (with all its tiles J = p+2 .. I) owned
                // by one warp, longest rows first, so that X_I is split once per row
                for (int I = T - 1 - (warp - 1); I >= p + 2; I -= NW - 1) {
                    AFrag A;
                    load_a(tiles + tc_tile(I, p) * kTF, lane, A);
                    for (int J = p + 2; J <= I; ++J)
                        tile_update_a(tiles + tc_tile(I, J) * kTF, A, tiles + tc_tile(J, p) * kTF, lane);
                }
            }
            __syncthreads();
            // the tile column below diagonal tile p+1
            if (nc1 > 0)
                for (int r = (p1 + 1) * kE + tid; r < T * kE; r += NT) {
                    float* rt = tiles + tc_tile(r >> 4, p1) * kTF;
                    panel_row(rt, r & 15, Lp, rs, nc1);
                }
            __syncthreads();
        }

        // the observation row's entries (z) and the pivots of the block columns, in FP64
        if (warp == 0) {
            if (a.ind_blk) {
                const float ind = warp_indicator(N, lane, s2 + tau2, [&](int k) { return piv[k]; });
                if (lane == 0) a.ind_blk[blk] = ind;
            }
            const int tN = N >> 4, rN = N & 15;
            const double2 s2v = warp_terms(
                m, N, lane,
                [&](int k) { return (double)tiles[tc_tile(tN, k >> 4) * kTF + toff(rN, k & 15)]; },
                [&](int k) { return log((double)piv[k]); });
            if (lane == 0) {
                finish_block(a, blk, b, s2v.x, s2v.y, s_fail);
                s_w = nx;
            }
        }
        __syncthreads();
    }
}

template <int NT>
cudaError_t set_cap() {
    constexpr int cap = 227 * 1024 - 3072;
    cudaError_t e = cudaFuncSetAttribute(k_ll_mixed_tc<NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ll_mixed_tc<NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    return e;
}

// Diagnostic: one warp applies tile_update to host tiles (plain row-major in, out).
__global__ void k_tc_update_check(const float* C, const float* XI, const float* XJ, float* out) {
    __shared__ __align__(16) float t[3][kTF];
    const int lane = threadIdx.x;
    for (int e = lane; e < kTF; e += 32) {
        const int r = e >> 4, c = e & 15;
        t[0][toff(r, c)] = C[e];
        t[1][toff(r, c)] = XI[e];
        t[2][toff(r, c)] = XJ[e];
    }
    __syncwarp();
    tile_update(t[0], t[1], t[2], lane);
    __syncwarp();
    for (int e = lane; e < kTF; e += 32) out[e] = t[0][toff(e >> 4, e & 15)];
}

}  // namespace

size_t bv_tc_smem_bytes(int nmax) { return sizeof(float) * (size_t)tc_floats(nmax); }

int bv_tc_occupancy(int threads, size_t smem) {
    int nb = 0;
    cudaError_t e = cudaSuccess;
#define BV_TCOCC(NT)                                                                                    \
    if (threads == NT) {                                                                                \
        e = set_cap<NT>();                                                                              \
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ll_mixed_tc<NT, false>, NT, smem); \
    }
    BV_TCOCC(128) BV_TCOCC(256) BV_TCOCC(384) BV_TCOCC(512)
#undef BV_TCOCC
    return e == cudaSuccess ? nb : 0;
}

cudaError_t bv_tc_launch(int threads, int grid, size_t smem, const LLArgs& a, cudaStream_t s) {
#define BV_TCL(NT)                                                                          \
    if (threads == NT) {                                                                    \
        cudaError_t e = set_cap<NT>();                                                      \
        if (e != cudaSuccess) return e;                                                     \
        if (a.gen) k_ll_mixed_tc<NT, true><<<grid, NT, smem, s>>>(a);                       \
        else k_ll_mixed_tc<NT, false><<<grid, NT, smem, s>>>(a);                            \
        return cudaGetLastError();                                                          \
    }
    BV_TCL(128) BV_TCL(256) BV_TCL(384) BV_TCL(512)
#undef BV_TCL
    return cudaErrorInvalidValue;
}

// C ABI diagnostic (include/bv.h).
extern "C" int bv_tc_update_check(const float* C, const float* XI, const float* XJ, float* out) {
    if (!C || !XI || !XJ || !out) return BV_EINVAL;
    float* dbuf = nullptr;
    BV_CUDA(cudaMalloc(&dbuf, sizeof(float) * 4 * kTF));
    cudaError_t e = cudaMemcpy(dbuf, C, sizeof(float) * kTF, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dbuf + kTF, XI, sizeof(float) * kTF, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dbuf + 2 * kTF, XJ, sizeof(float) * kTF, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_tc_update_check<<<1, 32>>>(dbuf, dbuf + kTF, dbuf + 2 * kTF, dbuf + 3 * kTF);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dbuf + 3 * kTF, sizeof(float) * kTF, cudaMemcpyDeviceToHost);
    cudaFree(dbuf);
    BV_CUDA(e);
    return BV_OK;
}
