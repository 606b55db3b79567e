// bv_pred.cu -- block-Vecchia prediction (Sec. 2.4, Algorithm 2) and univariate
// conditional simulation with the prediction interval coverage (Sec. 2.4; PICP, Sec. 3.2).
//
// Algorithm 2 for prediction block i with conditioning set NN_i (the m_i observations
// nearest to the block centroid) and b_i new locations:
//     mu_i    = Sigma^cross_i (Sigma^con_i)^{-1} y_NN,
//     Sigma_i = Sigma^lk_i - Sigma^cross_i (Sigma^con_i)^{-1} Sigma^cross_i^T.
// GPU formulation: both are one partial Cholesky factorisation.  Take the augmented
// (N+1) x (N+1) matrix, N = m_i + b_i,
//     [[ Sigma^con   .          . ],
//      [ Sigma^cross Sigma^lk   . ],
//      [ y_NN^T      0          . ]]
// and eliminate its first m_i columns only.  The trailing (b_i + 1) x (b_i + 1) Schur
// complement is then [[Sigma_i, .], [-mu_i^T, .]]: its b_i x b_i block is the conditional
// covariance and its last row is minus the conditional mean.  One kernel per call,
// the matrix in shared memory (or a global workspace slot for blocks too large for it),
// nothing but mu, diag(Sigma_i) and (optionally) Sigma_i written to HBM.
//
// Conditional simulation (the paper's univariate scheme): draw r of new location j is
// mu_j + sigma_j z_jr with z_jr standard normal by the Box-Muller transform (Box and
// Muller 1958), two normals per pair of SplitMix64 uniforms; the sample mean and sample
// standard deviation (divisor R - 1) of the R draws give the interval mean~ -/+ z_crit sd~,
// and the PICP is the fraction of held-out values inside it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bv_device.cuh"
#include "bv_internal.h"

struct PredState {
    int64_t n_star = 0;
    std::vector<double> h_locs;   // row-major n_star x d
    double* d_locs = nullptr;     // SoA d x n_star
    double* d_ytrue = nullptr;    // held-out values (may stay null)
    int64_t nblk = 0;
    std::vector<int64_t> h_bptr;
    std::vector<int32_t> h_pidx;
    std::vector<double> h_cent;
    int64_t* d_bptr = nullptr;
    int32_t* d_pidx = nullptr;
    double* d_cent = nullptr;
    std::vector<int64_t> h_nptr;
    int64_t* d_nptr = nullptr;
    int32_t* d_nidx = nullptr;
    std::vector<int64_t> h_coff;  // packed Sigma_i offsets, nblk + 1
    int64_t* d_coff = nullptr;
    double* d_mean = nullptr;     // n_star, by new-location index
    double* d_var = nullptr;
    double* d_cov = nullptr;      // h_coff.back()
    double* d_lo = nullptr;       // interval bounds, n_star
    double* d_up = nullptr;
    unsigned long long* d_count = nullptr;
    unsigned long long* d_fail = nullptr;
    double* d_ws = nullptr;
    int64_t ws_stride = 0;
    int ws_slots = 0;
    bool have_blocks = false, have_nn = false, have_pred = false;
    // launch shape of k_pred per instantiation (closed-form / general nu), set on first use
    int64_t launch_grid[2] = {0, 0};
    size_t launch_smem = 0;
    int launch_nsm = 0;
};

namespace {

constexpr int kPredNT = 256;
constexpr size_t kPredSmemCap = 227 * 1024 - 3072;

template <class T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void free_nn(PredState* p) {
    dfree(p->d_nptr);
    dfree(p->d_nidx);
    dfree(p->d_coff);
    dfree(p->d_cov);
    dfree(p->d_ws);
    p->h_nptr.clear();
    p->h_coff.clear();
    p->ws_stride = 0;
    p->ws_slots = 0;
    p->have_nn = false;
    p->have_pred = false;
}

void free_blocks(PredState* p) {
    free_nn(p);
    dfree(p->d_bptr);
    dfree(p->d_pidx);
    dfree(p->d_cent);
    p->h_bptr.clear();
    p->h_pidx.clear();
    p->h_cent.clear();
    p->nblk = 0;
    p->have_blocks = false;
}

struct PredArgs {
    const double* locs;    // observations, SoA d x n_obs
    int64_t n_obs;
    int d;
    const double* y;
    const double* plocs;   // new locations, SoA d x n_star
    int64_t n_star;
    const int64_t* bptr;
    const int32_t* pidx;
    const int64_t* nptr;
    const int32_t* nidx;
    const int64_t* coff;   // null: no packed covariance output
    DevTheta th;
    ExpConsts ex;
    double* mean;
    double* var;
    double* cov;
    double* ws;
    int64_t ws_stride;
    int smem_n;            // largest N whose matrix lives in shared memory
    int64_t nblk;
    unsigned long long* fail;
};

// Doubles of one block's storage: the packed (N+1)-row triangle, two column buffers of
// N+1 and d x N coordinates (d <= 3).
__host__ __device__ inline int64_t pred_doubles(int64_t N) { return (N + 1) * (N + 2) / 2 + 2 * (N + 1) + 3 * N; }

// One CTA per prediction block (grid-stride).  Gather (with the diagonal sigma^2 + nugget),
// covariance of the strictly lower triangle (flat index, table-driven exponential), then
// the first m columns eliminated
// right-looking with look-ahead: warp 0 finishes column k+1 (update by column k, pivot,
// scale into a column buffer) while the other warps apply column k to the rest of the
// trailing triangle, one barrier per column; a last pass applies column m-1 everywhere.
// GEN: general smoothness (series / continued-fraction Bessel function), instantiated
// apart so that the closed-form path keeps its small register footprint.
template <bool GEN>
__global__ void __launch_bounds__(kPredNT) k_pred(PredArgs a) {
    constexpr int NT = kPredNT, NU = NT - 32;
    extern __shared__ __align__(16) double sm[];
    __shared__ double etab[BV_EXP_TAB];
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < BV_EXP_TAB; i += NT) etab[i] = a.ex.tab[i];
    const double eK = a.ex.k, eL1 = a.ex.l1, eL2 = a.ex.l2;
    const DevTheta th = a.th;
    const int d = a.d;
    for (int64_t blk = blockIdx.x; blk < a.nblk; blk += gridDim.x) {
        const int64_t b0 = a.bptr[blk], n0 = a.nptr[blk];
        const int b = (int)(a.bptr[blk + 1] - b0), m = (int)(a.nptr[blk + 1] - n0);
        const int N = m + b, R = N + 1;
        double* A = N <= a.smem_n ? sm : a.ws + (int64_t)blockIdx.x * a.ws_stride;
        double* col0 = A + pk(R, 0);
        double* col1 = col0 + R;
        double* px = col1 + R;
        for (int t = tid; t < N; t += NT) {
            const bool obs = t < m;
            const int64_t g = obs ? a.nidx[n0 + t] : a.pidx[b0 + (t - m)];
            for (int k = 0; k < d; ++k)
                px[k * N + t] = (obs ? a.locs[(int64_t)k * a.n_obs + g] : a.plocs[(int64_t)k * a.n_star + g]) * inv_range_k(th, k);
            A[pk(N, t)] = obs ? a.y[g] : 0.0;  // data row: [y_NN, 0]
            A[pk(t, t)] = th.sigma2 + th.nugget; // every row is its own point: rho(0) = 1 + nugget
        }
        if (tid == 0) {
            A[pk(N, N)] = 0.0;
            s_fail = 0;
        }
        __syncthreads();
        // covariance (Eq. 5), strictly lower triangle of rows 1..N-1 (flat index f -> row
        // r' + 1, column c with (r', c) = tri_rc(f); packed index f + r' + 1)
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
            const double x = dist_of(acc);
            A[f + r] = GEN ? th.sigma2 * matern_gen_corr(th, x) : matern64t(th.nu_code, th.sigma2, x, etab, eK, eL1, eL2);
        }
        __syncthreads();
        if (m > 0) {
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
            for (int k = 0; k + 1 < m; ++k) {
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
                } else {
                    const int S = N - kk, TS = (S * (S + 1)) >> 1;
                    for (int f = tid - 32; f < TS; f += NU) {
                        int r, c;
                        tri_rc(f, r, c);
                        const int j = kk + 1 + r, i = kk + 1 + c;
                        A[pk(j, i)] = fma(-cur[j], cur[i], A[pk(j, i)]);
                    }
                }
                __syncthreads();
            }
            // column m-1 applied to the Schur complement (rows and columns m..N)
            const double* cur = ((m - 1) & 1) ? col1 : col0;
            const int S = N - m + 1, TS = (S * (S + 1)) >> 1;
            for (int f = tid; f < TS; f += NT) {
                int r, c;
                tri_rc(f, r, c);
                const int j = m + r, i = m + c;
                A[pk(j, i)] = fma(-cur[j], cur[i], A[pk(j, i)]);
            }
            __syncthreads();
        }
        const bool failed = s_fail != 0;
        for (int t = tid; t < b; t += NT) {
            const int g = a.pidx[b0 + t];
            a.mean[g] = failed ? NAN : -A[pk(N, m + t)];
            a.var[g] = failed ? NAN : A[pk(m + t, m + t)];
        }
        if (a.coff) {
            double* out = a.cov + a.coff[blk];
            const int TB = (b * (b + 1)) >> 1;
            for (int f = tid; f < TB; f += NT) {
                int r, c;
                tri_rc(f, r, c);
                out[f] = failed ? NAN : A[pk(m + r, m + c)];
            }
        }
        if (tid == 0 && failed) atomicMin(a.fail, (unsigned long long)blk);
        __syncthreads();
    }
}

// One warp per new location (grid-stride).  Lanes take Box-Muller pairs k = lane,
// lane + 32, ...: pair k of location j is built from SplitMix64 draws 2c and 2c + 1,
// c = j ceil(R/2) + k, and gives z_2k = rho cos(2 pi u2) and z_2k+1 = rho sin(2 pi u2)
// (the second dropped when 2k + 1 = R).  Because every draw is mu + sd z, the sample mean
// is mu + sd zbar and the sample variance sd^2 (sum z^2 - R zbar^2) / (R - 1), so one pass
// accumulating sum z and sum z^2 replaces the two passes over the draws.
__global__ void __launch_bounds__(256) k_cond_sim(const double* __restrict__ mean, const double* __restrict__ var,
                                                  const double* __restrict__ ytrue, int64_t n_star, int R,
                                                  uint64_t stream, double zc, double* __restrict__ lower,
                                                  double* __restrict__ upper, unsigned long long* covered) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int half = (R + 1) >> 1;
    for (int64_t j = w0; j < n_star; j += nw) {
        const uint64_t c0 = (uint64_t)j * (uint64_t)half;
        double s1 = 0.0, s2 = 0.0;
        for (int k = lane; k < half; k += 32) {
            const uint64_t c = c0 + (uint64_t)k;
            const double u1 = 1.0 - (double)(bv_sm64(stream, 2 * c) >> 11) * 0x1p-53;
            const double u2 = (double)(bv_sm64(stream, 2 * c + 1) >> 11) * 0x1p-53;
            const double rho = sqrt(-2.0 * log(u1));
            double sn, cs;
            sincospi(2.0 * u2, &sn, &cs);
            const double za = rho * cs;
            s1 += za;
            s2 = fma(za, za, s2);
            if (2 * k + 1 < R) {
                const double zb = rho * sn;
                s1 += zb;
                s2 = fma(zb, zb, s2);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            const double v = var[j];
            const double sd = sqrt(v > 0.0 ? v : 0.0);
            const double zbar = s1 / (double)R;
            const double vz = fmax(s2 - (double)R * zbar * zbar, 0.0) / (double)(R - 1);
            const double mt = mean[j] + sd * zbar, st = sd * sqrt(vz);
            const double lo = mt - zc * st, up = mt + zc * st;
            if (lower) lower[j] = lo;
            if (upper) upper[j] = up;
            if (ytrue && ytrue[j] >= lo && ytrue[j] <= up) atomicAdd(covered, 1ull);
        }
    }
}

PredState* state(bv_ctx* c) {
    if (!c->pred) c->pred = new PredState();
    return c->pred;
}

}  // namespace

void bv_pred_free(bv_ctx* c) {
    if (!c || !c->pred) return;
    PredState* p = c->pred;
    free_blocks(p);
    dfree(p->d_locs);
    dfree(p->d_ytrue);
    dfree(p->d_mean);
    dfree(p->d_var);
    dfree(p->d_lo);
    dfree(p->d_up);
    dfree(p->d_count);
    dfree(p->d_fail);
    delete p;
    c->pred = nullptr;
}

extern "C" int bv_set_pred_locations(bv_ctx* c, const double* locs_star, const double* y_true, int64_t n_star) {
    if (!c || !locs_star || n_star <= 0 || n_star > INT32_MAX) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    for (int64_t i = 0; i < n_star * c->d; ++i)
        if (!std::isfinite(locs_star[i])) return BV_EINVAL;
    BV_CUDA(cudaSetDevice(c->device));
    bv_pred_free(c);
    PredState* p = state(c);
    const int d = c->d;
    p->n_star = n_star;
    p->h_locs.assign(locs_star, locs_star + n_star * d);
    std::vector<double> soa((size_t)n_star * d);
    for (int64_t i = 0; i < n_star; ++i)
        for (int k = 0; k < d; ++k) soa[(size_t)k * n_star + i] = locs_star[(size_t)i * d + k];
    BV_CUDA(cudaMalloc(&p->d_locs, sizeof(double) * n_star * d));
    BV_CUDA(cudaMalloc(&p->d_mean, sizeof(double) * n_star));
    BV_CUDA(cudaMalloc(&p->d_var, sizeof(double) * n_star));
    BV_CUDA(cudaMalloc(&p->d_lo, sizeof(double) * n_star));
    BV_CUDA(cudaMalloc(&p->d_up, sizeof(double) * n_star));
    BV_CUDA(cudaMalloc(&p->d_count, sizeof(unsigned long long)));
    BV_CUDA(cudaMalloc(&p->d_fail, sizeof(unsigned long long)));
    BV_CUDA(cudaMemcpy(p->d_locs, soa.data(), sizeof(double) * n_star * d, cudaMemcpyHostToDevice));
    if (y_true) {
        BV_CUDA(cudaMalloc(&p->d_ytrue, sizeof(double) * n_star));
        BV_CUDA(cudaMemcpy(p->d_ytrue, y_true, sizeof(double) * n_star, cudaMemcpyHostToDevice));
    }
    return BV_OK;
}

extern "C" int bv_build_pred_blocks(bv_ctx* c, int64_t bc, uint64_t seed, int32_t iters, int64_t* block_ptr,
                                    int32_t* point_idx, int64_t* bc_eff) {
    if (!c || iters < 0) return BV_EINVAL;
    if (!c->pred) return BV_ESTATE;
    PredState* p = c->pred;
    const int64_t n = p->n_star;
    const int d = c->d;
    if (bc <= 0 || bc > n) return BV_EINVAL;
    BV_CUDA(cudaSetDevice(c->device));
    free_blocks(p);
    int32_t* d_label = nullptr;
    double* d_cent = nullptr;
    int64_t* d_counts = nullptr;
    BV_CUDA(cudaMalloc(&d_label, sizeof(int32_t) * n));
    BV_CUDA(cudaMalloc(&d_cent, sizeof(double) * bc * d));
    BV_CUDA(cudaMalloc(&d_counts, sizeof(int64_t) * bc));
    int st = bv_kmeans_device(p->d_locs, n, 0, n, d, bc, seed, iters, d_label, d_cent, c->stream);
    int sc = 0, q = 0;
    if (st == BV_OK) {
        bv_kmeans_scales(p->h_locs.data(), n, d, &sc, &q);
        st = bv_centroids_device(p->d_locs, n, 0, n, d, d_label, bc, q, d_cent, d_counts, c->stream);
    }
    std::vector<int32_t> label(n);
    std::vector<double> cent((size_t)bc * d);
    std::vector<int64_t> counts(bc);
    if (st == BV_OK) {
        cudaError_t e = cudaMemcpyAsync(label.data(), d_label, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cent.data(), d_cent, sizeof(double) * bc * d, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(counts.data(), d_counts, sizeof(int64_t) * bc, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            bv_record_cuda_error(e, "prediction kmeans copy-out", __FILE__, __LINE__);
            st = BV_ECUDA;
        }
    }
    cudaFree(d_label);
    cudaFree(d_cent);
    cudaFree(d_counts);
    if (st != BV_OK) return st;
    // non-empty clusters in cluster-index order (Algorithm 2 has no block permutation)
    std::vector<int64_t> blk_of(bc, -1);
    p->h_bptr.assign(1, 0);
    for (int64_t cl = 0; cl < bc; ++cl) {
        if (counts[cl] == 0) continue;
        blk_of[cl] = (int64_t)p->h_bptr.size() - 1;
        p->h_bptr.push_back(p->h_bptr.back() + counts[cl]);
        for (int k = 0; k < d; ++k) p->h_cent.push_back(cent[(size_t)cl * d + k]);
    }
    p->nblk = (int64_t)p->h_bptr.size() - 1;
    p->h_pidx.assign(n, 0);
    std::vector<int64_t> fill(p->nblk, 0);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t b = blk_of[label[i]];
        p->h_pidx[p->h_bptr[b] + fill[b]++] = (int32_t)i;
    }
    BV_CUDA(cudaMalloc(&p->d_bptr, sizeof(int64_t) * (p->nblk + 1)));
    BV_CUDA(cudaMalloc(&p->d_pidx, sizeof(int32_t) * n));
    BV_CUDA(cudaMalloc(&p->d_cent, sizeof(double) * p->nblk * d));
    BV_CUDA(cudaMemcpy(p->d_bptr, p->h_bptr.data(), sizeof(int64_t) * (p->nblk + 1), cudaMemcpyHostToDevice));
    BV_CUDA(cudaMemcpy(p->d_pidx, p->h_pidx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    BV_CUDA(cudaMemcpy(p->d_cent, p->h_cent.data(), sizeof(double) * p->nblk * d, cudaMemcpyHostToDevice));
    p->have_blocks = true;
    if (bc_eff) *bc_eff = p->nblk;
    if (block_ptr) memcpy(block_ptr, p->h_bptr.data(), sizeof(int64_t) * (p->nblk + 1));
    if (point_idx) memcpy(point_idx, p->h_pidx.data(), sizeof(int32_t) * n);
    return BV_OK;
}

extern "C" int bv_select_pred_neighbors(bv_ctx* c, int32_t m, int64_t* nn_ptr, int32_t* nn_idx) {
    if (!c || m < 0) return BV_EINVAL;
    if (!c->pred || !c->pred->have_blocks) return BV_ESTATE;
    PredState* p = c->pred;
    const int64_t mi = std::min<int64_t>(m, c->n_tot);
    if (mi > 4000) return BV_EINVAL;  // exact-key list capacity of the selection kernel
    BV_CUDA(cudaSetDevice(c->device));
    free_nn(p);
    const int d = c->d;
    p->h_nptr.assign(p->nblk + 1, 0);
    p->h_coff.assign(p->nblk + 1, 0);
    int64_t maxN = 0;
    for (int64_t i = 0; i < p->nblk; ++i) {
        const int64_t b = p->h_bptr[i + 1] - p->h_bptr[i];
        p->h_nptr[i + 1] = p->h_nptr[i] + mi;
        p->h_coff[i + 1] = p->h_coff[i] + b * (b + 1) / 2;
        maxN = std::max(maxN, mi + b);
    }
    if (maxN > BV_LARGE_MAX_N) return BV_EINVAL;
    BV_CUDA(cudaMalloc(&p->d_nptr, sizeof(int64_t) * (p->nblk + 1)));
    BV_CUDA(cudaMalloc(&p->d_nidx, sizeof(int32_t) * std::max<int64_t>(p->h_nptr.back(), 1)));
    BV_CUDA(cudaMalloc(&p->d_coff, sizeof(int64_t) * (p->nblk + 1)));
    BV_CUDA(cudaMalloc(&p->d_cov, sizeof(double) * std::max<int64_t>(p->h_coff.back(), 1)));
    BV_CUDA(cudaMemcpy(p->d_nptr, p->h_nptr.data(), sizeof(int64_t) * (p->nblk + 1), cudaMemcpyHostToDevice));
    BV_CUDA(cudaMemcpy(p->d_coff, p->h_coff.data(), sizeof(int64_t) * (p->nblk + 1), cudaMemcpyHostToDevice));
    double amax = 0.0;
    for (double v : c->h_locs) amax = std::max(amax, fabs(v));
    for (double v : p->h_locs) amax = std::max(amax, fabs(v));
    if (mi > 0)
        BV_TRY(bv_select_pred_neighbors_device(c->d_locs, c->n_tot, d, p->d_cent, p->nblk, p->d_nptr, p->d_nidx, amax,
                                               c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    // workspace slots for blocks whose matrix does not fit in shared memory
    int smem_n = 0;
    while (pred_doubles(smem_n + 1) * 8 <= (int64_t)kPredSmemCap) ++smem_n;
    if (maxN > smem_n) {
        int grid = 0;
        BV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&grid, k_pred<false>, kPredNT, 0));
        p->ws_slots = std::max(1, std::min<int>(grid * c->num_sms, 2 * c->num_sms));
        p->ws_stride = (pred_doubles(maxN) + 31) / 32 * 32;
        BV_CUDA(cudaMalloc(&p->d_ws, sizeof(double) * p->ws_stride * p->ws_slots));
    }
    p->launch_grid[0] = p->launch_grid[1] = 0;
    p->have_nn = true;
    if (nn_ptr) memcpy(nn_ptr, p->h_nptr.data(), sizeof(int64_t) * (p->nblk + 1));
    if (nn_idx && p->h_nptr.back() > 0)
        BV_CUDA(cudaMemcpy(nn_idx, p->d_nidx, sizeof(int32_t) * p->h_nptr.back(), cudaMemcpyDeviceToHost));
    return BV_OK;
}

extern "C" int bv_get_pred_sizes(bv_ctx* c, int64_t* n_star, int64_t* nblk, int64_t* n_nn, int64_t* n_cov) {
    if (!c) return BV_EINVAL;
    PredState* p = c->pred;
    if (n_star) *n_star = p ? p->n_star : 0;
    if (nblk) *nblk = p ? p->nblk : 0;
    if (n_nn) *n_nn = (p && p->have_nn) ? p->h_nptr.back() : 0;
    if (n_cov) *n_cov = (p && p->have_nn) ? p->h_coff.back() : 0;
    return BV_OK;
}

// Launch shape of the prediction kernel: one CTA per block up to the resident limit,
// dynamic shared memory for the largest block that fits.
static int pred_launch(bv_ctx* c, const DevTheta& th, bool with_cov) {
    PredState* p = c->pred;
    const bool gen = th.nu_code == NU_GENERAL;
    auto kern = gen ? k_pred<true> : k_pred<false>;
    if (p->launch_grid[gen] == 0) {
        int64_t maxN = 0;
        for (int64_t i = 0; i < p->nblk; ++i)
            maxN = std::max(maxN, (p->h_nptr[i + 1] - p->h_nptr[i]) + (p->h_bptr[i + 1] - p->h_bptr[i]));
        int smem_n = 0;
        while (pred_doubles(smem_n + 1) * 8 <= (int64_t)kPredSmemCap) ++smem_n;
        const int64_t nsm = std::min<int64_t>(maxN, smem_n);
        const size_t smem = (size_t)pred_doubles(nsm) * 8;
        BV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPredSmemCap));
        int per_sm = 0;
        BV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPredNT, smem));
        int64_t grid = std::max(1, per_sm) * (int64_t)c->num_sms;
        grid = std::min<int64_t>(grid, p->nblk);
        if (maxN > smem_n) grid = std::min<int64_t>(grid, p->ws_slots);
        p->launch_grid[gen] = std::max<int64_t>(1, grid);
        p->launch_smem = smem;
        p->launch_nsm = (int)nsm;
    }
    const int64_t grid = p->launch_grid[gen];
    const size_t smem = p->launch_smem;
    const int64_t nsm = p->launch_nsm;
    PredArgs a;
    a.locs = c->d_locs;
    a.n_obs = c->n_tot;
    a.d = c->d;
    a.y = c->d_y;
    a.plocs = p->d_locs;
    a.n_star = p->n_star;
    a.bptr = p->d_bptr;
    a.pidx = p->d_pidx;
    a.nptr = p->d_nptr;
    a.nidx = p->d_nidx;
    a.coff = with_cov ? p->d_coff : nullptr;
    a.th = th;
    bv_exp_consts(&a.ex);
    a.mean = p->d_mean;
    a.var = p->d_var;
    a.cov = p->d_cov;
    a.ws = p->d_ws;
    a.ws_stride = p->ws_stride;
    a.smem_n = (int)nsm;
    a.nblk = p->nblk;
    a.fail = p->d_fail;
    BV_CUDA(cudaMemsetAsync(p->d_fail, 0xff, sizeof(unsigned long long), c->stream));
    kern<<<(unsigned)grid, kPredNT, smem, c->stream>>>(a);
    BV_CUDA(cudaGetLastError());
    return BV_OK;
}

extern "C" int bv_predict(bv_ctx* c, const bv_theta* theta, double* mean, double* var, double* cov_packed) {
    if (!c || !theta) return BV_EINVAL;
    if (!c->pred || !c->pred->have_nn || !c->have_y) return BV_ESTATE;
    PredState* p = c->pred;
    DevTheta th;
    BV_TRY(bv_theta_to_dev(theta, c->d, &th));
    BV_CUDA(cudaSetDevice(c->device));
    BV_TRY(pred_launch(c, th, cov_packed != nullptr));
    unsigned long long fail = 0;
    BV_CUDA(cudaMemcpyAsync(&fail, p->d_fail, sizeof(fail), cudaMemcpyDeviceToHost, c->stream));
    if (mean) BV_CUDA(cudaMemcpyAsync(mean, p->d_mean, sizeof(double) * p->n_star, cudaMemcpyDeviceToHost, c->stream));
    if (var) BV_CUDA(cudaMemcpyAsync(var, p->d_var, sizeof(double) * p->n_star, cudaMemcpyDeviceToHost, c->stream));
    if (cov_packed && p->h_coff.back() > 0)
        BV_CUDA(cudaMemcpyAsync(cov_packed, p->d_cov, sizeof(double) * p->h_coff.back(), cudaMemcpyDeviceToHost,
                                c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    p->have_pred = true;
    return fail == ~0ull ? BV_OK : BV_ENOTPD;
}

extern "C" int bv_cond_sim(bv_ctx* c, int32_t rounds, uint64_t seed, double z_crit, double* lower, double* upper,
                           int64_t* covered) {
    if (!c || rounds < 2 || !(z_crit >= 0.0)) return BV_EINVAL;
    if (!c->pred || !c->pred->have_pred) return BV_ESTATE;
    PredState* p = c->pred;
    BV_CUDA(cudaSetDevice(c->device));
    BV_CUDA(cudaMemsetAsync(p->d_count, 0, sizeof(unsigned long long), c->stream));
    const int64_t warps = p->n_star;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, (int64_t)c->num_sms * 8));
    k_cond_sim<<<(unsigned)grid, 256, 0, c->stream>>>(p->d_mean, p->d_var, p->d_ytrue, p->n_star, rounds,
                                                      BV_STREAM_CSIM(seed), z_crit, p->d_lo, p->d_up, p->d_count);
    BV_CUDA(cudaGetLastError());
    unsigned long long cnt = 0;
    BV_CUDA(cudaMemcpyAsync(&cnt, p->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    if (lower) BV_CUDA(cudaMemcpyAsync(lower, p->d_lo, sizeof(double) * p->n_star, cudaMemcpyDeviceToHost, c->stream));
    if (upper) BV_CUDA(cudaMemcpyAsync(upper, p->d_up, sizeof(double) * p->n_star, cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    if (covered) *covered = p->d_ytrue ? (int64_t)cnt : -1;
    return BV_OK;
}

extern "C" int bv_pred_plan_info(bv_ctx* c, double* flops, double* cov_evals) {
    if (!c || !c->pred || !c->pred->have_nn) return BV_ESTATE;
    PredState* p = c->pred;
    double f = 0.0, e = 0.0;
    for (int64_t i = 0; i < p->nblk; ++i) {
        const double m = (double)(p->h_nptr[i + 1] - p->h_nptr[i]);
        const double N = m + (double)(p->h_bptr[i + 1] - p->h_bptr[i]);
        // eliminating column k of the (N+1)-row matrix: N - k scalings and (N - k)(N - k + 1) / 2
        // multiply-adds on the trailing triangle; summed over k < m
        for (int64_t k = 0; k < (int64_t)m; ++k) {
            const double r = N - (double)k;
            f += r + r * (r + 1.0);
        }
        e += N * (N + 1.0) / 2.0;
    }
    if (flops) *flops = f;
    if (cov_evals) *cov_evals = e;
    return BV_OK;
}
