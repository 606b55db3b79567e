// bv_warm.cu -- learned warm start: dataset features (semivariogram + structure
// statistics) and a small MLP trained and evaluated with this library's own kernels.
//
// The paper's non-learned heuristic (Sec. 2.3) is to start the estimation from a
// cheaper fit; here a network maps summary features to a starting theta.  The same
// search (bv_mle) runs from either start, and its cold-started result is the standard
// that the warm-started estimate must reproduce.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "bv_internal.h"

namespace {

// ---------------------------------------------------------------------------------
// Semivariogram: 32 bins of width 1/64 on (0, 0.5]; the bin decision is exact FP64
// (squared distance without contraction, correctly rounded sqrt, exact scaling by 64).
// ---------------------------------------------------------------------------------
constexpr int kVT = 128;   // points per tile
constexpr int kBins = 32;

__global__ void __launch_bounds__(kVT) k_variogram(const double* __restrict__ xs, const double* __restrict__ ys_,
                                                   const double* __restrict__ zs, const double* __restrict__ val,
                                                   int d, int64_t P, double* __restrict__ part_sum,
                                                   unsigned long long* __restrict__ part_cnt) {
    __shared__ double tx[kVT], ty[kVT], tz[kVT], tv[kVT];
    __shared__ double bsum[kVT / 32][kBins];
    __shared__ unsigned int bcnt[kVT / 32][kBins];
    const int tid = threadIdx.x, w = tid >> 5;
    for (int k = tid; k < (kVT / 32) * kBins; k += kVT) {
        bsum[k / kBins][k % kBins] = 0.0;
        bcnt[k / kBins][k % kBins] = 0u;
    }
    // this CTA's tile pair (it <= jt) from its linear index over the upper triangle
    const int64_t q = blockIdx.x;
    int64_t jt = (int64_t)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
    if ((jt + 1) * (jt + 2) / 2 <= q) ++jt;
    if (jt * (jt + 1) / 2 > q) --jt;
    const int64_t it = q - jt * (jt + 1) / 2;
    const int64_t i = it * kVT + tid;
    const bool live = i < P;
    double xi = 0, yi = 0, zi = 0, vi = 0;
    if (live) {
        xi = xs[i];
        yi = d > 1 ? ys_[i] : 0.0;
        zi = d > 2 ? zs[i] : 0.0;
        vi = val[i];
    }
    {
        __syncthreads();
        const int64_t j0 = jt * kVT;
        if (j0 + tid < P) {
            tx[tid] = xs[j0 + tid];
            ty[tid] = d > 1 ? ys_[j0 + tid] : 0.0;
            tz[tid] = d > 2 ? zs[j0 + tid] : 0.0;
            tv[tid] = val[j0 + tid];
        }
        __syncthreads();
        const int jn = (int)min((int64_t)kVT, P - j0);
        if (live) {
            for (int t = 0; t < jn; ++t) {
                if (j0 + t <= i) continue;
                const double dx = __dsub_rn(xi, tx[t]);
                double d2 = __dmul_rn(dx, dx);
                if (d > 1) {
                    const double dy = __dsub_rn(yi, ty[t]);
                    d2 = __dadd_rn(d2, __dmul_rn(dy, dy));
                }
                if (d > 2) {
                    const double dz = __dsub_rn(zi, tz[t]);
                    d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
                }
                if (!(d2 > 0.0) || d2 > 0.25) continue;
                int k = (int)floor(__dsqrt_rn(d2) * 64.0);
                k = min(k, kBins - 1);
                const double dv = vi - tv[t];
                atomicAdd(&bsum[w][k], 0.5 * dv * dv);
                atomicAdd(&bcnt[w][k], 1u);
            }
        }
    }
    __syncthreads();
    if (tid < kBins) {
        double s = 0.0;
        unsigned long long c = 0;
        for (int wq = 0; wq < kVT / 32; ++wq) {
            s += bsum[wq][tid];
            c += bcnt[wq][tid];
        }
        part_sum[q * kBins + tid] = s;
        part_cnt[q * kBins + tid] = c;
    }
}

// Nearest neighbour of every subsample point (exact FP64 squared distance without
// contraction; ties to the lowest index), in three passes over all ordered pairs:
// the minimum distance, then the lowest index attaining it, then the semivariance term.
// pass 1 (which = 0): best[i] = min_j d2 bits; pass 2 (which = 1): arg[i] = min j with
// d2 == best[i].  One thread per i, j streamed through shared memory.
__global__ void __launch_bounds__(kVT) k_nn_pass(const double* __restrict__ xs, const double* __restrict__ ys_,
                                                 const double* __restrict__ zs, int d, int64_t P, int which,
                                                 unsigned long long* __restrict__ best,
                                                 unsigned long long* __restrict__ arg) {
    __shared__ double tx[kVT], ty[kVT], tz[kVT];
    const int64_t i = blockIdx.x * (int64_t)kVT + threadIdx.x;
    const bool live = i < P;
    double xi = 0, yi = 0, zi = 0;
    if (live) {
        xi = xs[i];
        yi = d > 1 ? ys_[i] : 0.0;
        zi = d > 2 ? zs[i] : 0.0;
    }
    unsigned long long bi = ~0ull, ai = ~0ull;
    const unsigned long long target = (live && which == 1) ? best[i] : 0ull;
    for (int64_t j0 = 0; j0 < P; j0 += kVT) {
        __syncthreads();
        if (j0 + threadIdx.x < P) {
            tx[threadIdx.x] = xs[j0 + threadIdx.x];
            ty[threadIdx.x] = d > 1 ? ys_[j0 + threadIdx.x] : 0.0;
            tz[threadIdx.x] = d > 2 ? zs[j0 + threadIdx.x] : 0.0;
        }
        __syncthreads();
        if (!live) continue;
        const int jn = (int)min((int64_t)kVT, P - j0);
        for (int t = 0; t < jn; ++t) {
            const int64_t j = j0 + t;
            if (j == i) continue;
            const double dx = __dsub_rn(xi, tx[t]);
            double d2 = __dmul_rn(dx, dx);
            if (d > 1) {
                const double dy = __dsub_rn(yi, ty[t]);
                d2 = __dadd_rn(d2, __dmul_rn(dy, dy));
            }
            if (d > 2) {
                const double dz = __dsub_rn(zi, tz[t]);
                d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
            }
            const unsigned long long kb = (unsigned long long)__double_as_longlong(d2);
            if (which == 0) {
                if (kb < bi) bi = kb;
            } else if (kb == target && (unsigned long long)j < ai) {
                ai = (unsigned long long)j;
            }
        }
    }
    if (live) {
        if (which == 0) best[i] = bi;
        else arg[i] = ai;
    }
}

// ---------------------------------------------------------------------------------
// MLP kernels (FP32).  Activations are row-major [batch][features].
// ---------------------------------------------------------------------------------
constexpr int kH = 128, kOut = 6;
constexpr int kLayers = 4;
const int kIn[kLayers] = {BV_NFEAT, kH, kH, kH};
const int kOutDim[kLayers] = {kH, kH, kH, kOut};

__global__ void k_lin_fwd(const float* __restrict__ X, const float* __restrict__ W, const float* __restrict__ b,
                          float* __restrict__ Y, int B, int I, int O) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * O) return;
    const int r = idx / O, o = idx % O;
    float acc = b[o];
    for (int i = 0; i < I; ++i) acc = fmaf(X[r * I + i], W[i * O + o], acc);
    Y[idx] = acc;
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void k_gelu_fwd(const float* __restrict__ Y, float* __restrict__ Z, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) Z[i] = gelu(Y[i]);
}

// dZ and dY may be the same buffer (the backward pass scales a layer's gradient in place),
// so neither is declared __restrict__; each thread reads and writes its own element only.
__global__ void k_gelu_bwd(const float* __restrict__ Y, const float* dZ, float* dY, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dY[i] = dZ[i] * gelu_d(Y[i]);
}

// dX[r][i] = sum_o dY[r][o] W[i][o]
__global__ void k_lin_bwd_x(const float* __restrict__ dY, const float* __restrict__ W, float* __restrict__ dX,
                            int B, int I, int O) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * I) return;
    const int r = idx / I, i = idx % I;
    float acc = 0.f;
    for (int o = 0; o < O; ++o) acc = fmaf(dY[r * O + o], W[i * O + o], acc);
    dX[idx] = acc;
}

// dW[i][o] = sum_r X[r][i] dY[r][o];  db[o] = sum_r dY[r][o]  (fixed order: deterministic)
__global__ void k_lin_bwd_w(const float* __restrict__ X, const float* __restrict__ dY, float* __restrict__ dW,
                            float* __restrict__ db, int B, int I, int O) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < I * O) {
        const int i = idx / O, o = idx % O;
        float acc = 0.f;
        for (int r = 0; r < B; ++r) acc = fmaf(X[r * I + i], dY[r * O + o], acc);
        dW[idx] = acc;
    } else if (idx < I * O + O) {
        const int o = idx - I * O;
        float acc = 0.f;
        for (int r = 0; r < B; ++r) acc += dY[r * O + o];
        db[o] = acc;
    }
}

// Loss of one batch and d loss / d out.  out[r] = (3 standardised regressions, 3 logits);
// T[r] = (standardised log sigma^2, log beta, log tau^2, nu class index as float).
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ T, float* __restrict__ dout,
                       float* __restrict__ loss_rows, int B) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B) return;
    const float* o = out + r * kOut;
    const float* t = T + r * 4;
    float* g = dout + r * kOut;
    float l = 0.f;
    for (int k = 0; k < 3; ++k) {
        const float e = o[k] - t[k];
        l += e * e / 3.0f;
        g[k] = 2.0f * e / 3.0f / (float)B;
    }
    const float mx = fmaxf(o[3], fmaxf(o[4], o[5]));
    const float e0 = expf(o[3] - mx), e1 = expf(o[4] - mx), e2 = expf(o[5] - mx);
    const float z = e0 + e1 + e2;
    const int cls = (int)t[3];
    const float pr[3] = {e0 / z, e1 / z, e2 / z};
    l += -logf(pr[cls]);
    for (int k = 0; k < 3; ++k) g[3 + k] = (pr[k] - (k == cls ? 1.0f : 0.0f)) / (float)B;
    loss_rows[r] = l;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Parameter offsets inside the flat parameter vector.
struct Offs {
    int w[kLayers], b[kLayers];
};
Offs offsets() {
    Offs o;
    int p = 0;
    for (int l = 0; l < kLayers; ++l) {
        o.w[l] = p;
        p += kIn[l] * kOutDim[l];
        o.b[l] = p;
        p += kOutDim[l];
    }
    return o;
}

inline unsigned nb(int n) { return (unsigned)((n + 255) / 256); }

// Device workspace for forward/backward on batches of up to Bmax rows.
struct MLPWork {
    int Bmax = 0;
    float *X = nullptr, *T = nullptr, *P = nullptr, *G = nullptr;
    float* Y[kLayers] = {nullptr};   // pre-activations
    float* Z[kLayers] = {nullptr};   // activations (Z[3] = outputs)
    float *dA = nullptr, *dB = nullptr, *loss = nullptr;
    int alloc(int B) {
        Bmax = B;
        BV_CUDA(cudaMalloc(&X, sizeof(float) * B * BV_NFEAT));
        BV_CUDA(cudaMalloc(&T, sizeof(float) * B * 4));
        BV_CUDA(cudaMalloc(&P, sizeof(float) * BV_MLP_NPARAM));
        BV_CUDA(cudaMalloc(&G, sizeof(float) * BV_MLP_NPARAM));
        for (int l = 0; l < kLayers; ++l) {
            BV_CUDA(cudaMalloc(&Y[l], sizeof(float) * B * kOutDim[l]));
            BV_CUDA(cudaMalloc(&Z[l], sizeof(float) * B * kOutDim[l]));
        }
        BV_CUDA(cudaMalloc(&dA, sizeof(float) * B * kH));
        BV_CUDA(cudaMalloc(&dB, sizeof(float) * B * kH));
        BV_CUDA(cudaMalloc(&loss, sizeof(float) * B));
        return BV_OK;
    }
    ~MLPWork() {
        cudaFree(X);
        cudaFree(T);
        cudaFree(P);
        cudaFree(G);
        for (int l = 0; l < kLayers; ++l) {
            cudaFree(Y[l]);
            cudaFree(Z[l]);
        }
        cudaFree(dA);
        cudaFree(dB);
        cudaFree(loss);
    }
};

// Forward on W.X (B rows): Z[3] = outputs.
cudaError_t forward(MLPWork& w, int B) {
    const Offs o = offsets();
    const float* in = w.X;
    for (int l = 0; l < kLayers; ++l) {
        k_lin_fwd<<<nb(B * kOutDim[l]), 256>>>(in, w.P + o.w[l], w.P + o.b[l], w.Y[l], B, kIn[l], kOutDim[l]);
        if (l < kLayers - 1) {
            k_gelu_fwd<<<nb(B * kOutDim[l]), 256>>>(w.Y[l], w.Z[l], B * kOutDim[l]);
            in = w.Z[l];
        } else {
            cudaMemcpyAsync(w.Z[l], w.Y[l], sizeof(float) * B * kOut, cudaMemcpyDeviceToDevice);
        }
    }
    return cudaGetLastError();
}

// Loss + backward into w.G (after forward).
cudaError_t backward(MLPWork& w, int B) {
    const Offs o = offsets();
    float* dout = w.dA;  // B x 6
    k_loss<<<nb(B), 256>>>(w.Z[3], w.T, dout, w.loss, B);
    float* dcur = dout;
    float* dnext = w.dB;
    for (int l = kLayers - 1; l >= 0; --l) {
        const float* xin = l == 0 ? w.X : w.Z[l - 1];
        k_lin_bwd_w<<<nb(kIn[l] * kOutDim[l] + kOutDim[l]), 256>>>(xin, dcur, w.G + o.w[l], w.G + o.b[l], B, kIn[l],
                                                                    kOutDim[l]);
        if (l > 0) {
            k_lin_bwd_x<<<nb(B * kIn[l]), 256>>>(dcur, w.P + o.w[l], dnext, B, kIn[l], kOutDim[l]);
            k_gelu_bwd<<<nb(B * kIn[l]), 256>>>(w.Y[l - 1], dnext, dnext, B * kIn[l]);
            std::swap(dcur, dnext);
        }
    }
    return cudaGetLastError();
}

void standardise_rows(const float* blob, const float* X, int64_t n, std::vector<float>& out) {
    out.resize((size_t)n * BV_NFEAT);
    for (int64_t r = 0; r < n; ++r)
        for (int k = 0; k < BV_NFEAT; ++k)
            out[(size_t)r * BV_NFEAT + k] = (X[r * BV_NFEAT + k] - blob[k]) / blob[BV_NFEAT + k];
}

int nu_class(float nu) { return nu < 1.0f ? 0 : (nu < 2.0f ? 1 : 2); }

void standardise_targets(const float* blob, const float* T, int64_t n, std::vector<float>& out) {
    out.resize((size_t)n * 4);
    const float* ym = blob + 2 * BV_NFEAT;
    const float* ys = ym + 3;
    for (int64_t r = 0; r < n; ++r) {
        for (int k = 0; k < 3; ++k) out[(size_t)r * 4 + k] = (T[r * 4 + k] - ym[k]) / ys[k];
        out[(size_t)r * 4 + 3] = (float)nu_class(T[r * 4 + 3]);
    }
}

}  // namespace

// ------------------------------------------------------------------------------------
// features
// ------------------------------------------------------------------------------------
extern "C" int bv_features(bv_ctx* c, int32_t max_points, uint64_t seed, float* out) {
    if (!c || !out || max_points < 2) return BV_EINVAL;
    if (!c->have_nn) return BV_ESTATE;
    BV_CUDA(cudaSetDevice(c->device));
    const int d = c->d;
    std::vector<double> y(c->n_tot);
    BV_CUDA(cudaMemcpyAsync(y.data(), c->d_y, sizeof(double) * c->n_tot, cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    for (int ds = 0; ds < c->ndata; ++ds) {
        const int64_t off = c->pt_off[ds], n = c->pt_off[ds + 1] - off;
        // seeded subsample
        std::vector<int64_t> sel;
        for (int64_t j = 0; j < n; ++j) {
            const uint64_t r = bv_sm64(seed, (uint64_t)j);
            const uint64_t u = (uint64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)n) >> 64);
            if (n <= max_points || u < (uint64_t)max_points) sel.push_back(j);
        }
        const int64_t P = (int64_t)sel.size();
        std::vector<double> soa((size_t)P * 4, 0.0);
        for (int64_t q = 0; q < P; ++q) {
            for (int k = 0; k < d; ++k) soa[(size_t)k * P + q] = c->h_locs[(size_t)(off + sel[q]) * d + k];
            soa[(size_t)3 * P + q] = y[(size_t)(off + sel[q])];
        }
        const int64_t ntile0 = (P + kVT - 1) / kVT;
        const int64_t ntile = ntile0 * (ntile0 + 1) / 2;   // tile pairs
        double* dsoa = nullptr;
        double* psum = nullptr;
        unsigned long long* pcnt = nullptr;
        BV_CUDA(cudaMalloc(&dsoa, sizeof(double) * P * 4));
        BV_CUDA(cudaMalloc(&psum, sizeof(double) * ntile * kBins));
        BV_CUDA(cudaMalloc(&pcnt, sizeof(unsigned long long) * ntile * kBins));
        BV_CUDA(cudaMemcpyAsync(dsoa, soa.data(), sizeof(double) * P * 4, cudaMemcpyHostToDevice, c->stream));
        k_variogram<<<(unsigned)ntile, kVT, 0, c->stream>>>(dsoa, dsoa + P, dsoa + 2 * P, dsoa + 3 * P, d, P, psum,
                                                            pcnt);
        BV_CUDA(cudaGetLastError());
        std::vector<double> hs((size_t)ntile * kBins);
        std::vector<unsigned long long> hc((size_t)ntile * kBins);
        BV_CUDA(cudaMemcpyAsync(hs.data(), psum, sizeof(double) * ntile * kBins, cudaMemcpyDeviceToHost, c->stream));
        BV_CUDA(cudaMemcpyAsync(hc.data(), pcnt, sizeof(unsigned long long) * ntile * kBins, cudaMemcpyDeviceToHost,
                                c->stream));
        BV_CUDA(cudaStreamSynchronize(c->stream));
        // nearest neighbour inside the subsample: semivariance and distance at the
        // smallest lag the data offer (these carry the nugget)
        double nn_gamma = 0.0, nn_dist = 0.0;
        if (P >= 2) {
            unsigned long long *dbest = nullptr, *darg = nullptr;
            BV_CUDA(cudaMalloc(&dbest, sizeof(unsigned long long) * P));
            BV_CUDA(cudaMalloc(&darg, sizeof(unsigned long long) * P));
            const unsigned g = (unsigned)((P + kVT - 1) / kVT);
            k_nn_pass<<<g, kVT, 0, c->stream>>>(dsoa, dsoa + P, dsoa + 2 * P, d, P, 0, dbest, darg);
            k_nn_pass<<<g, kVT, 0, c->stream>>>(dsoa, dsoa + P, dsoa + 2 * P, d, P, 1, dbest, darg);
            BV_CUDA(cudaGetLastError());
            std::vector<unsigned long long> hb(P), ha(P);
            BV_CUDA(cudaMemcpyAsync(hb.data(), dbest, sizeof(unsigned long long) * P, cudaMemcpyDeviceToHost, c->stream));
            BV_CUDA(cudaMemcpyAsync(ha.data(), darg, sizeof(unsigned long long) * P, cudaMemcpyDeviceToHost, c->stream));
            BV_CUDA(cudaStreamSynchronize(c->stream));
            cudaFree(dbest);
            cudaFree(darg);
            for (int64_t q = 0; q < P; ++q) {
                double d2;
                memcpy(&d2, &hb[q], sizeof(d2));
                const double dv = soa[(size_t)3 * P + q] - soa[(size_t)3 * P + (int64_t)ha[q]];
                nn_gamma += 0.5 * dv * dv;
                nn_dist += sqrt(d2);
            }
            nn_gamma /= (double)P;
            nn_dist /= (double)P;
        }
        cudaFree(dsoa);
        cudaFree(psum);
        cudaFree(pcnt);
        // variance of y over the dataset (two-pass)
        double mean = 0.0;
        for (int64_t j = 0; j < n; ++j) mean += y[(size_t)(off + j)];
        mean /= (double)n;
        double var = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double t = y[(size_t)(off + j)] - mean;
            var += t * t;
        }
        var /= (double)n;
        if (!(var > 0.0)) var = 1e-300;
        float* f = out + (size_t)ds * BV_NFEAT;
        for (int k = 0; k < kBins; ++k) {
            double s = 0.0;
            unsigned long long cnt = 0;
            for (int64_t t = 0; t < ntile; ++t) {  // fixed order
                s += hs[(size_t)t * kBins + k];
                cnt += hc[(size_t)t * kBins + k];
            }
            f[k] = cnt ? (float)(s / (double)cnt / var) : 0.0f;
        }
        // block-size histogram: fractions of the dataset's blocks with b_i in 1-4, 5-8,
        // 9-12, 13-16 and 17 or more points (unlike extremes or means of the structure,
        // stable as n grows at a fixed points-per-block ratio)
        const int64_t b0 = c->ds_blk_off[ds], b1 = c->ds_blk_off[ds + 1], nbk = b1 - b0;
        int64_t hist[5] = {0, 0, 0, 0, 0};
        for (int64_t i = b0; i < b1; ++i) {
            const int64_t bs = c->h_bptr[i + 1] - c->h_bptr[i];
            ++hist[std::min<int64_t>(4, std::max<int64_t>(0, (bs - 1) / 4))];
        }
        f[32] = (float)log(var);
        for (int k = 0; k < 5; ++k) f[33 + k] = (float)((double)hist[k] / (double)nbk);
        f[38] = (float)(nn_gamma / var);
        f[39] = (float)(64.0 * nn_dist);
    }
    return BV_OK;
}

// ------------------------------------------------------------------------------------
// MLP training and inference
// ------------------------------------------------------------------------------------
extern "C" int bv_mlp_forward(const float* blob, const float* X, int64_t n, float* out) {
    if (!blob || !X || !out || n <= 0) return BV_EINVAL;
    std::vector<float> xs;
    standardise_rows(blob, X, n, xs);
    MLPWork w;
    const int B = (int)std::min<int64_t>(n, 4096);
    BV_TRY(w.alloc(B));
    BV_CUDA(cudaMemcpy(w.P, blob + 2 * BV_NFEAT + 6, sizeof(float) * BV_MLP_NPARAM, cudaMemcpyHostToDevice));
    for (int64_t r0 = 0; r0 < n; r0 += B) {
        const int b = (int)std::min<int64_t>(B, n - r0);
        BV_CUDA(cudaMemcpy(w.X, xs.data() + r0 * BV_NFEAT, sizeof(float) * b * BV_NFEAT, cudaMemcpyHostToDevice));
        BV_CUDA(forward(w, b));
        BV_CUDA(cudaMemcpy(out + r0 * kOut, w.Z[3], sizeof(float) * b * kOut, cudaMemcpyDeviceToHost));
    }
    return BV_OK;
}

extern "C" int bv_mlp_loss_grad(const float* blob, const float* X, const float* T, int64_t n, float* loss_out,
                                float* grad_out) {
    if (!blob || !X || !T || n <= 0 || n > 65536) return BV_EINVAL;
    std::vector<float> xs, ts;
    standardise_rows(blob, X, n, xs);
    standardise_targets(blob, T, n, ts);
    MLPWork w;
    BV_TRY(w.alloc((int)n));
    BV_CUDA(cudaMemcpy(w.P, blob + 2 * BV_NFEAT + 6, sizeof(float) * BV_MLP_NPARAM, cudaMemcpyHostToDevice));
    BV_CUDA(cudaMemcpy(w.X, xs.data(), sizeof(float) * n * BV_NFEAT, cudaMemcpyHostToDevice));
    BV_CUDA(cudaMemcpy(w.T, ts.data(), sizeof(float) * n * 4, cudaMemcpyHostToDevice));
    BV_CUDA(forward(w, (int)n));
    BV_CUDA(backward(w, (int)n));
    std::vector<float> l(n);
    BV_CUDA(cudaMemcpy(l.data(), w.loss, sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (grad_out) BV_CUDA(cudaMemcpy(grad_out, w.G, sizeof(float) * BV_MLP_NPARAM, cudaMemcpyDeviceToHost));
    double s = 0.0;
    for (float v : l) s += v;
    if (loss_out) *loss_out = (float)(s / (double)n);
    return BV_OK;
}

extern "C" int bv_mlp_train(const float* X, const float* T, int64_t n, int32_t epochs, int32_t batch, float lr,
                            uint64_t seed, float* blob, float* loss_out) {
    if (!X || !T || !blob || n < 2 || epochs < 1 || batch < 1 || !(lr > 0.f)) return BV_EINVAL;
    // standardisation from the training set (FP64 sums)
    for (int k = 0; k < BV_NFEAT; ++k) {
        double m = 0.0, q = 0.0;
        for (int64_t r = 0; r < n; ++r) m += X[r * BV_NFEAT + k];
        m /= (double)n;
        for (int64_t r = 0; r < n; ++r) {
            const double t = X[r * BV_NFEAT + k] - m;
            q += t * t;
        }
        const double sd = sqrt(q / (double)n);
        blob[k] = (float)m;
        // a feature constant over the training set carries no information: a huge scale
        // maps it to 0 for every input, so an unseen value cannot push the network out of
        // its training distribution
        blob[BV_NFEAT + k] = (float)(sd > 1e-6 * (fabs(m) + 1.0) ? sd : 1e30);
    }
    for (int k = 0; k < 3; ++k) {
        double m = 0.0, q = 0.0;
        for (int64_t r = 0; r < n; ++r) m += T[r * 4 + k];
        m /= (double)n;
        for (int64_t r = 0; r < n; ++r) {
            const double t = T[r * 4 + k] - m;
            q += t * t;
        }
        const double sd = sqrt(q / (double)n);
        blob[2 * BV_NFEAT + k] = (float)m;
        blob[2 * BV_NFEAT + 3 + k] = (float)(sd > 1e-12 ? sd : 1.0);
    }
    // initial parameters: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
    float* P = blob + 2 * BV_NFEAT + 6;
    {
        const Offs o = offsets();
        uint64_t ctr = 0;
        for (int l = 0; l < kLayers; ++l) {
            const float a = 1.0f / sqrtf((float)kIn[l]);
            for (int i = 0; i < kIn[l] * kOutDim[l]; ++i) {
                const double u = (double)(bv_sm64(seed ^ 0x6d6c7077ull, ctr++) >> 11) * (1.0 / 9007199254740992.0);
                P[o.w[l] + i] = (float)((2.0 * u - 1.0) * a);
            }
            for (int i = 0; i < kOutDim[l]; ++i) P[o.b[l] + i] = 0.0f;
        }
    }
    std::vector<float> xs, ts;
    standardise_rows(blob, X, n, xs);
    standardise_targets(blob, T, n, ts);
    const int B = (int)std::min<int64_t>(batch, n);
    MLPWork w;
    BV_TRY(w.alloc(B));
    struct Moments {  // Adam's first and second moment estimates, freed on every return path
        float *m1 = nullptr, *m2 = nullptr;
        ~Moments() {
            cudaFree(m1);
            cudaFree(m2);
        }
    } mom;
    BV_CUDA(cudaMalloc(&mom.m1, sizeof(float) * BV_MLP_NPARAM));
    BV_CUDA(cudaMalloc(&mom.m2, sizeof(float) * BV_MLP_NPARAM));
    BV_CUDA(cudaMemset(mom.m1, 0, sizeof(float) * BV_MLP_NPARAM));
    BV_CUDA(cudaMemset(mom.m2, 0, sizeof(float) * BV_MLP_NPARAM));
    BV_CUDA(cudaMemcpy(w.P, P, sizeof(float) * BV_MLP_NPARAM, cudaMemcpyHostToDevice));
    std::vector<int64_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::vector<float> bx((size_t)B * BV_NFEAT), bt((size_t)B * 4), lrow(B);
    int64_t step = 0;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = n - 1; i >= 1; --i) {  // seeded Fisher-Yates shuffle per epoch
            const uint64_t r = bv_sm64(seed + 1000003ull * (uint64_t)(ep + 1), (uint64_t)i);
            const int64_t j = (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(i + 1)) >> 64);
            std::swap(order[i], order[j]);
        }
        double lsum = 0.0;
        int64_t nb_ep = 0;
        for (int64_t r0 = 0; r0 + B <= n; r0 += B) {
            for (int q = 0; q < B; ++q) {
                memcpy(&bx[(size_t)q * BV_NFEAT], &xs[(size_t)order[r0 + q] * BV_NFEAT], sizeof(float) * BV_NFEAT);
                memcpy(&bt[(size_t)q * 4], &ts[(size_t)order[r0 + q] * 4], sizeof(float) * 4);
            }
            BV_CUDA(cudaMemcpy(w.X, bx.data(), sizeof(float) * B * BV_NFEAT, cudaMemcpyHostToDevice));
            BV_CUDA(cudaMemcpy(w.T, bt.data(), sizeof(float) * B * 4, cudaMemcpyHostToDevice));
            BV_CUDA(forward(w, B));
            BV_CUDA(backward(w, B));
            ++step;
            const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
            k_adam<<<nb(BV_MLP_NPARAM), 256>>>(w.P, w.G, mom.m1, mom.m2, BV_MLP_NPARAM, lr, b1, b2, eps, c1, c2);
            BV_CUDA(cudaGetLastError());
            BV_CUDA(cudaMemcpy(lrow.data(), w.loss, sizeof(float) * B, cudaMemcpyDeviceToHost));
            for (float v : lrow) lsum += v;
            ++nb_ep;
        }
        if (loss_out) loss_out[ep] = (float)(lsum / std::max<int64_t>(1, nb_ep * B));
    }
    BV_CUDA(cudaMemcpy(P, w.P, sizeof(float) * BV_MLP_NPARAM, cudaMemcpyDeviceToHost));
    return BV_OK;
}

// ------------------------------------------------------------------------------------
// warm start
// ------------------------------------------------------------------------------------
extern "C" int bv_warmstart_load(bv_ctx* c, const char* path) {
    if (!c || !path) return BV_EINVAL;
    FILE* f = fopen(path, "rb");
    if (!f) return BV_EINVAL;
    char hdr[16];
    int ok = fread(hdr, 1, 16, f) == 16 && memcmp(hdr, "BVWS", 4) == 0;
    int32_t ver = 0, cnt = 0;
    if (ok) {
        memcpy(&ver, hdr + 4, 4);
        memcpy(&cnt, hdr + 8, 4);
        ok = ver == 1 && cnt == BV_MLP_BLOB;
    }
    std::vector<float> w(BV_MLP_BLOB);
    if (ok) ok = fread(w.data(), sizeof(float), BV_MLP_BLOB, f) == (size_t)BV_MLP_BLOB;
    fclose(f);
    if (!ok) return BV_EINVAL;
    c->mlp_w = std::move(w);
    c->have_mlp = true;
    return BV_OK;
}

// The smoothness class of the network's three-way head: 1/2, 3/2 or 5/2 (arg-max logit).
static double nu_of_logits(const float* lg) {
    int c = 0;
    for (int j = 1; j < 3; ++j)
        if (lg[j] > lg[c]) c = j;
    return 0.5 + (double)c;
}

extern "C" int bv_warmstart_predict_multi(bv_ctx* c, const bv_theta* in, bv_theta* out) {
    if (!c || !in || !out) return BV_EINVAL;
    if (!c->have_mlp) return BV_ESTATE;
    if (c->ndata < 1) return BV_ESTATE;
    const int nd = c->ndata;
    std::vector<float> feat((size_t)nd * BV_NFEAT), o((size_t)nd * kOut);
    BV_TRY(bv_features(c, 10000, 0, feat.data()));
    BV_TRY(bv_mlp_forward(c->mlp_w.data(), feat.data(), nd, o.data()));
    const float* ym = c->mlp_w.data() + 2 * BV_NFEAT;
    const float* ys = ym + 3;
    for (int k = 0; k < nd; ++k) {
        double lt[3];
        for (int j = 0; j < 3; ++j) lt[j] = (double)(o[(size_t)k * kOut + j] * ys[j] + ym[j]);
        out[k] = in[k];
        out[k].sigma2 = exp(lt[0]);
        const double beta = exp(lt[1]);
        const double f = beta / in[k].range[0];
        for (int j = 0; j < 3; ++j) out[k].range[j] = in[k].aniso ? in[k].range[j] * f : beta;
        out[k].nugget = exp(lt[2]);
        if (!(in[k].nu > 0.0)) out[k].nu = nu_of_logits(&o[(size_t)k * kOut + 3]);
    }
    return BV_OK;
}

extern "C" int bv_warmstart_predict(bv_ctx* c, const bv_theta* in, bv_theta* out) {
    if (!c || !in || !out) return BV_EINVAL;
    if (!c->have_mlp) return BV_ESTATE;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    float feat[BV_NFEAT];
    BV_TRY(bv_features(c, 10000, 0, feat));
    float o[kOut];
    BV_TRY(bv_mlp_forward(c->mlp_w.data(), feat, 1, o));
    const float* ym = c->mlp_w.data() + 2 * BV_NFEAT;
    const float* ys = ym + 3;
    double lt[3];
    for (int k = 0; k < 3; ++k) lt[k] = (double)(o[k] * ys[k] + ym[k]);
    *out = *in;
    out->sigma2 = exp(lt[0]);
    const double beta = exp(lt[1]);
    const double f = beta / in->range[0];
    for (int k = 0; k < 3; ++k) out->range[k] = in->aniso ? in->range[k] * f : beta;
    out->nugget = exp(lt[2]);
    if (!(in->nu > 0.0)) out->nu = nu_of_logits(o + 3);
    return BV_OK;
}
