// bv_noalloc.cu -- bv_loglik_noalloc: the FP64 block-Vecchia log-likelihood for callers
// that cannot allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is not available or not allowed --
// inside a host callback or another library's stream-ordered section, under a memory
// manager that owns every device allocation (a framework's caching allocator, an
// embedded runtime with a fixed memory budget), or in a real-time loop where an
// allocation's implicit synchronisation is unacceptable.  Such a caller already holds
// its inputs and outputs on the device; this entry point only launches kernels.
//
// The per-block partial results and three status words live in one file-scope device
// array (g_na_scratch, BV_NOALLOC_MAX_BLOCKS + 32 doubles, about 8 MiB), which every GPU
// that loads the library keeps until the process exits.  Its device address is looked
// up once per device with cudaGetSymbolAddress on the first call made with that device
// current (host code may not use the array's name as a device pointer).
//
// Rules for callers:
//   - Make the first call on each device outside any CUDA stream capture: that call looks
//     up the array's device address.
//   - Every call returns only after its stream has drained: it reads the largest block
//     size and a structure check back to the host before the likelihood kernel runs, and
//     the failure word after it.
//   - All calls share the array: two calls whose kernels overlap on the GPU (different
//     streams, or concurrent host threads) race on it and give wrong results.  Order
//     them on one stream or synchronise between them.
//   - The status words are reset at the start of every call; the per-block entries are
//     all rewritten, so nothing from a previous call leaks into the result.
//   - The caller's structure is checked on the device before any point is read: the
//     pointer arrays must start at 0 and never decrease, the blocks must cover at most n
//     points, and every point and neighbour index must lie in [0, n); a violation
//     returns BV_EINVAL (an out-of-range index is recorded and never dereferenced).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "bv_device.cuh"
#include "bv_internal.h"

#define BV_NOALLOC_MAX_DEVICES 64

namespace {

constexpr double kLog2PiNA = 1.8378770664093454835606594728112;

// slots after the per-block entries
constexpr int64_t kFailSlot = BV_NOALLOC_MAX_BLOCKS;
constexpr int64_t kMaxNSlot = BV_NOALLOC_MAX_BLOCKS + 1;
constexpr int64_t kBadSlot = BV_NOALLOC_MAX_BLOCKS + 2;   // nonzero: the structure is malformed

static __device__ __align__(256) double g_na_scratch[BV_NOALLOC_MAX_BLOCKS + 32];

std::mutex g_na_mu;
double* g_na_ptr[BV_NOALLOC_MAX_DEVICES] = {nullptr};

__device__ __forceinline__ int na_pk(int r, int c) { return (r * (r + 1) >> 1) + c; }

__device__ __forceinline__ void na_tri(int f, int& r, int& c) {
    int rr = (int)((sqrtf(8.0f * (float)f + 1.0f) - 1.0f) * 0.5f);
    if (((rr + 1) * (rr + 2) >> 1) <= f) ++rr;
    if ((rr * (rr + 1) >> 1) > f) --rr;
    r = rr;
    c = f - (rr * (rr + 1) >> 1);
}

__device__ __forceinline__ double na_matern(const DevTheta& th, double x) {
    if (th.nu_code == NU_GENERAL) return th.sigma2 * matern_gen_corr(th, x);
    const double e = exp(-x);
    if (th.nu_code == NU_HALF) return th.sigma2 * e;
    if (th.nu_code == NU_3HALF) return th.sigma2 * ((1.0 + x) * e);
    return th.sigma2 * ((1.0 + x * (1.0 + x * (1.0 / 3.0))) * e);
}

__global__ void k_na_init(double* s) {
    reinterpret_cast<unsigned long long*>(s)[kFailSlot] = ~0ull;
    reinterpret_cast<unsigned long long*>(s)[kMaxNSlot] = 0ull;
    reinterpret_cast<unsigned long long*>(s)[kBadSlot] = 0ull;
}

// Largest augmented size m_i + b_i, and the structure check of the pointer arrays
// (both start at 0, neither decreases, the blocks cover at most n points).
__global__ void k_na_maxn(const int64_t* bptr, const int64_t* nptr, int64_t bc, int64_t n, double* s) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= bc) return;
    unsigned long long* w = reinterpret_cast<unsigned long long*>(s);
    const int64_t b = bptr[i + 1] - bptr[i], m = nptr[i + 1] - nptr[i];
    bool bad = b < 0 || m < 0;
    if (i == 0) bad = bad || bptr[0] != 0 || nptr[0] != 0;
    if (i == bc - 1) bad = bad || bptr[bc] > n;
    if (bad) {
        atomicOr(w + kBadSlot, 1ull);
        return;
    }
    atomicMax(w + kMaxNSlot, (unsigned long long)(b + m));
}

// Same fused algorithm as the library's FP64 shared-memory kernel (augmented Cholesky
// of [[Sigma^con, Sigma^cross, y_NN], [., Sigma^lk, y_B], [., ., *]]), with theta passed by
// value, blocks taken in index order and the per-block results written to the scratch.
template <int NT>
__global__ void __launch_bounds__(NT) k_na_ll(const double* __restrict__ locs, int64_t n_tot, int d,
                                              const double* __restrict__ y, const int64_t* __restrict__ bptr,
                                              const int32_t* __restrict__ pidx, const int64_t* __restrict__ nptr,
                                              const int32_t* __restrict__ nidx, int64_t bc, DevTheta th,
                                              double* s) {
    extern __shared__ __align__(16) unsigned char na_sm[];
    double* sm = reinterpret_cast<double*>(na_sm);
    __shared__ double red[NT / 32];
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int64_t blk = blockIdx.x; blk < bc; blk += gridDim.x) {
        const int64_t b0 = bptr[blk], n0 = nptr[blk];
        const int b = (int)(bptr[blk + 1] - b0), m = (int)(nptr[blk + 1] - n0);
        const int N = m + b, R = N + 1;
        double* A = sm;
        double* col0 = A + ((R * (R + 1)) >> 1);
        double* col1 = col0 + R;
        double* px = col1 + R;
        for (int t = tid; t < N; t += NT) {
            const int g = t < m ? nidx[n0 + t] : pidx[b0 + (t - m)];
            if (g < 0 || (int64_t)g >= n_tot) {  // recorded, never dereferenced
                atomicOr(reinterpret_cast<unsigned long long*>(s) + kBadSlot, 1ull);
                for (int k = 0; k < d; ++k) px[k * N + t] = 0.0;
                A[na_pk(N, t)] = 0.0;
                continue;
            }
            for (int k = 0; k < d; ++k) px[k * N + t] = locs[(int64_t)k * n_tot + g];
            A[na_pk(N, t)] = y[g];
        }
        if (tid == 0) {
            A[na_pk(N, N)] = 0.0;
            s_fail = 0;
        }
        __syncthreads();
        const int T = (N * (N + 1)) >> 1;
        for (int f = tid; f < T; f += NT) {
            int r, c;
            na_tri(f, r, c);
            double acc = 0.0;
            for (int k = 0; k < d; ++k) {
                const double t = (px[k * N + r] - px[k * N + c]) * inv_range_k(th, k);
                acc = fma(t, t, acc);
            }
            double v = na_matern(th, sqrt(acc));
            if (r == c) v += th.nugget;
            A[f] = v;
        }
        __syncthreads();
        if (warp == 0) {
            const double p = A[0];
            if (bad_pivot(p) && lane == 0) s_fail = 1;
            const double rs = rsqrt(p);
            for (int j = 1 + lane; j <= N; j += 32) {
                const double v = A[na_pk(j, 0)] * rs;
                A[na_pk(j, 0)] = v;
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
                for (int j = kk + lane; j <= N; j += 32) A[na_pk(j, kk)] = fma(-cur[j], ck, A[na_pk(j, kk)]);
                __syncwarp();
                const double p = A[na_pk(kk, kk)];
                if (bad_pivot(p) && lane == 0) s_fail = 1;
                const double rs = rsqrt(p);
                for (int j = kk + 1 + lane; j <= N; j += 32) {
                    const double v = A[na_pk(j, kk)] * rs;
                    A[na_pk(j, kk)] = v;
                    nxt[j] = v;
                }
            }
            const int S = N - kk;
            const int TS = (S * (S + 1)) >> 1;
            for (int f = tid; f < TS; f += NT) {
                int r, c;
                na_tri(f, r, c);
                const int j = kk + 1 + r, i = kk + 1 + c;
                A[na_pk(j, i)] = fma(-cur[j], cur[i], A[na_pk(j, i)]);
            }
            __syncthreads();
        }
        double part = 0.0;
        for (int k = m + tid; k < N; k += NT) {
            const double z = A[na_pk(N, k)];
            part += z * z + log(A[na_pk(k, k)]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (tid == 0) {
            double sum = 0.0;
            for (int i = 0; i < NT / 32; ++i) sum += red[i];
            double ell = -0.5 * (sum + (double)b * kLog2PiNA);
            if (s_fail || !(ell == ell)) {
                ell = -INFINITY;
                atomicMin(reinterpret_cast<unsigned long long*>(s) + kFailSlot, (unsigned long long)blk);
            }
            s[blk] = ell;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_na_reduce(const double* s, int64_t bc, double* out) {
    __shared__ double ss[256], sc[256];
    const int tid = threadIdx.x;
    double S = 0.0, C = 0.0;
    for (int64_t i = tid; i < bc; i += 256) {
        const double x = s[i];
        const double t = S + x;
        if (fabs(S) >= fabs(x)) C += (S - t) + x;
        else C += (x - t) + S;
        S = t;
    }
    ss[tid] = S;
    sc[tid] = C;
    __syncthreads();
    if (tid == 0) {
        double T = 0.0, K = 0.0;
        for (int i = 0; i < 256; ++i) {
            const double x = ss[i];
            const double t = T + x;
            if (fabs(T) >= fabs(x)) K += (T - t) + x;
            else K += (x - t) + T;
            T = t;
            K += sc[i];
        }
        double r = T + K;
        if (!(r == r)) r = -INFINITY;
        out[0] = r;
    }
}

constexpr int kNT = 128;

size_t na_smem(int nmax, int d) {
    const size_t R = (size_t)nmax + 1;
    return ((sizeof(double) * (R * (R + 1) / 2 + 2 * R + (size_t)d * nmax)) + 15) & ~(size_t)15;
}

}  // namespace

// Largest augmented size m_i + b_i the entry point accepts (shared-memory kernel):
// 235 for d = 1, 234 for d = 2, 233 for d = 3.
static int na_max_n(int32_t d) {
    if (d < 1 || d > 3) return 0;
    int n = 8;
    while (na_smem(n + 1, d) <= (size_t)(227 * 1024 - 2048)) ++n;
    return n;
}

extern "C" int bv_loglik_noalloc(const bv_theta* theta, const double* d_locs, const double* d_y, int64_t n,
                                 int32_t d, int64_t bc, const int64_t* d_block_ptr, const int32_t* d_point_idx,
                                 const int64_t* d_nn_ptr, const int32_t* d_nn_idx, double* d_out_loglik,
                                 double* d_out_per_block, void* cuda_stream) {
    if (!theta || !d_locs || !d_y || !d_block_ptr || !d_point_idx || !d_nn_ptr || !d_out_loglik) return BV_EINVAL;
    if (d < 1 || d > 3 || n <= 0 || n >= (int64_t)INT32_MAX) return BV_EINVAL;
    if (bc <= 0 || bc > BV_NOALLOC_MAX_BLOCKS) return BV_EINVAL;  // scratch holds at most this many blocks
    DevTheta th;
    BV_TRY(bv_theta_to_dev(theta, d, &th));
    int dev = 0;
    BV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= BV_NOALLOC_MAX_DEVICES) return BV_EINVAL;
    double* s = nullptr;
    {
        // once per device, with that device current: resolve the array's device address
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            BV_CUDA(cudaGetSymbolAddress(&p, g_na_scratch));
            g_na_ptr[dev] = static_cast<double*>(p);
        }
        s = g_na_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int nsm = 0;
    BV_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    k_na_init<<<1, 1, 0, st>>>(s);
    BV_CUDA(cudaGetLastError());
    k_na_maxn<<<(unsigned)((bc + 255) / 256), 256, 0, st>>>(d_block_ptr, d_nn_ptr, bc, n, s);
    BV_CUDA(cudaGetLastError());
    unsigned long long chk[2] = {0, 0};  // largest m_i + b_i, structure flag
    BV_CUDA(cudaMemcpyAsync(chk, reinterpret_cast<unsigned long long*>(s) + kMaxNSlot, sizeof(chk),
                            cudaMemcpyDeviceToHost, st));
    BV_CUDA(cudaStreamSynchronize(st));
    const unsigned long long maxn = chk[0];
    if (chk[1] != 0 || maxn == 0 || maxn > (unsigned long long)na_max_n(d)) return BV_EINVAL;
    const size_t smem = na_smem((int)maxn, d);
    BV_CUDA(cudaFuncSetAttribute(k_na_ll<kNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    BV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_na_ll<kNT>, kNT, smem));
    if (occ < 1) return BV_EINTERNAL;
    const int64_t grid = bc < (int64_t)occ * nsm ? bc : (int64_t)occ * nsm;
    k_na_ll<kNT><<<(unsigned)grid, kNT, smem, st>>>(d_locs, n, d, d_y, d_block_ptr, d_point_idx, d_nn_ptr,
                                                     d_nn_idx, bc, th, s);
    BV_CUDA(cudaGetLastError());
    k_na_reduce<<<1, 256, 0, st>>>(s, bc, d_out_loglik);
    BV_CUDA(cudaGetLastError());
    if (d_out_per_block)
        BV_CUDA(cudaMemcpyAsync(d_out_per_block, s, sizeof(double) * bc, cudaMemcpyDeviceToDevice, st));
    unsigned long long fin[3] = {0, 0, 0};  // failure word, largest size, structure flag
    BV_CUDA(cudaMemcpyAsync(fin, reinterpret_cast<unsigned long long*>(s) + kFailSlot, sizeof(fin),
                            cudaMemcpyDeviceToHost, st));
    BV_CUDA(cudaStreamSynchronize(st));
    if (fin[2] != 0) return BV_EINVAL;  // a point or neighbour index outside [0, n)
    return fin[0] != ~0ull ? BV_ENOTPD : BV_OK;
}
