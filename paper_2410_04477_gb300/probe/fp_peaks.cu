// fp_peaks.cu -- arithmetic-pipe throughput probe (FP64 FMA, FP32 FMA) used to derive the
// ALU rooflines of the log-likelihood kernels.  Each thread runs 8 independent FMA chains;
// `active_lanes` lanes per warp do the work (1 = single lane, 32 = full warp), so the probe
// also shows whether a partially active warp instruction costs a full warp slot.
#include <cuda_runtime.h>
#include <stdint.h>

template <typename T>
__global__ void k_fma(T* out, int iters, int active_lanes, T a, T b) {
    const int lane = threadIdx.x & 31;
    if (lane >= active_lanes) return;
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
      x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-1.2345) out[blockIdx.x] = s;  // keep the chains live
}

// Returns lane-FMA per second (x2 = flop/s) for the given type code (0 = FP64, 1 = FP32).
extern "C" int bvp_fma_rate(int type, int active_lanes, int blocks, int threads, int iters,
                            double* fma_per_s) {
    void* out = nullptr;
    if (cudaMalloc(&out, 8 * (size_t)blocks) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {
        cudaEventRecord(e0);
        if (type == 0)
            k_fma<double><<<blocks, threads>>>((double*)out, iters, active_lanes, 0.999999, 1e-7);
        else
            k_fma<float><<<blocks, threads>>>((float*)out, iters, active_lanes, 0.999999f, 1e-7f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;
    }
    const cudaError_t e = cudaGetLastError();
    cudaFree(out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return 2;
    const double lanes = (double)blocks * (threads / 32) * active_lanes;
    *fma_per_s = lanes * 8.0 * iters / (best * 1e-3);
    return 0;
}
