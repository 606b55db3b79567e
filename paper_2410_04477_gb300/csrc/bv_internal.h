// bv_internal.h -- shared declarations of the CUDA implementation of include/bv.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bv.h"

// ------------------------------------------------------------------------------------
// Error handling
// ------------------------------------------------------------------------------------
void bv_record_cuda_error(cudaError_t e, const char* expr, const char* file, int line);

#define BV_CUDA(expr)                                                        \
    do {                                                                     \
        cudaError_t bv_e_ = (expr);                                          \
        if (bv_e_ != cudaSuccess) {                                          \
            bv_record_cuda_error(bv_e_, #expr, __FILE__, __LINE__);          \
            return bv_e_ == cudaErrorMemoryAllocation ? BV_ENOMEM : BV_ECUDA; \
        }                                                                    \
    } while (0)

// Device allocation of an evaluation's buffers (the plan, the evaluation layout).  Test
// support: while the environment variable BV_FAULT_ALLOC is set to a non-zero value it
// fails as the runtime does when device memory is exhausted (cudaErrorMemoryAllocation)
// without calling the runtime, so that a caller can exercise the BV_ENOMEM path, and the
// context's recovery from it, with no real exhaustion of the device.
cudaError_t bv_plan_malloc(void** p, size_t bytes);
template <class T>
inline cudaError_t bv_plan_malloc(T** p, size_t bytes) {
    return bv_plan_malloc(reinterpret_cast<void**>(p), bytes);
}

#define BV_TRY(expr)                    \
    do {                                \
        int bv_s_ = (expr);             \
        if (bv_s_ != BV_OK) return bv_s_; \
    } while (0)

// ------------------------------------------------------------------------------------
// Device-side parameters
// ------------------------------------------------------------------------------------

// Matern smoothness codes: the closed forms of Eq. 5 at nu = 1/2, 3/2, 5/2, and any other
// nu through K_nu (NU_GENERAL).
enum { NU_HALF = 0, NU_3HALF = 1, NU_5HALF = 2, NU_GENERAL = 3 };

// Largest smoothness accepted for the general form.
#define BV_NU_MAX 20.0

// theta prepared for the kernels: reciprocal ranges per axis (isotropic: all equal).  For
// NU_GENERAL the smoothness is split as nu = nrec + mu, |mu| <= 1/2, with the constants
// of Temme's series at mu (gam1 = (1/G(1-mu) - 1/G(1+mu)) / (2 mu), gam2 = (1/G(1-mu) +
// 1/G(1+mu)) / 2, gampl = 1/G(1+mu), gammi = 1/G(1-mu)) and lognorm = log(2^{1-nu}/G(nu)).
struct DevTheta {
    double sigma2, nugget;
    double inv_range[3];
    int32_t nu_code;
    int32_t nrec;
    double nu, mu, gam1, gam2, gampl, gammi, lognorm;
    // FP32 copies for the mixed-precision kernels (converted once on the host), and the
    // part of the diagonal sigma^2 + tau^2 that its FP32 value sigma2_f + nugget_f misses
    // (added to every pivot, so that the FP32 factor is that of the exact diagonal)
    float sigma2_f, nugget_f, inv_range_f[3];
    float diag_lo_f;
};

// Constants of the table-driven FP64 exponential (Tang, "Table-driven implementation of
// the exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989):
// e^{-x} = 2^{n/256} e^{r},  n = round(-x 256/ln2),  r = -x - n (L1 + L2),
// L1 + L2 = ln2/256, 2^{n/256} = 2^{floor(n/256)} tab[n mod 256].  Filled on the host in
// long double.
#define BV_EXP_TAB 256
// work counters per group of launches (at most 15 shared-memory bins and one global-memory
// bin each): FP64 bins, mixed bins, the mixed check's FP64 sample bins and its FP64 redo bins
#define BV_WCTR_PER_PREC 32
#define BV_WCTR_GROUPS 4
struct ExpConsts {
    double tab[BV_EXP_TAB];   // 2^{j/256}, j = 0..255
    double k;                 // 256 / ln 2
    double l1, l2;            // ln2/256 split: l1 has its low 21 bits zero so n*l1 is exact
    // FP32 version of the same method with 32 table steps (mixed-precision kernels):
    // t32[j] + t32[32 + j] = 2^{-j/32} as two floats, k32 = 32 / ln 2, l1_32 + l2_32 =
    // ln2/32 with l1_32's low 12 bits zero
    float t32[64];
    float k32, l1_32, l2_32;
};
void bv_exp_consts(ExpConsts* out);

// Everything a log-likelihood kernel reads.  Locations are SoA: coordinate k of point j
// is locs[k * n_tot + j].  Block p has points pidx[bptr[p] .. bptr[p+1]) and
// conditioning points nidx[nptr[p] .. nptr[p+1]).
struct LLArgs {
    const double* locs;
    int64_t n_tot;
    int32_t d;
    const double* y;
    const int64_t* bptr;
    const int32_t* pidx;
    const int64_t* nptr;
    const int32_t* nidx;
    const double* cent;      // block centroids, row-major [nblk x d]
    const int32_t* bds;      // dataset of every block
    const DevTheta* theta;   // per dataset
    const int32_t* work;     // block ids of this launch, largest first
    int32_t nwork;
    const int* nwork_dev;    // or null; else the launch's work count is min(*nwork_dev, nwork)
    int* ctr;                // work counter of this launch (zeroed before it), or null: grid stride
    int gen;                 // host side: launch the general-smoothness instantiation
    int* fb;                 // mixed precision: [0] count, [1..] blocks to redo in FP64 (or null)
    int dyn;                 // global-memory kernel: take the work list and count from fb
    const double* gtab;      // per dataset: general-nu Matern table (GTAB_SIZE doubles)
    double* ell_blk;         // per-block conditional log-likelihood (output)
    double* u_blk;           // per-block quadratic form u_i = v_i^T v_i (output)
    float* ind_blk;          // mixed kernels, or null: per-block sum over all pivots of
                             // (sigma^2 + tau^2) / pivot, the conditioning indicator
    unsigned long long* fail;  // min over failing block ids (ULLONG_MAX = none)
    double* ws;              // global workspace (large-block path)
    int64_t ws_stride;       // doubles per workspace slot
    ExpConsts ex;            // FP64 exponential constants (and the FP32 table of exp_neg32)
};

// Per-size-bin launch plan entry.
struct BinPlan {
    int kind;            // 0: FP64 shared-memory, 1: mixed (CTA per block), 2: large (global),
                         // 3: mixed (warp per block), 4: FP64 (warp per block),
                         // 5: mixed with tensor-core updates (CTA per block),
                         // 6: FP64 shared-memory with two-column steps
    int nmax;            // largest augmented size N = m + b in the bin
    int threads;         // CTA size (autotuned)
    int grid;            // CTAs launched
    size_t smem;         // dynamic shared memory bytes
    int32_t* d_work;     // device block ids (largest N first)
    int32_t nwork;
    int* d_ctr;          // this bin's work counter (a slot of the context's counter array)
    int slot = -1;       // mixed check's redo launches: index of the bin's device count
    std::vector<int32_t> h_work;
};

// Tensor-core mixed-precision kernel (bv_mixed_tc.cu), kind 5 of a bin plan.
size_t bv_tc_smem_bytes(int nmax);
int bv_tc_occupancy(int threads, size_t smem);
cudaError_t bv_tc_launch(int threads, int grid, size_t smem, const LLArgs& a, cudaStream_t s);

// Launchers (bv_loglik.cu).
int bv_smem_max_n(int kind, int d);
size_t bv_smem_bytes(int kind, int nmax, int d, int threads);
int bv_max_threads_for(int kind);
int bv_occupancy(int kind, int threads, size_t smem);
// Largest augmented size the global-memory path accepts (packed indices stay in int32).
#define BV_LARGE_MAX_N 30000
cudaError_t bv_launch_bin(const BinPlan& bp, const LLArgs& a, cudaStream_t s);
// Per-dataset sums of ell_i and u_i in two deterministic stages; part holds
// ndata x maxchunks partials of 4 doubles; maxchunks = bv_reduce_chunks(largest dataset).
int bv_reduce_chunks(int64_t max_blocks_per_dataset);
cudaError_t bv_launch_reduce(const double* ell_blk, const double* u_blk, const int64_t* ds_blk_off,
                             int32_t ndata, int32_t maxchunks, void* part, double* out, double* out_quad,
                             cudaStream_t s);
cudaError_t bv_launch_fail_reset(unsigned long long* fail, cudaStream_t s);
// failure flag reset plus zeroing of n work counters (start of one evaluation)
cudaError_t bv_launch_eval_reset(unsigned long long* fail, int* ctr, int n, cudaStream_t s);
// FP64 recomputation (global-memory kernel) of the blocks listed in a.fb.
cudaError_t bv_launch_fallback(const LLArgs& a, int grid, cudaStream_t s);
// Mixed-precision error check of every dataset (one CTA each) from the FP64 values of its
// sampled blocks (samp[samp_ptr[ds] .. samp_ptr[ds+1])) and the blocks' conditioning
// indicators: per dataset a flag (0 keep, 1 redo blocks with ind > thr, 2 redo all), the
// threshold and the bound on the relative error of what stays in FP32 (bv_loglik.cu).
cudaError_t bv_launch_mixed_check(double* ell_blk, double* u_blk, const double* ell64, const double* u64,
                                  const float* ind, const int32_t* samp, const int64_t* samp_ptr,
                                  const int64_t* ds_blk_off, int32_t ndata, double tol, int32_t* flag, float* thr,
                                  double* est, cudaStream_t s);
// Queue every block the check sends back on the FP64 redo list of its bin.
cudaError_t bv_launch_mixed_redo_list(const int32_t* bds, int64_t nblk, const int32_t* flag, const float* thr,
                                      const float* ind, const int64_t* samp_ptr, const int64_t* ds_blk_off,
                                      const int32_t* blk_bin, const int64_t* roff, int32_t* redo, int* cnt,
                                      cudaStream_t s);
// Builds every general-nu dataset's Matern table (bv_device.cuh) from the device thetas.
cudaError_t bv_launch_gtab(const DevTheta* theta, int32_t ndata, double* gtab, cudaStream_t s);
#define BV_GTAB_DOUBLES 931  // GTAB_NOCT * GTAB_DEG

// K-means and neighbour search (bv_kmeans.cu, bv_nn.cu).
int bv_kmeans_device(const double* d_locs_soa, int64_t n_tot, int64_t off, int64_t n, int d,
                     int64_t k, uint64_t seed, int iters, int32_t* d_label, double* d_cent,
                     cudaStream_t s);
int bv_kmeans_scales(const double* h_locs_rowmajor, int64_t n, int d, int* s_out, int* q_out);
int bv_centroids_device(const double* d_locs_soa, int64_t n_tot, int64_t off, int64_t n, int d,
                        const int32_t* d_label, int64_t k, int q, double* d_cent,
                        int64_t* d_counts, cudaStream_t s);
int bv_select_neighbors_device(const double* d_locs_soa, int64_t n_tot, int d,
                               const int64_t* d_bptr, const int32_t* d_pidx,
                               const double* d_cent, int64_t blk_begin, int64_t blk_end,
                               const int64_t* h_nptr, int64_t* d_nptr, int32_t* d_nidx,
                               double amax, cudaStream_t s);

int bv_select_pred_neighbors_device(const double* d_locs, int64_t n_tot, int d, const double* d_qcent, int64_t nq,
                                    const int64_t* d_nptr, int32_t* d_nidx, double amax, cudaStream_t s);

// Block-Vecchia sampler (bv_sim.cu).
int bv_simulate_device(bv_ctx* ctx, const DevTheta& th, const double* d_z, double* d_y);

// SplitMix64 counter-form draws (Steele, Lea and Flood 2014), host and device.
__host__ __device__ inline uint64_t bv_sm64(uint64_t stream, uint64_t counter) {
    uint64_t z = stream + (counter + 1ull) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
#define BV_STREAM_KPP(seed) ((seed) ^ 0x6b6d65616e732b2bull)
#define BV_STREAM_ZETA(seed) ((seed) ^ 0x7a6574615f6f7264ull)
#define BV_STREAM_CSIM(seed) ((seed) ^ 0x636f6e6473696d5full)

// ------------------------------------------------------------------------------------
// The context
// ------------------------------------------------------------------------------------
struct bv_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    size_t smem_optin = 0;

    // data
    int32_t d = 0;
    int32_t ndata = 0;
    int64_t n_tot = 0;
    std::vector<int64_t> pt_off;     // ndata + 1
    std::vector<double> h_locs;      // row-major n_tot x d (host copy for planning)
    double* d_locs = nullptr;        // SoA d x n_tot
    double* d_y = nullptr;
    bool have_y = false;

    // blocks (all datasets, dataset after dataset)
    int64_t nblk = 0;
    std::vector<int64_t> ds_blk_off;  // ndata + 1
    std::vector<int64_t> h_bptr;
    std::vector<int32_t> h_pidx;
    std::vector<int32_t> h_bds;
    int64_t* d_bptr = nullptr;
    int32_t* d_pidx = nullptr;
    double* d_cent = nullptr;
    int32_t* d_bds = nullptr;
    int64_t* d_ds_blk_off = nullptr;
    bool have_blocks = false;

    // evaluation layout: the likelihood kernels read points in Hilbert order (per
    // dataset) so that a block's neighbours lie close together in memory; built at
    // planning time from the structures above (which keep the original numbering)
    bool have_layout = false;
    int32_t* d_inv = nullptr;         // internal position -> original point
    double* d_locs_int = nullptr;     // SoA d x n_tot, internal order
    double* d_y_int = nullptr;        // internal order
    int32_t* d_pidx_int = nullptr;    // block members, internal positions
    int32_t* d_nidx_int = nullptr;    // conditioning points, internal positions

    // neighbours
    std::vector<int64_t> h_nptr;
    int64_t* d_nptr = nullptr;
    int32_t* d_nidx = nullptr;
    bool have_nn = false;

    // evaluation state
    double* d_ell_blk = nullptr;
    double* d_u_blk = nullptr;        // per-block quadratic forms
    double* d_red_part = nullptr;     // reduction partials (ndata x red_chunks x 4)
    int* d_fb = nullptr;              // mixed-precision FP64 fallback list: [0] count, [1..] blocks
    int* h_fb = nullptr;              // pinned copy of the count
    double* d_fb_ws = nullptr;        // FP64 workspace slots for the fallback pass
    float* d_ind = nullptr;           // mixed: per-block conditioning indicator (LLArgs::ind_blk)
    double mixed_tol = 1e-6;          // mixed: bound enforced by the FP64 check (0: no check)
    int64_t fb_stride = 0;
    int fb_slots = 0;
    int32_t red_chunks = 1;
    double* d_quad = nullptr;         // ndata: sum of the quadratic forms
    double* h_quad = nullptr;         // pinned, ndata
    unsigned long long* d_fail = nullptr;
    int* d_wctr = nullptr;  // per-bin work counters, BV_WCTR_PER_PREC per precision
    double* d_out = nullptr;          // ndata
    double* h_out = nullptr;          // pinned, ndata
    DevTheta* d_theta = nullptr;      // ndata
    double* d_gtab = nullptr;         // ndata x BV_GTAB_DOUBLES general-nu Matern tables
    std::vector<DevTheta> h_theta;    // ndata (pageable: copies are staged by the driver)
    unsigned long long* h_fail = nullptr;  // pinned
    double* d_ws = nullptr;
    int64_t ws_stride = 0;
    int ws_slots = 0;

    // mixed precision's error check (built with the mixed plan): FP64 bins over all blocks
    // (the sampled blocks' static lists and the redo lists filled per evaluation), the
    // sample CSR by dataset, per-block FP64 bin, per-dataset flags and error estimates
    struct MixedCheck {
        std::vector<BinPlan> sbins;        // FP64 launches of the sampled blocks (own d_work)
        std::vector<BinPlan> rbins;        // FP64 launches of the redo lists (d_work inside d_redo)
        int32_t* d_samp = nullptr;         // sampled blocks, dataset after dataset
        int64_t* d_samp_ptr = nullptr;     // ndata + 1
        int32_t* d_blk_bin = nullptr;      // FP64 bin of every block
        int64_t* d_roff = nullptr;         // per bin: offset of its redo segment
        int32_t* d_redo = nullptr;         // nblk
        int* d_cnt = nullptr;              // per bin: blocks queued for redo this evaluation
        double* d_ell = nullptr;           // FP64 ell_i of the sampled blocks (by block id)
        double* d_u = nullptr;
        int32_t* d_flag = nullptr;         // per dataset: 0 kept, 1 worst blocks redone, 2 all redone
        float* d_thr = nullptr;            // per dataset: indicator threshold of flag 1
        double* d_est = nullptr;           // per dataset: estimated bound of the FP32 part's relative error
        int64_t nsamp = 0;
    } chk;

    // per precision: plan, graph
    std::vector<BinPlan> plan[2];
    bool plan_valid[2] = {false, false};
    bool tuned[2] = {false, false};
    // per precision: the size-bin launches of an evaluation run one after another in
    // descending order of work instead of as parallel branches (chosen by timing both)
    bool bin_serial[2] = {false, false};
    // graphs of one evaluation: [0] FP64, [1] mixed with its check (captured at tolerance
    // graph_tol), [2] mixed without the check
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
    // per graph slot: launch the evaluation's kernels directly instead of the graph
    // (decided once per plan by timing both), and whether that was decided
    bool eval_direct[3] = {false, false, false};
    bool eval_direct_known[3] = {false, false, false};
    double graph_tol = 0.0;
    bool graph_gen[3] = {false, false, false};  // whether each graph holds the general-nu kernels
    bool cur_gen = false;                 // whether the current theta needs them
    std::vector<cudaStream_t> side;   // fork/join streams of the captured graph
    std::vector<cudaEvent_t> side_ev; // [0] fork, [1..] joins
    double* graph_out[2] = {nullptr, nullptr};

    // warm start
    std::vector<float> mlp_w;
    bool have_mlp = false;

    // prediction (bv_pred.cu)
    struct PredState* pred = nullptr;
};

// prediction state teardown (bv_pred.cu); also called when the observations change
void bv_pred_free(bv_ctx* ctx);

// Hilbert order of the points of one dataset (bv_order.cu): global indices.
void bv_hilbert_order(const double* locs_rowmajor, int64_t off, int64_t n, int d, std::vector<int32_t>& order);

// helpers in bv_api.cu
int bv_theta_to_dev(const bv_theta* t, int d, DevTheta* out);
int bv_ensure_plan(bv_ctx* ctx, int precision);
int bv_refresh_layout_y(bv_ctx* ctx);
void bv_invalidate_plans(bv_ctx* ctx);
int bv_enqueue_loglik(bv_ctx* ctx, int precision, double* d_out, bool with_theta_copy);
