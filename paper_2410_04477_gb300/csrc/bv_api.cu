// bv_api.cu -- host side of the C ABI in include/bv.h: context, data, preprocessing
// drivers, the size-bin launch planner with its autotuner, and the CUDA-graph launch of
// one log-likelihood evaluation.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "bv_internal.h"

// ------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------
static thread_local std::string g_cuda_err;

void bv_record_cuda_error(cudaError_t e, const char* expr, const char* file, int line) {
    g_cuda_err = std::string(cudaGetErrorString(e)) + " in " + expr + " at " + file + ":" +
                 std::to_string(line);
}

extern "C" const char* bv_last_cuda_error(void) { return g_cuda_err.c_str(); }

extern "C" const char* bv_strerror(int s) {
    switch (s) {
        case BV_OK: return "ok";
        case BV_EINVAL: return "invalid argument";
        case BV_ENOMEM: return "out of memory";
        case BV_ECUDA: return "CUDA error";
        case BV_ENOTPD: return "covariance matrix not positive definite";
        case BV_ETIMEOUT: return "device wait timed out (reserved: no call returns it)";
        case BV_ESTATE: return "call out of order (missing data, blocks or neighbours)";
        case BV_EINTERNAL: return "internal consistency check failed";
        default: return "unknown status";
    }
}

cudaError_t bv_plan_malloc(void** p, size_t bytes) {
    const char* f = getenv("BV_FAULT_ALLOC");
    if (f && *f && strcmp(f, "0") != 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

template <class T>
static void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

static void free_check(bv_ctx* c) {
    auto& k = c->chk;
    for (auto& b : k.sbins) dfree(b.d_work);
    k.sbins.clear();
    k.rbins.clear();  // their lists live inside d_redo
    dfree(k.d_samp);
    dfree(k.d_samp_ptr);
    dfree(k.d_blk_bin);
    dfree(k.d_roff);
    dfree(k.d_redo);
    dfree(k.d_cnt);
    dfree(k.d_ell);
    dfree(k.d_u);
    dfree(k.d_flag);
    dfree(k.d_thr);
    dfree(k.d_est);
    k.nsamp = 0;
}

static void free_plan(bv_ctx* c, int prec) {
    if (prec == BV_MIXED) free_check(c);
    for (auto& b : c->plan[prec]) dfree(b.d_work);
    c->plan[prec].clear();
    c->plan_valid[prec] = false;
    c->tuned[prec] = false;
    for (int slot : {prec, prec == BV_MIXED ? 2 : prec}) {
        if (c->graph[slot]) cudaGraphExecDestroy(c->graph[slot]);
        c->graph[slot] = nullptr;
        c->eval_direct_known[slot] = false;
    }
}

void bv_invalidate_plans(bv_ctx* c) {
    free_plan(c, 0);
    free_plan(c, 1);
}

static void free_layout(bv_ctx* c) {
    dfree(c->d_inv);
    dfree(c->d_locs_int);
    dfree(c->d_y_int);
    dfree(c->d_pidx_int);
    dfree(c->d_nidx_int);
    c->have_layout = false;
}

static void free_neighbors(bv_ctx* c) {
    bv_invalidate_plans(c);
    free_layout(c);
    dfree(c->d_nptr);
    dfree(c->d_nidx);
    c->h_nptr.clear();
    c->have_nn = false;
}

static void free_blocks(bv_ctx* c) {
    free_neighbors(c);
    dfree(c->d_bptr);
    dfree(c->d_pidx);
    dfree(c->d_cent);
    dfree(c->d_bds);
    dfree(c->d_ds_blk_off);
    dfree(c->d_ell_blk);
    dfree(c->d_u_blk);
    dfree(c->d_red_part);
    dfree(c->d_fb);
    dfree(c->d_fb_ws);
    dfree(c->d_ind);
    c->fb_slots = 0;
    c->h_bptr.clear();
    c->h_pidx.clear();
    c->h_bds.clear();
    c->ds_blk_off.clear();
    c->nblk = 0;
    c->have_blocks = false;
}

__global__ void k_gather_soa(const double* __restrict__ src, int64_t n, int d, const int32_t* __restrict__ inv,
                             double* __restrict__ dst) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t g = inv[j];
    for (int k = 0; k < d; ++k) dst[(int64_t)k * n + j] = src[(int64_t)k * n + g];
}

__global__ void k_map_index(const int32_t* __restrict__ idx, int64_t cnt, const int32_t* __restrict__ pos,
                            int32_t* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < cnt) out[i] = pos[idx[i]];
}

__global__ void k_inverse_perm(const int32_t* __restrict__ inv, int64_t n, int32_t* __restrict__ pos) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < n) pos[inv[j]] = (int32_t)j;
}

// The observations in the evaluation layout (after any change of d_y).
static int refresh_layout_y(bv_ctx* c) {
    if (!c->have_layout || !c->d_y) return BV_OK;
    const int64_t n = c->n_tot;
    k_gather_soa<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->d_y, n, 1, c->d_inv, c->d_y_int);
    BV_CUDA(cudaGetLastError());
    return BV_OK;
}

int bv_refresh_layout_y(bv_ctx* c) { return refresh_layout_y(c); }

// Hilbert order of every dataset's points; internal copies of the locations and y and the
// block / neighbour lists mapped to internal positions.  Results do not change: every
// kernel reads the same values, only from other addresses.
static int build_layout(bv_ctx* c) {
    if (c->have_layout) return BV_OK;
    free_layout(c);  // whatever an earlier attempt that failed part-way allocated
    const int64_t n = c->n_tot;
    const int d = c->d;
    std::vector<int32_t> inv;
    inv.reserve(n);
    for (int ds = 0; ds < c->ndata; ++ds) {
        std::vector<int32_t> o;
        bv_hilbert_order(c->h_locs.data(), c->pt_off[ds], c->pt_off[ds + 1] - c->pt_off[ds], d, o);
        inv.insert(inv.end(), o.begin(), o.end());
    }
    struct DevBuf {  // scratch freed on every return path
        int32_t* p = nullptr;
        ~DevBuf() {
            if (p) cudaFree(p);
        }
    } pos;
    BV_CUDA(bv_plan_malloc(&c->d_inv, sizeof(int32_t) * n));
    BV_CUDA(bv_plan_malloc(&pos.p, sizeof(int32_t) * n));
    int32_t* d_pos = pos.p;
    BV_CUDA(bv_plan_malloc(&c->d_locs_int, sizeof(double) * n * d));
    BV_CUDA(bv_plan_malloc(&c->d_y_int, sizeof(double) * n));
    BV_CUDA(bv_plan_malloc(&c->d_pidx_int, sizeof(int32_t) * n));
    const int64_t nn = std::max<int64_t>(c->h_nptr.back(), 1);
    BV_CUDA(bv_plan_malloc(&c->d_nidx_int, sizeof(int32_t) * nn));
    BV_CUDA(cudaMemcpyAsync(c->d_inv, inv.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream));
    const unsigned g = (unsigned)((n + 255) / 256);
    k_inverse_perm<<<g, 256, 0, c->stream>>>(c->d_inv, n, d_pos);
    k_gather_soa<<<g, 256, 0, c->stream>>>(c->d_locs, n, d, c->d_inv, c->d_locs_int);
    k_map_index<<<g, 256, 0, c->stream>>>(c->d_pidx, n, d_pos, c->d_pidx_int);
    if (c->h_nptr.back() > 0)
        k_map_index<<<(unsigned)((c->h_nptr.back() + 255) / 256), 256, 0, c->stream>>>(c->d_nidx, c->h_nptr.back(),
                                                                                     d_pos, c->d_nidx_int);
    BV_CUDA(cudaGetLastError());
    BV_CUDA(cudaStreamSynchronize(c->stream));
    c->have_layout = true;
    return refresh_layout_y(c);
}

static void free_data(bv_ctx* c) {
    bv_pred_free(c);
    free_blocks(c);
    dfree(c->d_locs);
    dfree(c->d_y);
    dfree(c->d_out);
    dfree(c->d_quad);
    if (c->h_quad) cudaFreeHost(c->h_quad);
    c->h_quad = nullptr;
    dfree(c->d_theta);
    dfree(c->d_gtab);
    if (c->h_out) cudaFreeHost(c->h_out);
    c->h_out = nullptr;
    c->h_theta.clear();
    c->h_locs.clear();
    c->pt_off.clear();
    c->n_tot = 0;
    c->ndata = 0;
    c->have_y = false;
}

// ------------------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------------------
extern "C" int bv_create(bv_ctx** out, int device, void* stream) {
    if (!out) return BV_EINVAL;
    *out = nullptr;
    int ndev = 0;
    BV_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return BV_EINVAL;
    BV_CUDA(cudaSetDevice(device));
    bv_ctx* c = new bv_ctx();
    c->device = device;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            bv_record_cuda_error(e, "cudaStreamCreateWithFlags", __FILE__, __LINE__);
            delete c;
            return BV_ECUDA;
        }
        c->own_stream = true;
    }
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_fail, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_wctr, sizeof(int) * BV_WCTR_GROUPS * BV_WCTR_PER_PREC);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_fail, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_fb, sizeof(int));
    if (e == cudaSuccess) *c->h_fb = 0;
    if (e != cudaSuccess) {
        bv_record_cuda_error(e, "bv_create", __FILE__, __LINE__);
        bv_destroy(c);
        return BV_ECUDA;
    }
    c->num_sms = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    *out = c;
    return BV_OK;
}

extern "C" void bv_destroy(bv_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_data(c);
    dfree(c->d_fail);
    dfree(c->d_wctr);
    dfree(c->d_ws);
    for (auto s : c->side) cudaStreamDestroy(s);
    for (auto e : c->side_ev) cudaEventDestroy(e);
    if (c->h_fail) cudaFreeHost(c->h_fail);
    if (c->h_fb) cudaFreeHost(c->h_fb);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// ------------------------------------------------------------------------------------
// data
// ------------------------------------------------------------------------------------
extern "C" int bv_set_datasets(bv_ctx* c, int32_t ndata, const int64_t* n_per, const double* locs,
                               const double* y, int32_t d) {
    if (!c || ndata <= 0 || !n_per || !locs || d < 1 || d > 3) return BV_EINVAL;
    int64_t n_tot = 0;
    for (int k = 0; k < ndata; ++k) {
        if (n_per[k] <= 0) return BV_EINVAL;
        n_tot += n_per[k];
    }
    if (n_tot >= (int64_t)INT32_MAX) return BV_EINVAL;
    for (int64_t i = 0; i < n_tot * d; ++i)
        if (!std::isfinite(locs[i])) return BV_EINVAL;
    if (y)
        for (int64_t i = 0; i < n_tot; ++i)
            if (!std::isfinite(y[i])) return BV_EINVAL;
    BV_CUDA(cudaSetDevice(c->device));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    free_data(c);
    c->d = d;
    c->ndata = ndata;
    c->n_tot = n_tot;
    c->pt_off.assign(ndata + 1, 0);
    for (int k = 0; k < ndata; ++k) c->pt_off[k + 1] = c->pt_off[k] + n_per[k];
    c->h_locs.assign(locs, locs + n_tot * d);
    std::vector<double> soa((size_t)n_tot * d);
    for (int64_t i = 0; i < n_tot; ++i)
        for (int k = 0; k < d; ++k) soa[(size_t)k * n_tot + i] = locs[i * d + k];
    BV_CUDA(cudaMalloc(&c->d_locs, sizeof(double) * n_tot * d));
    BV_CUDA(cudaMalloc(&c->d_y, sizeof(double) * n_tot));
    BV_CUDA(cudaMalloc(&c->d_out, sizeof(double) * ndata));
    BV_CUDA(cudaMalloc(&c->d_quad, sizeof(double) * ndata));
    BV_CUDA(cudaMallocHost(&c->h_quad, sizeof(double) * ndata));
    BV_CUDA(cudaMalloc(&c->d_theta, sizeof(DevTheta) * ndata));
    BV_CUDA(cudaMalloc(&c->d_gtab, sizeof(double) * BV_GTAB_DOUBLES * ndata));
    BV_CUDA(cudaMallocHost(&c->h_out, sizeof(double) * ndata));
    c->h_theta.assign(ndata, DevTheta{});
    BV_CUDA(cudaMemcpyAsync(c->d_locs, soa.data(), sizeof(double) * n_tot * d, cudaMemcpyHostToDevice,
                            c->stream));
    if (y) {
        BV_CUDA(cudaMemcpyAsync(c->d_y, y, sizeof(double) * n_tot, cudaMemcpyHostToDevice, c->stream));
        c->have_y = true;
    } else {
        BV_CUDA(cudaMemsetAsync(c->d_y, 0, sizeof(double) * n_tot, c->stream));
    }
    BV_CUDA(cudaStreamSynchronize(c->stream));
    return BV_OK;
}

extern "C" int bv_set_data(bv_ctx* c, const double* locs, const double* y, int64_t n, int32_t d) {
    return bv_set_datasets(c, 1, &n, locs, y, d);
}

extern "C" int bv_set_observations(bv_ctx* c, const double* y, int32_t on_device) {
    if (!c || !y) return BV_EINVAL;
    if (!c->d_y) return BV_ESTATE;
    if (on_device) {
        BV_CUDA(cudaMemcpyAsync(c->d_y, y, sizeof(double) * c->n_tot, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        for (int64_t i = 0; i < c->n_tot; ++i)
            if (!std::isfinite(y[i])) return BV_EINVAL;
        BV_CUDA(cudaMemcpyAsync(c->d_y, y, sizeof(double) * c->n_tot, cudaMemcpyHostToDevice, c->stream));
        BV_CUDA(cudaStreamSynchronize(c->stream));
    }
    c->have_y = true;
    return refresh_layout_y(c);
}

// ------------------------------------------------------------------------------------
// blocks
// ------------------------------------------------------------------------------------

// Upload the host block structure (h_bptr, h_pidx, h_bds, ds_blk_off) and centroids.
static int upload_blocks(bv_ctx* c, const std::vector<double>& cent) {
    const int64_t nb = c->nblk;
    BV_CUDA(cudaMalloc(&c->d_bptr, sizeof(int64_t) * (nb + 1)));
    BV_CUDA(cudaMalloc(&c->d_pidx, sizeof(int32_t) * c->n_tot));
    BV_CUDA(cudaMalloc(&c->d_cent, sizeof(double) * nb * c->d));
    BV_CUDA(cudaMalloc(&c->d_bds, sizeof(int32_t) * nb));
    BV_CUDA(cudaMalloc(&c->d_ds_blk_off, sizeof(int64_t) * (c->ndata + 1)));
    BV_CUDA(cudaMalloc(&c->d_ell_blk, sizeof(double) * nb));
    BV_CUDA(cudaMalloc(&c->d_u_blk, sizeof(double) * nb));
    {
        int64_t mx = 1;
        for (int k = 0; k < c->ndata; ++k) mx = std::max<int64_t>(mx, c->ds_blk_off[k + 1] - c->ds_blk_off[k]);
        c->red_chunks = bv_reduce_chunks(mx);
        BV_CUDA(cudaMalloc(&c->d_red_part, sizeof(double) * 4 * (size_t)c->ndata * c->red_chunks));
    }
    BV_CUDA(cudaMemcpyAsync(c->d_bptr, c->h_bptr.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice,
                            c->stream));
    BV_CUDA(cudaMemcpyAsync(c->d_pidx, c->h_pidx.data(), sizeof(int32_t) * c->n_tot, cudaMemcpyHostToDevice,
                            c->stream));
    BV_CUDA(cudaMemcpyAsync(c->d_cent, cent.data(), sizeof(double) * nb * c->d, cudaMemcpyHostToDevice,
                            c->stream));
    BV_CUDA(cudaMemcpyAsync(c->d_bds, c->h_bds.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, c->stream));
    BV_CUDA(cudaMemcpyAsync(c->d_ds_blk_off, c->ds_blk_off.data(), sizeof(int64_t) * (c->ndata + 1),
                            cudaMemcpyHostToDevice, c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    c->have_blocks = true;
    return BV_OK;
}

extern "C" int bv_build_blocks_multi(bv_ctx* c, const int64_t* bc_per, uint64_t seed, int32_t iters,
                                     int64_t* bc_eff_per) {
    if (!c || !bc_per || iters < 0) return BV_EINVAL;
    if (!c->d_locs) return BV_ESTATE;
    for (int k = 0; k < c->ndata; ++k)
        if (bc_per[k] <= 0 || bc_per[k] > c->pt_off[k + 1] - c->pt_off[k]) return BV_EINVAL;
    BV_CUDA(cudaSetDevice(c->device));
    free_blocks(c);
    const int d = c->d;
    std::vector<int64_t> bptr(1, 0);
    std::vector<int32_t> pidx;
    std::vector<int32_t> bds;
    std::vector<double> cent_all;
    std::vector<int64_t> dsoff(1, 0);
    pidx.reserve(c->n_tot);
    for (int ds = 0; ds < c->ndata; ++ds) {
        const int64_t off = c->pt_off[ds], n = c->pt_off[ds + 1] - off, k = bc_per[ds];
        const uint64_t sd = seed + (uint64_t)ds;
        int32_t* d_label = nullptr;
        double* d_cent = nullptr;
        int64_t* d_counts = nullptr;
        BV_CUDA(cudaMalloc(&d_label, sizeof(int32_t) * n));
        BV_CUDA(cudaMalloc(&d_cent, sizeof(double) * k * d));
        BV_CUDA(cudaMalloc(&d_counts, sizeof(int64_t) * k));
        int st = bv_kmeans_device(c->d_locs, c->n_tot, off, n, d, k, sd, iters, d_label, d_cent, c->stream);
        int sc = 0, q = 0;
        if (st == BV_OK) {
            bv_kmeans_scales(c->h_locs.data() + off * d, n, d, &sc, &q);
            // block centroids: exact-integer means of the final members
            st = bv_centroids_device(c->d_locs, c->n_tot, off, n, d, d_label, k, q, d_cent, d_counts, c->stream);
        }
        std::vector<int32_t> label(n);
        std::vector<double> cent((size_t)k * d);
        std::vector<int64_t> counts(k);
        if (st == BV_OK) {
            cudaError_t e = cudaMemcpyAsync(label.data(), d_label, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(cent.data(), d_cent, sizeof(double) * k * d, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(counts.data(), d_counts, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) {
                bv_record_cuda_error(e, "kmeans copy-out", __FILE__, __LINE__);
                st = BV_ECUDA;
            }
        }
        cudaFree(d_label);
        cudaFree(d_cent);
        cudaFree(d_counts);
        if (st != BV_OK) return st;
        // drop empty clusters, random block order zeta (Fisher-Yates on SplitMix64 draws)
        std::vector<int64_t> clus_of_blk;
        for (int64_t cl = 0; cl < k; ++cl)
            if (counts[cl] > 0) clus_of_blk.push_back(cl);
        const int64_t nb = (int64_t)clus_of_blk.size();
        std::vector<int64_t> perm(nb);
        std::iota(perm.begin(), perm.end(), 0);
        const uint64_t zs = BV_STREAM_ZETA(sd);
        for (int64_t i = nb - 1; i >= 1; --i) {
            const uint64_t r = bv_sm64(zs, (uint64_t)i);
            const int64_t j = (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(i + 1)) >> 64);
            std::swap(perm[i], perm[j]);
        }
        std::vector<int64_t> pos_of_clus(k, -1);
        const int64_t b0 = (int64_t)bptr.size() - 1;
        for (int64_t p = 0; p < nb; ++p) {
            const int64_t cl = clus_of_blk[perm[p]];
            pos_of_clus[cl] = p;
            bptr.push_back(bptr.back() + counts[cl]);
            for (int j = 0; j < d; ++j) cent_all.push_back(cent[cl * d + j]);
            bds.push_back(ds);
        }
        pidx.resize(off + n);
        std::vector<int64_t> fill(nb, 0);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t p = pos_of_clus[label[i]];
            pidx[bptr[b0 + p] + fill[p]++] = (int32_t)(off + i);
        }
        dsoff.push_back(dsoff.back() + nb);
        if (bc_eff_per) bc_eff_per[ds] = nb;
    }
    c->h_bptr = std::move(bptr);
    c->h_pidx = std::move(pidx);
    c->h_bds = std::move(bds);
    c->ds_blk_off = std::move(dsoff);
    c->nblk = c->ds_blk_off.back();
    return upload_blocks(c, cent_all);
}

extern "C" int bv_build_blocks(bv_ctx* c, int64_t bc, uint64_t seed, int32_t iters, int64_t* block_ptr,
                               int32_t* point_idx, int64_t* bc_eff) {
    if (!c) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    int64_t nb = 0;
    BV_TRY(bv_build_blocks_multi(c, &bc, seed, iters, &nb));
    if (bc_eff) *bc_eff = nb;
    if (block_ptr) memcpy(block_ptr, c->h_bptr.data(), sizeof(int64_t) * (nb + 1));
    if (point_idx) memcpy(point_idx, c->h_pidx.data(), sizeof(int32_t) * c->n_tot);
    return BV_OK;
}

// Reorders the blocks: new position q holds the block at current position perm[q]
// (ncent: the centroids in the new order).  Neighbour sets are dropped.
int bv_apply_block_order(bv_ctx* c, const std::vector<int64_t>& perm, const std::vector<double>& ncent) {
    const int64_t bc = c->nblk;
    std::vector<int64_t> bptr(bc + 1, 0);
    std::vector<int32_t> pidx;
    pidx.reserve(c->n_tot);
    for (int64_t q = 0; q < bc; ++q) {
        const int64_t p = perm[q];
        bptr[q + 1] = bptr[q] + (c->h_bptr[p + 1] - c->h_bptr[p]);
        pidx.insert(pidx.end(), c->h_pidx.begin() + c->h_bptr[p], c->h_pidx.begin() + c->h_bptr[p + 1]);
    }
    std::vector<int32_t> bds(bc, 0);
    std::vector<int64_t> dsoff = c->ds_blk_off;
    free_blocks(c);
    c->h_bptr = std::move(bptr);
    c->h_pidx = std::move(pidx);
    c->h_bds = std::move(bds);
    c->ds_blk_off = std::move(dsoff);
    c->nblk = bc;
    return upload_blocks(c, ncent);
}

extern "C" int bv_build_singletons(bv_ctx* c, uint64_t seed, int64_t* block_ptr, int32_t* point_idx) {
    if (!c) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    const int64_t n = c->n_tot;
    const int d = c->d;
    BV_CUDA(cudaSetDevice(c->device));
    free_blocks(c);
    std::vector<int32_t> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    const uint64_t zs = BV_STREAM_ZETA(seed);
    for (int64_t i = n - 1; i >= 1; --i) {
        const uint64_t r = bv_sm64(zs, (uint64_t)i);
        const int64_t j = (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(i + 1)) >> 64);
        std::swap(perm[i], perm[j]);
    }
    std::vector<double> cent((size_t)n * d);
    for (int64_t p = 0; p < n; ++p)
        for (int k = 0; k < d; ++k) cent[(size_t)p * d + k] = c->h_locs[(size_t)perm[p] * d + k];
    c->h_bptr.resize(n + 1);
    std::iota(c->h_bptr.begin(), c->h_bptr.end(), (int64_t)0);
    c->h_pidx = std::move(perm);
    c->h_bds.assign(n, 0);
    c->ds_blk_off = {0, n};
    c->nblk = n;
    BV_TRY(upload_blocks(c, cent));
    if (block_ptr) memcpy(block_ptr, c->h_bptr.data(), sizeof(int64_t) * (n + 1));
    if (point_idx) memcpy(point_idx, c->h_pidx.data(), sizeof(int32_t) * n);
    return BV_OK;
}

extern "C" int bv_set_blocks(bv_ctx* c, int64_t bc, const int64_t* block_ptr, const int32_t* point_idx,
                             const double* centroids) {
    if (!c || bc <= 0 || !block_ptr || !point_idx) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    const int64_t n = c->n_tot;
    if (block_ptr[0] != 0 || block_ptr[bc] != n) return BV_EINVAL;
    for (int64_t i = 0; i < bc; ++i)
        if (block_ptr[i + 1] <= block_ptr[i]) return BV_EINVAL;
    std::vector<char> seen(n, 0);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t p = point_idx[i];
        if (p < 0 || p >= n || seen[p]) return BV_EINVAL;
        seen[p] = 1;
    }
    BV_CUDA(cudaSetDevice(c->device));
    free_blocks(c);
    const int d = c->d;
    std::vector<double> cent((size_t)bc * d);
    if (centroids) {
        std::copy(centroids, centroids + bc * d, cent.begin());
    } else {
        for (int64_t i = 0; i < bc; ++i)
            for (int k = 0; k < d; ++k) {
                double s = 0.0;
                for (int64_t p = block_ptr[i]; p < block_ptr[i + 1]; ++p) s += c->h_locs[(size_t)point_idx[p] * d + k];
                cent[(size_t)i * d + k] = s / (double)(block_ptr[i + 1] - block_ptr[i]);
            }
    }
    c->h_bptr.assign(block_ptr, block_ptr + bc + 1);
    c->h_pidx.assign(point_idx, point_idx + n);
    c->h_bds.assign(bc, 0);
    c->ds_blk_off = {0, bc};
    c->nblk = bc;
    return upload_blocks(c, cent);
}

// ------------------------------------------------------------------------------------
// neighbours
// ------------------------------------------------------------------------------------
static int upload_nptr(bv_ctx* c) {
    BV_CUDA(cudaMalloc(&c->d_nptr, sizeof(int64_t) * (c->nblk + 1)));
    BV_CUDA(cudaMemcpyAsync(c->d_nptr, c->h_nptr.data(), sizeof(int64_t) * (c->nblk + 1), cudaMemcpyHostToDevice,
                            c->stream));
    const int64_t tot = c->h_nptr.back();
    BV_CUDA(cudaMalloc(&c->d_nidx, sizeof(int32_t) * std::max<int64_t>(tot, 1)));
    return BV_OK;
}

extern "C" int bv_select_neighbors(bv_ctx* c, int32_t m, const int32_t* m_per_block, int64_t* nn_ptr,
                                   int32_t* nn_idx) {
    if (!c) return BV_EINVAL;
    if (!c->have_blocks) return BV_ESTATE;
    if (!m_per_block && m < 0) return BV_EINVAL;
    BV_CUDA(cudaSetDevice(c->device));
    free_neighbors(c);
    c->h_nptr.assign(c->nblk + 1, 0);
    for (int ds = 0; ds < c->ndata; ++ds) {
        const int64_t base = c->h_bptr[c->ds_blk_off[ds]];
        for (int64_t i = c->ds_blk_off[ds]; i < c->ds_blk_off[ds + 1]; ++i) {
            const int64_t want = m_per_block ? (int64_t)m_per_block[i] : (int64_t)m;
            if (want < 0) return BV_EINVAL;
            const int64_t avail = c->h_bptr[i] - base;
            const int64_t mi = std::min(want, avail);
            if (mi > 4000) return BV_EINVAL;  // exact-key list capacity of the selection kernel
            c->h_nptr[i + 1] = c->h_nptr[i] + mi;
        }
    }
    BV_TRY(upload_nptr(c));
    for (int ds = 0; ds < c->ndata; ++ds) {
        const int64_t off = c->pt_off[ds], n = c->pt_off[ds + 1] - off;
        double amax = 0.0;
        for (int64_t i = 0; i < n * c->d; ++i) amax = std::max(amax, fabs(c->h_locs[(size_t)off * c->d + i]));
        BV_TRY(bv_select_neighbors_device(c->d_locs, c->n_tot, c->d, c->d_bptr, c->d_pidx, c->d_cent,
                                          c->ds_blk_off[ds], c->ds_blk_off[ds + 1], c->h_nptr.data(), c->d_nptr,
                                          c->d_nidx, amax, c->stream));
    }
    BV_CUDA(cudaStreamSynchronize(c->stream));
    c->have_nn = true;
    if (nn_ptr) memcpy(nn_ptr, c->h_nptr.data(), sizeof(int64_t) * (c->nblk + 1));
    if (nn_idx && c->h_nptr.back() > 0)
        BV_CUDA(cudaMemcpy(nn_idx, c->d_nidx, sizeof(int32_t) * c->h_nptr.back(), cudaMemcpyDeviceToHost));
    return BV_OK;
}

extern "C" int bv_set_neighbors(bv_ctx* c, const int64_t* nn_ptr, const int32_t* nn_idx) {
    if (!c || !nn_ptr) return BV_EINVAL;
    if (!c->have_blocks) return BV_ESTATE;
    if (nn_ptr[0] != 0) return BV_EINVAL;
    for (int64_t i = 0; i < c->nblk; ++i)
        if (nn_ptr[i + 1] < nn_ptr[i]) return BV_EINVAL;
    const int64_t tot = nn_ptr[c->nblk];
    if (tot > 0 && !nn_idx) return BV_EINVAL;
    for (int ds = 0; ds < c->ndata; ++ds)
        for (int64_t i = c->ds_blk_off[ds]; i < c->ds_blk_off[ds + 1]; ++i)
            for (int64_t p = nn_ptr[i]; p < nn_ptr[i + 1]; ++p)
                if (nn_idx[p] < c->pt_off[ds] || nn_idx[p] >= c->pt_off[ds + 1]) return BV_EINVAL;
    BV_CUDA(cudaSetDevice(c->device));
    free_neighbors(c);
    c->h_nptr.assign(nn_ptr, nn_ptr + c->nblk + 1);
    BV_TRY(upload_nptr(c));
    if (tot > 0)
        BV_CUDA(cudaMemcpyAsync(c->d_nidx, nn_idx, sizeof(int32_t) * tot, cudaMemcpyHostToDevice, c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    c->have_nn = true;
    return BV_OK;
}

extern "C" int bv_get_sizes(bv_ctx* c, int64_t* nb, int64_t* nn) {
    if (!c) return BV_EINVAL;
    if (nb) *nb = c->nblk;
    if (nn) *nn = c->have_nn ? c->h_nptr.back() : 0;
    return BV_OK;
}

extern "C" int bv_get_blocks(bv_ctx* c, int64_t* block_ptr, int32_t* point_idx, double* centroids) {
    if (!c) return BV_EINVAL;
    if (!c->have_blocks) return BV_ESTATE;
    if (block_ptr) memcpy(block_ptr, c->h_bptr.data(), sizeof(int64_t) * (c->nblk + 1));
    if (point_idx) memcpy(point_idx, c->h_pidx.data(), sizeof(int32_t) * c->n_tot);
    if (centroids)
        BV_CUDA(cudaMemcpy(centroids, c->d_cent, sizeof(double) * c->nblk * c->d, cudaMemcpyDeviceToHost));
    return BV_OK;
}

extern "C" int bv_get_neighbors(bv_ctx* c, int64_t* nn_ptr, int32_t* nn_idx) {
    if (!c) return BV_EINVAL;
    if (!c->have_nn) return BV_ESTATE;
    if (nn_ptr) memcpy(nn_ptr, c->h_nptr.data(), sizeof(int64_t) * (c->nblk + 1));
    if (nn_idx && c->h_nptr.back() > 0)
        BV_CUDA(cudaMemcpy(nn_idx, c->d_nidx, sizeof(int32_t) * c->h_nptr.back(), cudaMemcpyDeviceToHost));
    return BV_OK;
}

// ------------------------------------------------------------------------------------
// evaluation plan: size bins, launch shapes, workspace
// ------------------------------------------------------------------------------------
// Temme's gamma-function combinations at |mu| <= 1/2, from the series
//   log(1/G(1+z)) = gamma z - sum_{k>=2} (-1)^k zeta(k) z^k / k   (|z| < 1),
// split into its even part E(mu) and odd part O(mu): 1/G(1 +- mu) = exp(E +- O), so
// gam2 = e^E cosh(O) and gam1 = -e^E sinh(O) / mu (no cancellation as mu -> 0).  zeta(k)
// by direct summation to 1000 with the Euler-Maclaurin tail; all in long double.
static void temme_constants(double mu, double* gam1, double* gam2, double* gampl, double* gammi) {
    static long double zeta[65];
    static bool init = false;
    if (!init) {
        for (int k = 2; k <= 64; ++k) {
            const long double N = 1000.0L;
            long double s = 0.0L;
            for (int j = 999; j >= 1; --j) s += powl((long double)j, -(long double)k);
            const long double Nk = powl(N, -(long double)k);
            // sum_{j>=N} j^-k = N^{1-k}/(k-1) + N^-k/2 + k N^{-k-1}/12 - k(k+1)(k+2) N^{-k-3}/720 + ...
            s += N * Nk / (k - 1) + 0.5L * Nk + (long double)k * Nk / N / 12.0L -
                 (long double)k * (k + 1) * (k + 2) * Nk / (N * N * N) / 720.0L;
            zeta[k] = s;
        }
        init = true;
    }
    const long double eg = 0.57721566490153286060651209008240243L;  // Euler's gamma
    const long double m = mu;
    long double E = 0.0L, Oq = eg;  // O = mu * Oq
    long double pk = m;             // m^(k-1)
    for (int k = 2; k <= 64; ++k) {
        pk *= m;                    // m^k ... for even k add to E; odd k add m^(k-1) to Oq
        if (k % 2 == 0) E -= zeta[k] * pk / k;
        else Oq += zeta[k] * (pk / m) / k;
        if (m == 0.0L) break;
    }
    const long double O = m * Oq;
    long double shq;  // sinh(O) / O
    if (fabsl(O) < 1e-4L) shq = 1.0L + O * O / 6.0L + O * O * O * O / 120.0L;
    else shq = sinhl(O) / O;
    const long double eE = expl(E);
    *gam1 = (double)(-eE * shq * Oq);
    *gam2 = (double)(eE * coshl(O));
    *gampl = (double)expl(E + O);
    *gammi = (double)expl(E - O);
}

int bv_theta_to_dev(const bv_theta* t, int d, DevTheta* o) {
    if (!t) return BV_EINVAL;
    if (!(t->sigma2 > 0.0) || !(t->nugget >= 0.0) || !std::isfinite(t->sigma2) || !std::isfinite(t->nugget))
        return BV_EINVAL;
    *o = DevTheta{};
    o->nu = t->nu;
    if (t->nu == 0.5) o->nu_code = NU_HALF;
    else if (t->nu == 1.5) o->nu_code = NU_3HALF;
    else if (t->nu == 2.5) o->nu_code = NU_5HALF;
    else if (t->nu > 0.0 && t->nu <= BV_NU_MAX) {
        o->nu_code = NU_GENERAL;
        o->nrec = (int32_t)floor(t->nu + 0.5);
        o->mu = t->nu - (double)o->nrec;
        temme_constants(o->mu, &o->gam1, &o->gam2, &o->gampl, &o->gammi);
        o->lognorm = (double)((1.0L - (long double)t->nu) * logl(2.0L) - lgammal((long double)t->nu));
    } else {
        return BV_EINVAL;
    }
    for (int k = 0; k < 3; ++k) {
        const double r = t->aniso ? t->range[k] : t->range[0];
        if (k < d && !(r > 0.0 && std::isfinite(r))) return BV_EINVAL;
        o->inv_range[k] = (k < d) ? 1.0 / r : 0.0;
    }
    o->sigma2 = t->sigma2;
    o->nugget = t->nugget;
    o->sigma2_f = (float)o->sigma2;
    o->nugget_f = (float)o->nugget;
    // the kernels' diagonal is the FP32 sum sigma2_f + nugget_f; its rounding is the same
    // in every block, a systematic error that a small nugget turns into a bias of ell
    const float d32 = o->sigma2_f + o->nugget_f;
    o->diag_lo_f = (float)((o->sigma2 + o->nugget) - (double)d32);
    for (int k = 0; k < 3; ++k) o->inv_range_f[k] = (float)o->inv_range[k];
    return BV_OK;
}

static const int kBinEdges[] = {16, 32, 48, 64, 80, 96, 112, 128, 160, 192, 224, 256, 288, 320};

// CTA sizes of the shared-memory kernels: one panel warp plus 2, 4, 8 or 16 update warps.
static int default_threads(int kind, int nmax) {
    if (kind == 2) return 256;
    if (nmax <= 48) return 96;
    if (nmax <= 128) return 160;
    return 288;
}

static LLArgs make_args(bv_ctx* c) {
    LLArgs a;
    const bool lay = c->have_layout;
    a.locs = lay ? c->d_locs_int : c->d_locs;
    a.n_tot = c->n_tot;
    a.d = c->d;
    a.y = lay ? c->d_y_int : c->d_y;
    a.bptr = c->d_bptr;
    a.pidx = lay ? c->d_pidx_int : c->d_pidx;
    a.nptr = c->d_nptr;
    a.nidx = lay ? c->d_nidx_int : c->d_nidx;
    a.cent = c->d_cent;
    a.bds = c->d_bds;
    a.theta = c->d_theta;
    a.work = nullptr;
    a.nwork = 0;
    a.nwork_dev = nullptr;
    a.ctr = nullptr;
    a.ell_blk = c->d_ell_blk;
    a.u_blk = c->d_u_blk;
    a.ind_blk = nullptr;
    a.fail = c->d_fail;
    a.ws = c->d_ws;
    a.ws_stride = c->ws_stride;
    a.gen = c->cur_gen ? 1 : 0;
    a.fb = nullptr;
    a.dyn = 0;
    a.gtab = c->d_gtab;
    bv_exp_consts(&a.ex);
    return a;
}

static int set_grid(bv_ctx* c, BinPlan& bp) {
    bp.smem = bv_smem_bytes(bp.kind, bp.nmax, c->d, bp.threads);
    if (bp.kind == 2) {
        bp.grid = std::min<int>(bp.nwork, c->ws_slots);
        return BV_OK;
    }
    const int occ = bv_occupancy(bp.kind, bp.threads, bp.smem);
    if (occ <= 0) return BV_EINTERNAL;
    const int64_t per_cta = (bp.kind == 3 || bp.kind == 4) ? bp.threads / 32 : 1;  // blocks in flight per CTA
    bp.grid = (int)std::min<int64_t>((bp.nwork + per_cta - 1) / per_cta, (int64_t)occ * c->num_sms);
    return BV_OK;
}

// Samples per dataset of the mixed path's error check: every block of a small dataset,
// else at least kChkMinSamples and 1/kChkFrac of the blocks, at evenly spaced positions
// of the (random) block order.
static const int64_t kChkMinSamples = 64, kChkFrac = 256;

// FP64 bins of the mixed path's error check: one launch per bin for the sampled blocks
// (static lists) and one for the blocks of datasets that fail the check (lists filled on
// the device during the evaluation).  Blocks beyond the FP64 shared-memory limit use the
// global-memory kernel with the fallback workspace.
static int build_check(bv_ctx* c, const std::vector<int>& Nof) {
    free_check(c);
    auto& k = c->chk;
    const int nsm = bv_smem_max_n(0, c->d);
    std::vector<int> edges;
    for (int e : kBinEdges)
        if (e < nsm) edges.push_back(e);
    edges.push_back(nsm);
    const size_t nbin = edges.size() + 1;
    std::vector<int32_t> bin_of(c->nblk);
    std::vector<std::vector<int32_t>> all(nbin), smp(nbin);
    for (int64_t i = 0; i < c->nblk; ++i) {
        size_t b = 0;
        while (b < edges.size() && Nof[i] > edges[b]) ++b;
        bin_of[i] = (int32_t)b;
        all[b].push_back((int32_t)i);
    }
    std::vector<int64_t> sptr(c->ndata + 1, 0);
    std::vector<int32_t> samp;
    for (int ds = 0; ds < c->ndata; ++ds) {
        const int64_t lo = c->ds_blk_off[ds], B = c->ds_blk_off[ds + 1] - lo;
        const int64_t sn = std::min<int64_t>(B, std::max<int64_t>(kChkMinSamples, (B + kChkFrac - 1) / kChkFrac));
        for (int64_t q = 0; q < sn; ++q) {
            const int32_t blk = (int32_t)(lo + (q * B) / sn);
            samp.push_back(blk);
            smp[bin_of[blk]].push_back(blk);
        }
        sptr[ds + 1] = (int64_t)samp.size();
    }
    // (the positions are fixed by (B, s) alone: the check kernel and the redo list
    // recognise a sampled block from its position, bv_loglik.cu)
    k.nsamp = (int64_t)samp.size();
    std::vector<int64_t> roff(nbin + 1, 0);
    for (size_t b = 0; b < nbin; ++b) roff[b + 1] = roff[b] + (int64_t)all[b].size();
    BV_CUDA(bv_plan_malloc(&k.d_samp, sizeof(int32_t) * std::max<size_t>(samp.size(), 1)));
    BV_CUDA(bv_plan_malloc(&k.d_samp_ptr, sizeof(int64_t) * (c->ndata + 1)));
    BV_CUDA(bv_plan_malloc(&k.d_blk_bin, sizeof(int32_t) * c->nblk));
    BV_CUDA(bv_plan_malloc(&k.d_roff, sizeof(int64_t) * (nbin + 1)));
    BV_CUDA(bv_plan_malloc(&k.d_redo, sizeof(int32_t) * c->nblk));
    BV_CUDA(bv_plan_malloc(&k.d_cnt, sizeof(int) * BV_WCTR_PER_PREC));
    BV_CUDA(bv_plan_malloc(&k.d_ell, sizeof(double) * c->nblk));
    BV_CUDA(bv_plan_malloc(&k.d_u, sizeof(double) * c->nblk));
    BV_CUDA(bv_plan_malloc(&k.d_flag, sizeof(int32_t) * c->ndata));
    BV_CUDA(bv_plan_malloc(&k.d_thr, sizeof(float) * c->ndata));
    BV_CUDA(bv_plan_malloc(&k.d_est, sizeof(double) * c->ndata));
    BV_CUDA(cudaMemcpyAsync(k.d_samp, samp.data(), sizeof(int32_t) * samp.size(), cudaMemcpyHostToDevice, c->stream));
    BV_CUDA(cudaMemcpyAsync(k.d_samp_ptr, sptr.data(), sizeof(int64_t) * sptr.size(), cudaMemcpyHostToDevice,
                            c->stream));
    BV_CUDA(cudaMemcpyAsync(k.d_blk_bin, bin_of.data(), sizeof(int32_t) * c->nblk, cudaMemcpyHostToDevice, c->stream));
    BV_CUDA(cudaMemcpyAsync(k.d_roff, roff.data(), sizeof(int64_t) * roff.size(), cudaMemcpyHostToDevice, c->stream));
    BV_CUDA(cudaMemsetAsync(k.d_flag, 0, sizeof(int32_t) * c->ndata, c->stream));
    BV_CUDA(cudaMemsetAsync(k.d_est, 0, sizeof(double) * c->ndata, c->stream));
    if (nbin > (size_t)BV_WCTR_PER_PREC) return BV_EINTERNAL;
    for (size_t b = 0; b < nbin; ++b) {
        if (all[b].empty()) continue;
        BinPlan bp;
        int nmax = 0;
        for (int32_t i : all[b]) nmax = std::max(nmax, Nof[i]);
        bp.nmax = nmax;
        // (not timed by the autotuner: two-column steps from N = 112, where they win)
        bp.kind = b < edges.size() ? (nmax >= 112 && bv_smem_bytes(6, nmax, c->d, 0) <= (size_t)(227 * 1024 - 3072) ? 6 : 0) : 2;
        bp.threads = default_threads(bp.kind, bp.nmax);
        // redo launch: the whole bin's capacity, count from the device
        bp.nwork = (int32_t)all[b].size();
        bp.d_work = k.d_redo + roff[b];
        bp.d_ctr = c->d_wctr + 3 * BV_WCTR_PER_PREC + b;
        bp.smem = bv_smem_bytes(bp.kind, bp.nmax, c->d, bp.threads);
        if (bp.kind == 2) {
            bp.grid = std::min<int>(bp.nwork, c->fb_slots);
        } else {
            const int occ = bv_occupancy(bp.kind, bp.threads, bp.smem);
            if (occ <= 0) return BV_EINTERNAL;
            bp.grid = (int)std::min<int64_t>(bp.nwork, (int64_t)occ * c->num_sms);
        }
        bp.slot = (int)b;
        k.rbins.push_back(bp);
        if (!smp[b].empty()) {
            BinPlan sb = bp;
            sb.nwork = (int32_t)smp[b].size();
            sb.d_ctr = c->d_wctr + 2 * BV_WCTR_PER_PREC + b;
            sb.grid = std::min(sb.grid, sb.nwork);
            sb.d_work = nullptr;
            BV_CUDA(bv_plan_malloc(&sb.d_work, sizeof(int32_t) * smp[b].size()));
            k.sbins.push_back(sb);
            BV_CUDA(cudaMemcpyAsync(k.sbins.back().d_work, smp[b].data(), sizeof(int32_t) * smp[b].size(),
                                    cudaMemcpyHostToDevice, c->stream));
        }
    }
    return BV_OK;
}

int bv_ensure_plan(bv_ctx* c, int prec) {
    if (c->plan_valid[prec]) return BV_OK;
    BV_TRY(build_layout(c));
    free_plan(c, prec);
    const int smem_kind = prec == BV_MIXED ? 1 : 0;
    const int nsm = bv_smem_max_n(smem_kind, c->d);
    std::vector<int> Nof(c->nblk);
    int64_t maxlarge = 0;
    for (int64_t i = 0; i < c->nblk; ++i) {
        const int64_t N = (c->h_bptr[i + 1] - c->h_bptr[i]) + (c->h_nptr[i + 1] - c->h_nptr[i]);
        if (N > BV_LARGE_MAX_N) return BV_EINVAL;
        Nof[i] = (int)N;
        if (N > nsm) maxlarge = std::max<int64_t>(maxlarge, N);
    }
    // bins: edges up to the shared-memory limit, then one global-memory bin
    std::vector<int> edges;
    for (int e : kBinEdges)
        if (e < nsm) edges.push_back(e);
    edges.push_back(nsm);
    std::vector<std::vector<int32_t>> lists(edges.size() + 1);
    for (int64_t i = 0; i < c->nblk; ++i) {
        const int N = Nof[i];
        size_t b = 0;
        while (b < edges.size() && N > edges[b]) ++b;
        lists[b].push_back((int32_t)i);
    }
    // workspace for the global-memory bin
    if (maxlarge > 0) {
        const int64_t R = maxlarge + 1;
        const int64_t stride = (R * (R + 1)) / 2 + 2 * R + 3 * maxlarge + 8;
        const int64_t nlarge = (int64_t)lists.back().size();
        int slots = (int)std::min<int64_t>(nlarge, 2 * (int64_t)c->num_sms);
        // keep the workspace within a few GB
        while (slots > 1 && (double)slots * stride * 8.0 > 8e9) --slots;
        if (!c->d_ws || stride > c->ws_stride || slots > c->ws_slots) {
            dfree(c->d_ws);
            c->ws_stride = 0;
            c->ws_slots = 0;
            BV_CUDA(bv_plan_malloc(&c->d_ws, sizeof(double) * stride * slots));
            c->ws_stride = stride;
            c->ws_slots = slots;
        }
    }
    // mixed precision: FP64 fallback list and workspace slots sized for the largest block
    if (prec == BV_MIXED) {
        int64_t maxN = 1;
        for (int v : Nof) maxN = std::max<int64_t>(maxN, v);
        const int64_t R = maxN + 1;
        const int64_t stride = (R * (R + 1)) / 2 + 2 * R + 3 * maxN + 8;
        int slots = (int)std::min<int64_t>(c->nblk, (int64_t)c->num_sms);
        while (slots > 1 && (double)slots * stride * 8.0 > 2e9) --slots;
        dfree(c->d_fb_ws);
        dfree(c->d_fb);
        dfree(c->d_ind);
        c->fb_slots = 0;
        BV_CUDA(bv_plan_malloc(&c->d_ind, sizeof(float) * c->nblk));
        BV_CUDA(bv_plan_malloc(&c->d_fb_ws, sizeof(double) * stride * slots));
        BV_CUDA(bv_plan_malloc(&c->d_fb, sizeof(int) * (c->nblk + 1)));
        BV_CUDA(cudaMemsetAsync(c->d_fb, 0, sizeof(int), c->stream));
        c->fb_stride = stride;
        c->fb_slots = slots;
    }
    for (size_t b = 0; b < lists.size(); ++b) {
        auto& L = lists[b];
        if (L.empty()) continue;
        std::stable_sort(L.begin(), L.end(), [&](int32_t x, int32_t y) { return Nof[x] > Nof[y]; });
        BinPlan bp;
        bp.d_ctr = nullptr;
        bp.kind = b < edges.size() ? smem_kind : 2;
        bp.nmax = Nof[L.front()];
        bp.threads = default_threads(bp.kind, bp.nmax);
        bp.nwork = (int32_t)L.size();
        bp.h_work = L;
        bp.d_work = nullptr;
        BV_CUDA(bv_plan_malloc(&bp.d_work, sizeof(int32_t) * L.size()));
        c->plan[prec].push_back(bp);  // owned by the plan from here on (freed with it on any failure)
        BinPlan& pb = c->plan[prec].back();
        BV_CUDA(cudaMemcpyAsync(pb.d_work, L.data(), sizeof(int32_t) * L.size(), cudaMemcpyHostToDevice, c->stream));
        BV_TRY(set_grid(c, pb));
    }
    // largest bins first so the long blocks start early
    std::stable_sort(c->plan[prec].begin(), c->plan[prec].end(),
                     [](const BinPlan& x, const BinPlan& y) { return x.nmax > y.nmax; });
    if (c->plan[prec].size() > BV_WCTR_PER_PREC) return BV_EINVAL;
    for (size_t i = 0; i < c->plan[prec].size(); ++i) c->plan[prec][i].d_ctr = c->d_wctr + prec * BV_WCTR_PER_PREC + i;
    if (prec == BV_MIXED) BV_TRY(build_check(c, Nof));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    c->plan_valid[prec] = true;
    return BV_OK;
}

// Time one bin with the given CTA size (ms, best of `reps`).
static float time_bin(bv_ctx* c, BinPlan& bp, int reps) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const LLArgs a = make_args(c);
    float best = 1e30f;
    const bool ok = !c->cur_gen || bv_launch_gtab(c->d_theta, c->ndata, c->d_gtab, c->stream) == cudaSuccess;
    for (int r = 0; ok && r < reps + 1; ++r) {
        if (bv_launch_eval_reset(c->d_fail, c->d_wctr, BV_WCTR_GROUPS * BV_WCTR_PER_PREC, c->stream) != cudaSuccess)
            break;
        cudaEventRecord(e0, c->stream);
        cudaError_t e = bv_launch_bin(bp, a, c->stream);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            best = 1e30f;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

static int enqueue_eval_forked(bv_ctx* c, int prec);

// Time of one whole evaluation (best of three after one warm-up), launched directly.
static float time_eval(bv_ctx* c, int prec) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {
        cudaEventRecord(e0, c->stream);
        const int st = enqueue_eval_forked(c, prec);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st != BV_OK) {
            best = 1e30f;
            break;
        }
        if (r > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

static int autotune(bv_ctx* c, int prec) {
    if (c->tuned[prec]) return BV_OK;
    // theta of the current h_theta must be valid: use it as is (the caller set it)
    BV_CUDA(cudaMemcpyAsync(c->d_theta, c->h_theta.data(), sizeof(DevTheta) * c->ndata, cudaMemcpyHostToDevice,
                            c->stream));
    BV_CUDA(bv_launch_fail_reset(c->d_fail, c->stream));
    for (auto& bp : c->plan[prec]) {
        if (bp.kind == 2) continue;
        // candidates: CTA per block with 1 panel warp + 2/4/8/16 update warps (FP64 bins
        // with N >= 128 also 31); for small
        // blocks also a warp per block with 2/4/8 warps per CTA (mixed up to N = 128,
        // FP64 up to N = 64)
        // BV_KERNEL_FORM=cta or =warp restricts the choice to one form where both exist
        // (tests use it to check each kernel against the oracle); FP64 CTA bins try the
        // one-column and the two-column step (=cta keeps the first, =cta2 the second)
        const char* form = getenv("BV_KERNEL_FORM");
        const bool only_cta2 = form && strcmp(form, "cta2") == 0;
        const bool only_cta = (form && strcmp(form, "cta") == 0) || only_cta2;
        const bool only_warp = form && strcmp(form, "warp") == 0;
        // mixed bins with N >= 64 also try the tensor-core kernel (BV_KERNEL_FORM=tc
        // restricts them to it, =cta to the SIMT CTA kernel)
        std::vector<std::pair<int, int>> cands;
        const bool warp_ok = (bp.kind == 1 && bp.nmax <= 128) || (bp.kind == 0 && bp.nmax <= 64);
        const bool only_tc = form && strcmp(form, "tc") == 0;
        const bool tc_ok = bp.kind == 1 && bp.nmax >= 64 &&
                           bv_smem_bytes(5, bp.nmax, c->d, 256) <= (size_t)(227 * 1024 - 3072);
        const bool w2_ok = bp.kind == 0 && bv_smem_bytes(6, bp.nmax, c->d, 0) <= (size_t)(227 * 1024 - 3072);
        if (!(only_warp && warp_ok) && !(only_tc && tc_ok) && !(only_cta2 && w2_ok))
            for (int t : {96, 160, 288, 544, 1024})
                if (t < 1024 || (bp.kind == 0 && bp.nmax >= 128)) cands.push_back({bp.kind, t});
        if (w2_ok && !only_warp && !(only_cta && !only_cta2))
            for (int t : {96, 160, 288, 544, 1024})
                if (t < 1024 || bp.nmax >= 128) cands.push_back({6, t});
        if (!only_cta && !only_tc && warp_ok)
            for (int t : {64, 128, 256}) cands.push_back({bp.kind == 1 ? 3 : 4, t});
        if (!only_cta && !only_warp && tc_ok)
            for (int t : {128, 256, 384, 512}) cands.push_back({5, t});
        int best_k = bp.kind, best_t = bp.threads;
        float best_ms = 1e30f;
        for (auto kt : cands) {
            BinPlan trial = bp;
            trial.kind = kt.first;
            trial.threads = kt.second;
            if (set_grid(c, trial) != BV_OK) continue;
            const float ms = time_bin(c, trial, 2);
            if (getenv("BV_LOG_PLAN") && atoi(getenv("BV_LOG_PLAN")) >= 2)
                fprintf(stderr, "[bv plan]   candidate kind %d threads %d grid %d: %.3f ms\n", trial.kind,
                        trial.threads, trial.grid, ms);
            if (ms < best_ms) {
                best_ms = ms;
                best_k = kt.first;
                best_t = kt.second;
            }
        }
        bp.kind = best_k;
        bp.threads = best_t;
        BV_TRY(set_grid(c, bp));
        if (getenv("BV_LOG_PLAN"))
            fprintf(stderr, "[bv plan] prec %d bin nmax %d nwork %d -> kind %d threads %d grid %d smem %zu (%.3f ms)\n",
                    prec, bp.nmax, bp.nwork, bp.kind, bp.threads, bp.grid, bp.smem, best_ms);
    }
    BV_CUDA(cudaGetLastError());
    // Bins beside one another or one after another: the bins are timed alone above, but
    // beside a persistent bin that fills every SM the others compete for its slots, so
    // the evaluation is timed both ways (bins forked as parallel branches, or in sequence,
    // largest work first) and the faster kept.
    int nonempty = 0;
    for (const auto& bp : c->plan[prec]) nonempty += bp.nwork > 0;
    c->bin_serial[prec] = false;
    if (nonempty > 1) {
        const float t_fork = time_eval(c, prec);
        c->bin_serial[prec] = true;
        const float t_serial = time_eval(c, prec);
        BV_CUDA(cudaGetLastError());
        c->bin_serial[prec] = t_serial < t_fork;
        if (getenv("BV_LOG_PLAN"))
            fprintf(stderr, "[bv plan] prec %d evaluation: bins forked %.3f ms, in sequence %.3f ms -> %s\n", prec,
                    t_fork, t_serial, c->bin_serial[prec] ? "in sequence" : "forked");
    }
    c->tuned[prec] = true;
    return BV_OK;
}

extern "C" int bv_autotune(bv_ctx* c, int32_t prec) {
    if (!c || (prec != BV_FP64 && prec != BV_MIXED)) return BV_EINVAL;
    if (!c->have_nn) return BV_ESTATE;
    BV_CUDA(cudaSetDevice(c->device));
    BV_TRY(bv_ensure_plan(c, prec));
    // a neutral theta for timing if none was set yet
    for (int k = 0; k < c->ndata; ++k)
        if (c->h_theta[k].sigma2 <= 0.0) {
            bv_theta t = {1.0, {0.1, 0.1, 0.1}, 0.5, 1e-3, 0, 0};
            bv_theta_to_dev(&t, c->d, &c->h_theta[k]);
        }
    c->tuned[prec] = false;
    for (int slot : {prec, prec == BV_MIXED ? 2 : prec}) {
        if (c->graph[slot]) cudaGraphExecDestroy(c->graph[slot]);
        c->graph[slot] = nullptr;
        c->eval_direct_known[slot] = false;
    }
    return autotune(c, prec);
}

static int ensure_side(bv_ctx* c, size_t nb) {
    while (c->side.size() < nb) {
        cudaStream_t s;
        BV_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        c->side.push_back(s);
    }
    while (c->side_ev.size() < nb + 1) {
        cudaEvent_t e;
        BV_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->side_ev.push_back(e);
    }
    return BV_OK;
}

// Launch `bins` as parallel branches off the context's stream and join them (with
// dyn, each launch's work count is its bin's slot of the mixed check's device counts).
static int fork_bins(bv_ctx* c, const std::vector<BinPlan>& bins, const LLArgs& a, bool dyn) {
    BV_TRY(ensure_side(c, bins.size()));
    BV_CUDA(cudaEventRecord(c->side_ev[0], c->stream));
    for (size_t i = 0; i < bins.size(); ++i) {
        LLArgs ai = a;
        if (dyn) ai.nwork_dev = c->chk.d_cnt + bins[i].slot;
        BV_CUDA(cudaStreamWaitEvent(c->side[i], c->side_ev[0], 0));
        BV_CUDA(bv_launch_bin(bins[i], ai, c->side[i]));
        BV_CUDA(cudaEventRecord(c->side_ev[i + 1], c->side[i]));
    }
    for (size_t i = 0; i < bins.size(); ++i) BV_CUDA(cudaStreamWaitEvent(c->stream, c->side_ev[i + 1], 0));
    return BV_OK;
}

// The mixed path's error check (after the FP32 bins and their FP64 fallback): the sampled
// blocks in FP64, the per-dataset test against kMixedTol, and the FP64 recomputation of
// every block of a dataset that fails it.
static LLArgs check_args(bv_ctx* c, const LLArgs& a, bool sample) {
    LLArgs a64 = a;
    a64.fb = nullptr;
    a64.dyn = 0;
    a64.ind_blk = nullptr;
    a64.ws = c->d_fb_ws;
    a64.ws_stride = c->fb_stride;
    if (sample) {
        a64.ell_blk = c->chk.d_ell;
        a64.u_blk = c->chk.d_u;
    }
    return a64;
}

static int enqueue_check(bv_ctx* c, const LLArgs& a) {
    auto& k = c->chk;
    BV_CUDA(bv_launch_mixed_check(c->d_ell_blk, c->d_u_blk, k.d_ell, k.d_u, c->d_ind, k.d_samp, k.d_samp_ptr,
                                  c->d_ds_blk_off, c->ndata, c->mixed_tol, k.d_flag, k.d_thr, k.d_est, c->stream));
    BV_CUDA(cudaMemsetAsync(k.d_cnt, 0, sizeof(int) * BV_WCTR_PER_PREC, c->stream));
    BV_CUDA(bv_launch_mixed_redo_list(c->d_bds, c->nblk, k.d_flag, k.d_thr, c->d_ind, k.d_samp_ptr, c->d_ds_blk_off,
                                      k.d_blk_bin, k.d_roff, k.d_redo, k.d_cnt, c->stream));
    return fork_bins(c, k.rbins, check_args(c, a, false), true);
}

// The bins of one evaluation as parallel branches: failure reset, fork, every bin on its
// own side stream, join, reduction.  Captured into the graph, the branches become
// independent kernel nodes, so the CTAs of small bins fill the SMs that the tail of a
// large bin leaves idle.
static int enqueue_eval_forked(bv_ctx* c, int prec) {
    const size_t nb = c->plan[prec].size();
    // with the mixed check, its FP64 sample runs as further branches beside the bins: it
    // needs only the inputs, and its latency hides behind theirs
    const bool check = prec == BV_MIXED && c->mixed_tol > 0.0 && !c->chk.rbins.empty();
    const size_t ns = check ? c->chk.sbins.size() : 0;
    BV_TRY(ensure_side(c, nb + ns));
    BV_CUDA(bv_launch_eval_reset(c->d_fail, c->d_wctr, BV_WCTR_GROUPS * BV_WCTR_PER_PREC, c->stream));
    if (c->cur_gen) BV_CUDA(bv_launch_gtab(c->d_theta, c->ndata, c->d_gtab, c->stream));
    const bool fallback = prec == BV_MIXED && c->d_fb;
    if (fallback) BV_CUDA(cudaMemsetAsync(c->d_fb, 0, sizeof(int), c->stream));
    BV_CUDA(cudaEventRecord(c->side_ev[0], c->stream));
    LLArgs a = make_args(c);
    if (fallback) a.fb = c->d_fb;
    if (prec == BV_MIXED) a.ind_blk = c->d_ind;
    if (c->bin_serial[prec]) {
        // in sequence on the context's stream, largest work (blocks x N^3) first
        std::vector<size_t> order(nb);
        std::iota(order.begin(), order.end(), (size_t)0);
        const auto& pl = c->plan[prec];
        auto work = [&](size_t i) { return (double)pl[i].nwork * pl[i].nmax * pl[i].nmax * pl[i].nmax; };
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return work(x) > work(y); });
        for (size_t i : order) BV_CUDA(bv_launch_bin(pl[i], a, c->stream));
        for (size_t i = 0; i < ns; ++i) BV_CUDA(bv_launch_bin(c->chk.sbins[i], check_args(c, a, true), c->stream));
    } else {
        for (size_t i = 0; i < nb + ns; ++i) {
            BV_CUDA(cudaStreamWaitEvent(c->side[i], c->side_ev[0], 0));
            if (i < nb) BV_CUDA(bv_launch_bin(c->plan[prec][i], a, c->side[i]));
            else BV_CUDA(bv_launch_bin(c->chk.sbins[i - nb], check_args(c, a, true), c->side[i]));
            BV_CUDA(cudaEventRecord(c->side_ev[i + 1], c->side[i]));
        }
        for (size_t i = 0; i < nb + ns; ++i) BV_CUDA(cudaStreamWaitEvent(c->stream, c->side_ev[i + 1], 0));
    }
    if (fallback) {
        LLArgs fa = a;
        fa.ws = c->d_fb_ws;
        fa.ws_stride = c->fb_stride;
        BV_CUDA(bv_launch_fallback(fa, c->fb_slots, c->stream));
    }
    if (check) BV_TRY(enqueue_check(c, a));
    BV_CUDA(bv_launch_reduce(c->d_ell_blk, c->d_u_blk, c->d_ds_blk_off, c->ndata, c->red_chunks, c->d_red_part,
                             c->d_out, c->d_quad, c->stream));
    return BV_OK;
}

// Graph of one evaluation, captured once per precision after tuning.  theta is copied in
// front of each launch.
static int graph_slot(const bv_ctx* c, int prec) { return prec == BV_MIXED && c->mixed_tol <= 0.0 ? 2 : prec; }

static int ensure_graph(bv_ctx* c, int prec) {
    const int slot = graph_slot(c, prec);
    if (c->graph[slot] && (c->graph_gen[slot] != c->cur_gen || (slot == 1 && c->graph_tol != c->mixed_tol))) {
        cudaGraphExecDestroy(c->graph[slot]);
        c->graph[slot] = nullptr;
    }
    if (c->graph[slot]) return BV_OK;
    c->graph_gen[slot] = c->cur_gen;
    if (slot == 1) c->graph_tol = c->mixed_tol;
    cudaGraph_t g = nullptr;
    BV_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int st = enqueue_eval_forked(c, prec);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != BV_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    BV_CUDA(e);
    e = cudaGraphInstantiate(&c->graph[slot], g, 0);
    cudaGraphDestroy(g);
    BV_CUDA(e);
    if (!c->eval_direct_known[slot]) {
        // The graph against the same launches issued directly: with several size bins as
        // parallel branches the graph has run up to 20% slower than the streams (config
        // 2: 5.55 against 4.65 ms per evaluation), so the faster of the two is kept.
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float tg = 1e30f;
        for (int r = 0; r < 4; ++r) {
            cudaEventRecord(e0, c->stream);
            const cudaError_t el = cudaGraphLaunch(c->graph[slot], c->stream);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (el != cudaSuccess) break;
            if (r > 0) tg = std::min(tg, ms);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        BV_CUDA(cudaGetLastError());
        const float td = time_eval(c, prec);
        BV_CUDA(cudaGetLastError());
        c->eval_direct[slot] = td < 0.98f * tg;
        c->eval_direct_known[slot] = true;
        if (getenv("BV_LOG_PLAN"))
            fprintf(stderr, "[bv plan] graph slot %d: graph %.3f ms, direct launches %.3f ms -> %s\n", slot, tg, td,
                    c->eval_direct[slot] ? "direct" : "graph");
    }
    return BV_OK;
}

int bv_enqueue_loglik(bv_ctx* c, int prec, double* d_out, bool) {
    BV_TRY(bv_ensure_plan(c, prec));
    BV_TRY(autotune(c, prec));
    BV_TRY(ensure_graph(c, prec));
    BV_CUDA(cudaMemcpyAsync(c->d_theta, c->h_theta.data(), sizeof(DevTheta) * c->ndata, cudaMemcpyHostToDevice,
                            c->stream));
    const int slot = graph_slot(c, prec);
    if (c->eval_direct[slot]) BV_TRY(enqueue_eval_forked(c, prec));
    else BV_CUDA(cudaGraphLaunch(c->graph[slot], c->stream));
    if (d_out && d_out != c->d_out)
        BV_CUDA(cudaMemcpyAsync(d_out, c->d_out, sizeof(double) * c->ndata, cudaMemcpyDeviceToDevice, c->stream));
    return BV_OK;
}

static int prepare_eval(bv_ctx* c, const bv_theta* thetas, int32_t prec) {
    if (!c || !thetas) return BV_EINVAL;
    if (prec != BV_FP64 && prec != BV_MIXED) return BV_EINVAL;
    if (!c->have_nn || !c->have_blocks) return BV_ESTATE;
    BV_CUDA(cudaSetDevice(c->device));
    bool gen = false;
    for (int k = 0; k < c->ndata; ++k) {
        BV_TRY(bv_theta_to_dev(&thetas[k], c->d, &c->h_theta[k]));
        gen = gen || c->h_theta[k].nu_code == NU_GENERAL;
    }
    c->cur_gen = gen;
    return BV_OK;
}

static int finish_sync(bv_ctx* c, double* out, int nout) {
    BV_CUDA(cudaMemcpyAsync(c->h_out, c->d_out, sizeof(double) * c->ndata, cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaMemcpyAsync(c->h_quad, c->d_quad, sizeof(double) * c->ndata, cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaMemcpyAsync(c->h_fail, c->d_fail, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    if (c->d_fb) BV_CUDA(cudaMemcpyAsync(c->h_fb, c->d_fb, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < nout; ++k) out[k] = c->h_out[k];
    return *c->h_fail != ~0ull ? BV_ENOTPD : BV_OK;
}

extern "C" int bv_loglik_multi(bv_ctx* c, const bv_theta* thetas, int32_t prec, double* out) {
    if (!out) return BV_EINVAL;
    BV_TRY(prepare_eval(c, thetas, prec));
    BV_TRY(bv_enqueue_loglik(c, prec, nullptr, true));
    return finish_sync(c, out, c->ndata);
}

extern "C" int bv_loglik_terms_multi(bv_ctx* c, const bv_theta* thetas, int32_t prec, double* out_loglik,
                                     double* out_quad) {
    if (!c || !out_loglik) return BV_EINVAL;
    BV_TRY(prepare_eval(c, thetas, prec));
    BV_TRY(bv_enqueue_loglik(c, prec, nullptr, true));
    const int st = finish_sync(c, out_loglik, c->ndata);
    if (out_quad) memcpy(out_quad, c->h_quad, sizeof(double) * c->ndata);
    return st;
}

extern "C" int bv_loglik(bv_ctx* c, const bv_theta* theta, int32_t prec, double* out, double* per_block) {
    if (!c || !out) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    BV_TRY(prepare_eval(c, theta, prec));
    BV_TRY(bv_enqueue_loglik(c, prec, nullptr, true));
    const int st = finish_sync(c, out, 1);
    if (per_block)
        BV_CUDA(cudaMemcpy(per_block, c->d_ell_blk, sizeof(double) * c->nblk, cudaMemcpyDeviceToHost));
    return st;
}

extern "C" int bv_loglik_async(bv_ctx* c, const bv_theta* thetas, int32_t prec, double* d_out) {
    if (!d_out) return BV_EINVAL;
    BV_TRY(prepare_eval(c, thetas, prec));
    return bv_enqueue_loglik(c, prec, d_out, true);
}

extern "C" int bv_sync(bv_ctx* c, int64_t* failed_block) {
    if (!c) return BV_EINVAL;
    BV_CUDA(cudaSetDevice(c->device));
    BV_CUDA(cudaMemcpyAsync(c->h_fail, c->d_fail, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    const bool failed = *c->h_fail != ~0ull;
    if (failed_block) *failed_block = failed ? (int64_t)*c->h_fail : -1;
    return failed ? BV_ENOTPD : BV_OK;
}

extern "C" int bv_plan_info(bv_ctx* c, int32_t prec, int32_t* launches, int32_t* nbins, double* flops,
                            double* entries) {
    if (!c || (prec != BV_FP64 && prec != BV_MIXED)) return BV_EINVAL;
    if (!c->have_nn) return BV_ESTATE;
    BV_CUDA(cudaSetDevice(c->device));
    BV_TRY(bv_ensure_plan(c, prec));
    // bins + failure reset + two reduction stages (+ the general-nu table)
    // (mixed: + the FP64 fallback pass, the check's sample and redo launches, the check
    // and the redo-list kernels)
    int32_t nl = (int32_t)c->plan[prec].size() + 3 + (c->cur_gen ? 1 : 0);
    if (prec == BV_MIXED) {
        nl += 1;
        if (c->mixed_tol > 0.0) nl += (int32_t)c->chk.sbins.size() + (int32_t)c->chk.rbins.size() + 2;
    }
    if (launches) *launches = nl;
    if (nbins) *nbins = (int32_t)c->plan[prec].size();
    double f = 0.0, e = 0.0;
    for (int64_t i = 0; i < c->nblk; ++i) {
        const double N = (double)((c->h_bptr[i + 1] - c->h_bptr[i]) + (c->h_nptr[i + 1] - c->h_nptr[i]));
        f += N * N * N / 3.0 + N * N;
        e += N * (N + 1.0) / 2.0;
    }
    if (flops) *flops = f;
    if (entries) *entries = e;
    return BV_OK;
}

extern "C" int bv_loglik_terms(bv_ctx* c, const bv_theta* theta, int32_t prec, double* out_loglik, double* out_quad,
                               double* out_logdet) {
    if (!c || !out_loglik) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    BV_TRY(prepare_eval(c, theta, prec));
    BV_TRY(bv_enqueue_loglik(c, prec, nullptr, true));
    const int st = finish_sync(c, out_loglik, 1);
    const double q = c->h_quad[0];
    if (out_quad) *out_quad = q;
    if (out_logdet) *out_logdet = -2.0 * c->h_out[0] - q - (double)c->n_tot * 1.8378770664093454835606594728112;
    return st;
}

extern "C" int bv_last_error_block(bv_ctx* c, int64_t* block) {
    if (!c || !block) return BV_EINVAL;
    *block = (c->h_fail && *c->h_fail != ~0ull) ? (int64_t)*c->h_fail : -1;
    return BV_OK;
}

extern "C" int bv_set_mixed_tolerance(bv_ctx* c, double tol) {
    if (!c || !(tol >= 0.0) || !(tol < 1.0)) return BV_EINVAL;
    c->mixed_tol = tol;  // the evaluation graph of this setting is (re)captured on next use
    return BV_OK;
}

extern "C" int bv_mixed_block_indicator(bv_ctx* c, float* out) {
    if (!c || !out) return BV_EINVAL;
    if (!c->d_ind || !c->plan_valid[BV_MIXED]) return BV_ESTATE;
    BV_CUDA(cudaSetDevice(c->device));
    BV_CUDA(cudaMemcpyAsync(out, c->d_ind, sizeof(float) * c->nblk, cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    return BV_OK;
}

extern "C" int bv_mixed_check_info(bv_ctx* c, int64_t* blocks_fp64, int32_t* datasets_touched, double* est_rel) {
    if (!c || !blocks_fp64) return BV_EINVAL;
    *blocks_fp64 = 0;
    if (datasets_touched) *datasets_touched = 0;
    if (!c->chk.d_flag || !c->plan_valid[BV_MIXED]) return BV_ESTATE;
    if (c->mixed_tol <= 0.0) return BV_OK;  // no check ran
    BV_CUDA(cudaSetDevice(c->device));
    std::vector<int32_t> f(c->ndata);
    std::vector<double> e(c->ndata);
    std::vector<int> cnt(BV_WCTR_PER_PREC);
    BV_CUDA(cudaMemcpyAsync(f.data(), c->chk.d_flag, sizeof(int32_t) * c->ndata, cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaMemcpyAsync(e.data(), c->chk.d_est, sizeof(double) * c->ndata, cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaMemcpyAsync(cnt.data(), c->chk.d_cnt, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost, c->stream));
    BV_CUDA(cudaStreamSynchronize(c->stream));
    int64_t nb = c->chk.nsamp;
    for (int v : cnt) nb += v;
    *blocks_fp64 = nb;
    for (int k = 0; k < c->ndata; ++k) {
        if (datasets_touched) *datasets_touched += f[k] ? 1 : 0;
        if (est_rel) est_rel[k] = e[k];
    }
    return BV_OK;
}

extern "C" int bv_mixed_fallbacks(bv_ctx* c, int64_t* count) {
    if (!c || !count) return BV_EINVAL;
    *count = c->h_fb ? *c->h_fb : 0;
    return BV_OK;
}
