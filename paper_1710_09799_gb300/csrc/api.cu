// C-ABI of the MLN solver: context life cycle, step loop and state I/O.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "pstd.h"
#include "dispatch.cuh"
#include "jit.h"
#include "mln.h"
#include "setup.h"
#include "tc_kernel.h"

namespace {

thread_local std::string g_create_err_store;

const char *kVersion = "mln-gb300 0.2 (sm_103a)";

#define MLN_CK(ctx, call)                                                       \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);    \
            return MLN_ECUDA;                                                   \
        }                                                                       \
    } while (0)

// out[c * rows + r] = tab[rows * D + r] + sum_k tab[r * D + k] * state[k * stride + m0 + c]
template <typename R>
__global__ void state_to_rows(const R *__restrict__ state, int64_t stride, int64_t m0, int64_t count, int D,
                              int rows, const double *__restrict__ tab, double *__restrict__ out) {
    int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (c >= count) return;
    for (int r = 0; r < rows; ++r) {
        double acc = tab[rows * D + r];
        for (int k = 0; k < D; ++k) acc += tab[r * D + k] * static_cast<double>(state[k * stride + m0 + c]);
        out[c * rows + r] = acc;
    }
}

// state[k * stride + c] = tab[D * D + k] + sum_j tab[k * D + j] * in[c * D + j]
template <typename R>
__global__ void rows_to_state(const double *__restrict__ in, int64_t count, int D, const double *__restrict__ tab,
                              R *__restrict__ state, int64_t stride) {
    int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (c >= count) return;
    for (int k = 0; k < D; ++k) {
        double acc = tab[D * D + k];
        for (int j = 0; j < D; ++j) acc += tab[k * D + j] * in[c * D + j];
        state[k * stride + c] = static_cast<R>(acc);
    }
}

// Every medium cell starts from the same state vector v (D doubles).
template <typename R>
__global__ void fill_state(R *__restrict__ state, int64_t stride, int64_t count, int D, const double *__restrict__ v) {
    int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (c >= count) return;
    for (int k = 0; k < D; ++k) state[k * stride + c] = static_cast<R>(v[k]);
}

__global__ void f32_to_f64(const float *__restrict__ in, double *__restrict__ out, int64_t n) {
    int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < n) out[i] = in[i];
}

__global__ void f64_to_f32(const double *__restrict__ in, float *__restrict__ out, int64_t n) {
    int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < n) out[i] = static_cast<float>(in[i]);
}

inline unsigned grid_for(int64_t n, int bs) { return static_cast<unsigned>((n + bs - 1) / bs); }

mln_status ensure_scratch(mln_ctx *c, size_t bytes) {
    if (c->scratch_bytes >= bytes) return MLN_OK;
    if (c->scratch) cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    MLN_CK(c, cudaMalloc(&c->scratch, bytes));
    c->scratch_bytes = bytes;
    return MLN_OK;
}

// Upload a rows x D table and its offsets (row-major, offsets after the matrix).
mln_status upload_table(mln_ctx *c, double **dst, const std::vector<double> &mat, const std::vector<double> &off) {
    std::vector<double> buf(mat);
    buf.insert(buf.end(), off.begin(), off.end());
    MLN_CK(c, cudaMalloc(dst, buf.size() * sizeof(double)));
    MLN_CK(c, cudaMemcpy(*dst, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice));
    return MLN_OK;
}

void pick_launch_shape(mln_ctx *c) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->sms = sms;
    if (c->tc) {
        // tiles of one MMA (128 rows) including the halo of K cells on both sides
        c->K = std::min(c->p.block_steps > 0 ? c->p.block_steps : 8, 32);
        c->tile = mln::tc_rows() - 2 * c->K;
        c->threads = 512;
        return;
    }
    const int maxt = c->max_threads;
    c->K = c->p.block_steps > 0 ? c->p.block_steps : 16;
    if (2 * c->K > maxt - 32) c->K = (maxt - 32) / 2;
    const int64_t n = c->p.n_cells;
    int tile = c->p.tile_cells;
    if (tile <= 0) {
        // one tile per SM (or per SM multiple) while a block stays <= maxt threads
        int64_t ntiles = sms;
        tile = static_cast<int>((n + ntiles - 1) / ntiles);
        while (tile + 2 * c->K > maxt) {
            ntiles += sms;
            tile = static_cast<int>((n + ntiles - 1) / ntiles);
        }
        tile = std::max(tile, 1);
    }
    if (tile > n) tile = static_cast<int>(n);
    if (tile + 2 * c->K > maxt) tile = maxt - 2 * c->K;
    c->tile = tile;
    c->threads = (tile + 2 * c->K + 31) / 32 * 32;
}

cudaError_t launch(mln_ctx *c, const mln::BlockArgs<double> &a, dim3 g, dim3 b, size_t smem) {
    if (c->jit_fn) return mln::jit_launch(c->jit_fn, a, g, b, smem, c->stream);
    if (c->sparse) return mln::launch_block_sparse(c->p.N, a, c->consts, g, b, smem, c->stream);
    return mln::launch_block(c->p.N, c->p.form, a, c->consts, g, b, smem, c->stream);
}

cudaError_t launch(mln_ctx *c, const mln::BlockArgs<float> &a, dim3 g, dim3 b, size_t smem) {
    if (c->tc && c->tcr) return mln::launch_tcr(c->p.N, a, c->tc_scal, c->tc_img, c->sms, c->stream);
    if (c->tc) return mln::launch_tc(c->p.N, a, c->tc_scal, c->tc_img, c->sms, c->stream);
    if (c->jit_fn) return mln::jit_launch(c->jit_fn, a, g, b, smem, c->stream);
    return mln::launch_block(c->p.N, c->p.form, a, c->consts, g, b, smem, c->stream);
}

// Largest block (multiple of 32, <= kMaxThreads) whose shared memory fits.
int sparse_max_threads(mln_ctx *c) {
    const size_t limit = 227 * 1024 - 1024;
    int best = 0;
    for (int t = 32; t <= mln::kMaxThreads; t += 32) {
        size_t bytes = mln::field_smem<double>(t) + mln::sparse_smem_bytes(c->p.N, t, c->nnz, c->nrowptr);
        if (bytes <= limit) best = t;
    }
    return best;
}

template <typename R>
size_t smem_for(mln_ctx *c, int threads) {
    size_t smem = mln::field_smem<R>(threads);
    if (c->sparse) smem += mln::sparse_smem_bytes(c->p.N, threads, c->nnz, c->nrowptr);
    return smem;
}

// Time candidate (K, tile) shapes; each candidate repeats one launch reading
// buffer set 0 and writing set 1, which leaves the caller's state untouched.
template <typename R>
mln_status autotune_t(mln_ctx *c, int trials) {
    if (c->pstd) return MLN_OK;  // one step per launch: no launch shape to choose
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n = c->p.n_cells;
    const int maxt = c->max_threads;
    const int Ks[] = {2, 4, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64};
    cudaEvent_t e0, e1;
    MLN_CK(c, cudaEventCreate(&e0));
    MLN_CK(c, cudaEventCreate(&e1));
    double best = 1e300;
    int bestK = c->K, bestTile = c->tile;
    for (int K : Ks) {
        if (2 * K > maxt - 32) continue;
        if (c->tc && K > 32) continue;
        std::vector<int> tiles;
        for (int m = 1; m <= 8; m *= 2) {
            int64_t nt = static_cast<int64_t>(m) * sms;
            int tile = static_cast<int>((n + nt - 1) / nt);
            if (tile + 2 * K <= maxt && tile >= 1) tiles.push_back(tile);
        }
        int whole = maxt - 2 * K;  // as few blocks as possible
        if (whole >= 1) tiles.push_back(static_cast<int>(std::min<int64_t>(whole, n)));
        if (c->tc) tiles.assign(1, mln::tc_rows() - 2 * K);  // the tile is fixed by the MMA rows
        std::sort(tiles.begin(), tiles.end());
        tiles.erase(std::unique(tiles.begin(), tiles.end()), tiles.end());
        for (int tile : tiles) {
            c->K = K;
            c->tile = tile;
            c->threads = c->tc ? 512 : (tile + 2 * K + 31) / 32 * 32;
            mln::BlockArgs<R> a = mln::base_args<R>(c);
            a.E_in = static_cast<const R *>(c->E[0]);
            a.H_in = static_cast<const R *>(c->H[0]);
            a.s_in = static_cast<const R *>(c->st[0]);
            a.E_out = static_cast<R *>(c->E[1]);
            a.H_out = static_cast<R *>(c->H[1]);
            a.s_out = static_cast<R *>(c->st[1]);
            a.src = nullptr;
            a.nsteps = K;
            const dim3 g(static_cast<unsigned>((n + tile - 1) / tile)), b(c->threads);
            const size_t smem = smem_for<R>(c, c->threads);
            if (launch(c, a, g, b, smem) != cudaSuccess) continue;
            MLN_CK(c, cudaEventRecord(e0, c->stream));
            for (int t = 0; t < trials; ++t) MLN_CK(c, launch(c, a, g, b, smem));
            MLN_CK(c, cudaEventRecord(e1, c->stream));
            MLN_CK(c, cudaEventSynchronize(e1));
            float ms = 0;
            MLN_CK(c, cudaEventElapsedTime(&ms, e0, e1));
            double per_step = ms / (static_cast<double>(trials) * K);
            if (per_step < best) {
                best = per_step;
                bestK = K;
                bestTile = tile;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->K = bestK;
    c->tile = bestTile;
    c->threads = c->tc ? 512 : (bestTile + 2 * bestK + 31) / 32 * 32;
    MLN_CK(c, cudaMemsetAsync(c->flags, 0, sizeof(unsigned int), c->stream));
    MLN_CK(c, cudaStreamSynchronize(c->stream));
    return MLN_OK;
}

template <typename R>
mln_status run_steps(mln_ctx *c, int64_t n_steps, const double *src) {
    if (c->pstd) return mln::pstd_steps(c, n_steps, src);
    const int64_t ntiles = (c->p.n_cells + c->tile - 1) / c->tile;
    mln::BlockArgs<R> a = mln::base_args<R>(c);
    const size_t smem = smem_for<R>(c, c->threads);
    int cur = 0;
    for (int64_t done = 0; done < n_steps;) {
        int ns = static_cast<int>(std::min<int64_t>(c->K, n_steps - done));
        a.E_in = static_cast<const R *>(c->E[cur]);
        a.H_in = static_cast<const R *>(c->H[cur]);
        a.s_in = static_cast<const R *>(c->st[cur]);
        a.E_out = static_cast<R *>(c->E[cur ^ 1]);
        a.H_out = static_cast<R *>(c->H[cur ^ 1]);
        a.s_out = static_cast<R *>(c->st[cur ^ 1]);
        a.src = (src && c->p.source_kind != MLN_SRC_NONE) ? src + done : nullptr;
        a.nsteps = ns;
        cudaError_t e = launch(c, a, dim3(static_cast<unsigned>(ntiles)), dim3(c->threads), smem);
        if (e != cudaSuccess) {
            c->err = std::string("step kernel launch: ") + cudaGetErrorString(e);
            return MLN_ECUDA;
        }
        ++c->launches;
        cur ^= 1;
        done += ns;
    }
    if (cur == 1) {
        MLN_CK(c, cudaMemcpyAsync(c->st[0], c->st[1], c->state_bytes, cudaMemcpyDeviceToDevice, c->stream));
        MLN_CK(c, cudaMemcpyAsync(c->E[0], c->E[1], c->field_bytes, cudaMemcpyDeviceToDevice, c->stream));
        MLN_CK(c, cudaMemcpyAsync(c->H[0], c->H[1], c->field_bytes, cudaMemcpyDeviceToDevice, c->stream));
    }
    return MLN_OK;
}

// Rows of the output table for medium cells [m0, m0 + count) into host memory.
mln_status read_rows(mln_ctx *c, int64_t m0, int64_t count, const double *tab, int rows, double *host) {
    if (count == 0) return MLN_OK;
    mln_status st = ensure_scratch(c, static_cast<size_t>(count) * rows * sizeof(double));
    if (st != MLN_OK) return st;
    double *out = static_cast<double *>(c->scratch);
    if (c->p.precision == MLN_FP64)
        state_to_rows<double><<<grid_for(count, 128), 128, 0, c->stream>>>(
            static_cast<const double *>(c->st[0]), c->stride, m0, count, c->D, rows, tab, out);
    else
        state_to_rows<float><<<grid_for(count, 128), 128, 0, c->stream>>>(
            static_cast<const float *>(c->st[0]), c->stride, m0, count, c->D, rows, tab, out);
    MLN_CK(c, cudaGetLastError());
    MLN_CK(c, cudaMemcpyAsync(host, out, static_cast<size_t>(count) * rows * sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
    MLN_CK(c, cudaStreamSynchronize(c->stream));
    return MLN_OK;
}

mln_status read_field(mln_ctx *c, const void *dev, double *host) {
    const int64_t n = c->p.n_cells;
    if (c->p.precision == MLN_FP64) {
        MLN_CK(c, cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    } else {
        mln_status st = ensure_scratch(c, n * sizeof(double));
        if (st != MLN_OK) return st;
        f32_to_f64<<<grid_for(n, 256), 256, 0, c->stream>>>(static_cast<const float *>(dev),
                                                               static_cast<double *>(c->scratch), n);
        MLN_CK(c, cudaGetLastError());
        MLN_CK(c, cudaMemcpyAsync(host, c->scratch, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    MLN_CK(c, cudaStreamSynchronize(c->stream));
    return MLN_OK;
}

mln_status write_field(mln_ctx *c, void *dev, const double *host) {
    const int64_t n = c->p.n_cells;
    if (c->p.precision == MLN_FP64) {
        MLN_CK(c, cudaMemcpyAsync(dev, host, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    } else {
        mln_status st = ensure_scratch(c, n * sizeof(double));
        if (st != MLN_OK) return st;
        MLN_CK(c, cudaMemcpyAsync(c->scratch, host, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        f64_to_f32<<<grid_for(n, 256), 256, 0, c->stream>>>(static_cast<const double *>(c->scratch),
                                                               static_cast<float *>(dev), n);
        MLN_CK(c, cudaGetLastError());
    }
    MLN_CK(c, cudaStreamSynchronize(c->stream));
    return MLN_OK;
}

mln_status check_cells(mln_ctx *c, int64_t cell0, int64_t count, int64_t *m0) {
    if (count < 0 || cell0 < c->p.medium_begin || cell0 + count > c->p.medium_end) {
        c->err = "cell range outside the medium";
        return MLN_EINVAL;
    }
    *m0 = cell0 - c->p.medium_begin;
    return MLN_OK;
}

}  // namespace

namespace mln {
std::string &create_error() { return g_create_err_store; }
}  // namespace mln

extern "C" {

const char *mln_version(void) { return kVersion; }

mln_status mln_kernel_source(const mln_params *p, char *buf, size_t cap, size_t *len) {
    if (!p) return MLN_EINVAL;
    std::string err;
    mln_status st = mln::validate(*p, err);
    mln::Setup s;
    if (st == MLN_OK) st = mln::build_setup(*p, s, err);
    if (st != MLN_OK) {
        mln::create_error() = err;
        return st;
    }
    if (p->kernel == MLN_KERNEL_DF32 && !mln::df_constants_in_range(s, p->dt, p->form == MLN_FORM_ROTATED)) {
        mln::create_error() = "MLN_KERNEL_DF32: a constant of the step is outside the double-float range";
        return MLN_EUNSUPPORTED;
    }
    const std::string src =
        p->kernel == MLN_KERNEL_DF32
            ? mln::jit_df_source(s, p->dt, mln::jit_body_flags(*p), p->form == MLN_FORM_ROTATED)
            : mln::jit_merged_source(s, p->dt, p->precision == MLN_FP32, p->form == MLN_FORM_ROTATED,
                                     mln::jit_body_flags(*p));
    if (len) *len = src.size();
    if (buf && cap > 0) {
        const size_t k = std::min(cap - 1, src.size());
        std::memcpy(buf, src.data(), k);
        buf[k] = '\0';
    }
    return MLN_OK;
}

mln_status mln_rotation_terms(int32_t precision, const double *x, int64_t n, double *s, double *c1) {
    if ((n > 0 && (!x || !s || !c1)) || n < 0 || (precision != MLN_FP64 && precision != MLN_FP32)) return MLN_EINVAL;
    if (n == 0) return MLN_OK;
    double *dx = nullptr;
    size_t bytes = static_cast<size_t>(n) * sizeof(double);
    if (cudaMalloc(&dx, 3 * bytes) != cudaSuccess) {
        cudaGetLastError();
        return MLN_ENOMEM;
    }
    mln_status st = MLN_OK;
    if (cudaMemcpy(dx, x, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        mln::launch_sin_cosm1(precision, dx, n, dx + n, dx + 2 * n, nullptr) != cudaSuccess ||
        cudaMemcpy(s, dx + n, bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(c1, dx + 2 * n, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        st = MLN_ECUDA;
    cudaFree(dx);
    return st;
}

mln_status mln_tc_product(int32_t nc, int32_t kc, int32_t a_in_tmem, const float *A, const double *B, float *C) {
    if (!A || !B || !C) {
        mln::create_error() = "NULL argument";
        return MLN_EINVAL;
    }
    std::string err;
    cudaError_t e = mln::tc_product(nc, kc, a_in_tmem != 0, A, B, C, err);
    if (e == cudaErrorInvalidValue) {
        mln::create_error() = "unsupported (nc, kc)";
        return MLN_EINVAL;
    }
    if (e != cudaSuccess) {
        mln::create_error() = std::string("tensor-core product: ") + cudaGetErrorString(e);
        return MLN_ECUDA;
    }
    if (!err.empty()) {
        mln::create_error() = err;
        return MLN_ETIMEOUT;
    }
    return MLN_OK;
}

mln_status mln_tc_product_f16(int32_t nc, int32_t kc, const float *A, const double *B, float *C) {
    if (!A || !B || !C) {
        mln::create_error() = "NULL argument";
        return MLN_EINVAL;
    }
    std::string err;
    cudaError_t e = mln::tcr_product(nc, kc, A, B, C, err);
    if (e == cudaErrorInvalidValue) {
        mln::create_error() = "unsupported (nc, kc)";
        return MLN_EINVAL;
    }
    if (e != cudaSuccess) {
        mln::create_error() = std::string("tensor-core product: ") + cudaGetErrorString(e);
        return MLN_ECUDA;
    }
    if (!err.empty()) {
        mln::create_error() = err;
        return MLN_ETIMEOUT;
    }
    return MLN_OK;
}

mln_status mln_tc_wait_selftest(void) {
    int dev = 0, major = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess || major < 10) {
        cudaGetLastError();
        mln::create_error() = "no tcgen05 device";
        return MLN_EUNSUPPORTED;
    }
    std::string err;
    cudaError_t e = mln::tc_wait_selftest(err);
    if (e != cudaSuccess) {
        mln::create_error() = std::string("tensor-core wait self-test: ") + cudaGetErrorString(e);
        return MLN_ECUDA;
    }
    if (!err.empty()) {
        mln::create_error() = err;
        return MLN_ETIMEOUT;
    }
    return MLN_OK;
}

const char *mln_status_string(mln_status s) {
    switch (s) {
    case MLN_OK: return "ok";
    case MLN_EINVAL: return "invalid argument";
    case MLN_ENOMEM: return "out of memory";
    case MLN_ECUDA: return "CUDA error";
    case MLN_ENUMERIC: return "numerical set-up check failed";
    case MLN_ETIMEOUT: return "device wait timed out";
    case MLN_EUNSUPPORTED: return "unsupported configuration";
    case MLN_ENONFINITE: return "non-finite field value";
    }
    return "unknown status";
}

const char *mln_last_error(const mln_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

const char *mln_create_error(void) { return mln::create_error().c_str(); }

mln_status mln_query_buffers(const mln_params *p, size_t *state_bytes, size_t *field_bytes) {
    if (!p) return MLN_EINVAL;
    std::string err;
    mln_status st = mln::validate(*p, err);
    if (st != MLN_OK) {
        mln::create_error() = err;
        return st;
    }
    size_t r = p->precision == MLN_FP64 ? 8 : 4;
    const int64_t D = p->N * p->N - 1;
    if (state_bytes) *state_bytes = static_cast<size_t>(D * mln::state_stride(*p)) * r;
    if (field_bytes) *field_bytes = static_cast<size_t>(p->n_cells) * r;
    return MLN_OK;
}

mln_status mln_setup_host(const mln_params *p, mln_setup *out) {
    if (!p || !out) return MLN_EINVAL;
    std::string err;
    mln_status st = mln::validate(*p, err);
    mln::Setup s;
    if (st == MLN_OK) st = mln::build_setup(*p, s, err);
    if (st != MLN_OK) {
        mln::create_error() = err;
        return st;
    }
    std::memset(out, 0, sizeof(*out));
    out->N = s.N;
    out->D = s.D;
    out->q = s.q;
    const int D = s.D;
    for (int i = 0; i < D * D; ++i) {
        out->M[i] = s.M[i];
        out->U[i] = s.U[i];
        out->A0[i] = s.A0[i];
        out->T[i] = s.T[i];
        out->C1[i] = s.C1[i];
    }
    for (int i = 0; i < D; ++i) {
        out->d_eq[i] = s.d_eq[i];
        out->v[i] = s.v[i];
        out->b[i] = s.b[i];
        out->w[i] = s.w[i];
        out->d0[i] = s.d0[i];
    }
    for (int i = 0; i < s.q; ++i) out->theta[i] = s.theta[i];
    out->c = s.c;
    for (size_t i = 0; i < s.gen.size(); ++i) {
        out->gen[2 * i] = s.gen[i].real();
        out->gen[2 * i + 1] = s.gen[i].imag();
    }
    return MLN_OK;
}

mln_status mln_lindblad_superop(int32_t N, const double *rates, const double *dephasing, double *G_out) {
    auto fail = [](const char *m) {
        mln::create_error() = m;
        return MLN_EINVAL;
    };
    if (N < MLN_MIN_N || N > MLN_MAX_N) return fail("N out of range");
    if (!G_out) return fail("G_out is NULL");
    for (int i = 0; i < N * N; ++i) {
        if (rates && !(std::isfinite(rates[i]) && rates[i] >= 0.0)) return fail("rates must be finite and >= 0");
        if (dephasing) {
            const int j = i / N, k = i % N;
            if (j == k) continue;
            if (!(std::isfinite(dephasing[i]) && dephasing[i] >= 0.0)) return fail("dephasing must be finite and >= 0");
            if (dephasing[i] != dephasing[k * N + j]) return fail("dephasing must be symmetric");
        }
    }
    const int n2 = N * N;
    std::fill(G_out, G_out + 2 * n2 * n2, 0.0);
    // real part of entry (row, col) of the superoperator; all entries are real
    auto at = [&](int j, int k, int l, int m) -> double & { return G_out[2 * ((j * N + k) * n2 + l * N + m)]; };
    if (rates) {
        for (int b = 0; b < N; ++b)
            for (int a = 0; a < N; ++a) {
                const double g = rates[b * N + a];
                if (g == 0.0) continue;
                at(a, a, b, b) += g;  // L rho L^+ = rho_bb |a><a|
                for (int m = 0; m < N; ++m) {
                    at(b, m, b, m) -= 0.5 * g;  // -(|b><b| rho) / 2
                    at(m, b, m, b) -= 0.5 * g;  // -(rho |b><b|) / 2
                }
            }
    }
    if (dephasing)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k)
                if (j != k) at(j, k, j, k) -= dephasing[j * N + k];
    return MLN_OK;
}

void mln_destroy(mln_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->st[1]);
    cudaFree(c->E[1]);
    cudaFree(c->H[1]);
    cudaFree(c->flags);
    cudaFree(c->tab_rho);
    cudaFree(c->tab_pop);
    cudaFree(c->tab_d);
    cudaFree(c->tab_in);
    cudaFree(c->scratch);
    cudaFree(c->prog);
    cudaFree(c->tc_img);
    cudaFree(c->adj_buf);
    mln::pstd_free(c);
    delete c;
}

mln_status mln_create(const mln_params *p, void *d_state, void *Ez, void *Hy, void *stream, mln_ctx **out) {
    if (out) *out = nullptr;
    if (!p || !out || !d_state || !Ez || !Hy) {
        mln::create_error() = "null argument";
        return MLN_EINVAL;
    }
    std::string err;
    mln_status st = mln::validate(*p, err);
    if (st != MLN_OK) {
        mln::create_error() = err;
        return st;
    }
    mln_ctx *c = new (std::nothrow) mln_ctx();
    if (!c) return MLN_ENOMEM;
    c->p = *p;
    c->p.H0 = c->p.mu = c->p.G = c->p.rho0 = nullptr;
    st = mln::build_setup(*p, c->s, err);
    if (st != MLN_OK) {
        mln::create_error() = err;
        delete c;
        return st;
    }
    c->D = c->s.D;
    c->n_med = p->medium_end - p->medium_begin;
    c->stride = mln::state_stride(*p);
    c->rsz = p->precision == MLN_FP64 ? 8 : 4;
    c->state_bytes = static_cast<size_t>(c->D) * c->stride * c->rsz;
    c->field_bytes = static_cast<size_t>(p->n_cells) * c->rsz;
    c->st[0] = d_state;
    c->E[0] = Ez;
    c->H[0] = Hy;
    c->stream = static_cast<cudaStream_t>(stream);
    // FP64 merged form under AUTO: the run-time compiled kernel on FDTD grids
    // when NVRTC is there (the same bits as the sparse model, measured faster:
    // three-level ring 4.34e9 against 4.28e9, two-level SIT 1.27e9 against
    // 8.3e8 cell-updates/s), else and for PSTD the sparse model
    const bool auto64 = p->kernel == MLN_KERNEL_AUTO && p->precision == MLN_FP64 && p->form == MLN_FORM_MERGED;
    const bool auto64_jit = auto64 && p->maxwell == MLN_MAXWELL_FDTD && mln::jit_available(nullptr);
    c->sparse = p->kernel == MLN_KERNEL_SPARSE || (auto64 && !auto64_jit);
    auto fail = [&](mln_status s_) {
        mln::create_error() = c->err.empty() ? err : c->err;
        mln_destroy(c);
        return s_;
    };
    bool ok;
    if (c->sparse) {
        std::vector<int32_t> rowptr, cols;
        std::vector<double> vals;
        mln::build_sparse_program(c->s, rowptr, cols, vals);
        c->nnz = static_cast<int>(vals.size());
        c->nrowptr = static_cast<int>(rowptr.size());
        // the kernel indexes rows by this layout: check it before anything reaches the device
        const int P = 2 * c->s.q, D = c->s.D;
        bool layout_ok = c->nrowptr == P + 2 * D + 2 && rowptr.front() == 0 && rowptr.back() == c->nnz;
        for (size_t r = 0; layout_ok && r + 1 < rowptr.size(); ++r) {
            const int lim = (static_cast<int>(r) >= P && static_cast<int>(r) < P + D) ? P : D;
            layout_ok = rowptr[r] <= rowptr[r + 1];
            for (int e = rowptr[r]; layout_ok && e < rowptr[r + 1]; ++e) layout_ok = cols[e] >= 0 && cols[e] < lim;
        }
        if (!layout_ok) {
            c->err = "sparse program layout check failed";
            return fail(MLN_ENUMERIC);
        }
        size_t b_rp = rowptr.size() * 4, b_cols = cols.size() * 4;
        size_t off_vals = (b_rp + b_cols + 15) / 16 * 16;
        size_t bytes = off_vals + vals.size() * 8 + 16;
        std::vector<unsigned char> host(bytes, 0);
        std::memcpy(host.data(), rowptr.data(), b_rp);
        std::memcpy(host.data() + b_rp, cols.data(), b_cols);
        std::memcpy(host.data() + off_vals, vals.data(), vals.size() * 8);
        if (cudaMalloc(&c->prog, bytes) != cudaSuccess ||
            cudaMemcpy(c->prog, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            c->err = "upload of the sparse program failed";
            return fail(MLN_ENOMEM);
        }
        unsigned char *base = static_cast<unsigned char *>(c->prog);
        ok = mln::pack_sparse_consts(c->s, p->dt, reinterpret_cast<const int32_t *>(base),
                                     reinterpret_cast<const int32_t *>(base + b_rp),
                                     reinterpret_cast<const double *>(base + off_vals), c->nnz, c->nrowptr, c->consts);
        c->max_threads = sparse_max_threads(c);
        if (c->max_threads < 64) {
            c->err = "sparse program does not fit in shared memory";
            return fail(MLN_EUNSUPPORTED);
        }
    } else if (p->kernel == MLN_KERNEL_TENSOR ||
               (p->kernel == MLN_KERNEL_AUTO && p->precision == MLN_FP32 &&
                (p->form == MLN_FORM_MERGED || p->form == MLN_FORM_ROTATED) && p->maxwell == MLN_MAXWELL_FDTD &&
                mln::tc_supported(p->N))) {
        std::vector<unsigned char> img;
        c->tcr = p->form == MLN_FORM_ROTATED;
        ok = mln::tc_supported(p->N) && (c->tcr ? mln::pack_tcr(c->s, p->dt, img, c->tc_scal)
                                                 : mln::pack_tc(c->s, p->dt, img, c->tc_scal));
        if (ok) {
            if (cudaMalloc(&c->tc_img, img.size()) != cudaSuccess ||
                cudaMemcpy(c->tc_img, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
                cudaGetLastError();
                c->err = "upload of the tensor-core operands failed";
                return fail(MLN_ENOMEM);
            }
            c->tc = MLN_KERNEL_TENSOR;
        }
    } else {
        ok = p->precision == MLN_FP64 ? mln::pack_consts(c->s, p->form, p->dt, 0.0, c->consts)
                                      : mln::pack_consts(c->s, p->form, p->dt, 0.0f, c->consts);
        // the rotated form exists only as a run-time compiled kernel
        const bool rotated = p->form == MLN_FORM_ROTATED;
        const bool want_jit = p->kernel == MLN_KERNEL_JIT || rotated || auto64_jit ||
                              (p->kernel == MLN_KERNEL_AUTO && p->precision == MLN_FP32 && p->form == MLN_FORM_MERGED &&
                               p->maxwell == MLN_MAXWELL_FDTD);
        if (ok && p->kernel == MLN_KERNEL_DF32) {
            // the step in double-float arithmetic: run-time compiled or nothing
            std::string why, log;
            cudaError_t e = cudaErrorNotSupported;
            if (!mln::df_constants_in_range(c->s, p->dt, rotated)) {
                c->err = "MLN_KERNEL_DF32: a constant of the step is outside the double-float range";
                return fail(MLN_EUNSUPPORTED);
            }
            if (mln::jit_available(&why))
                e = mln::jit_compile(mln::jit_df_source(c->s, p->dt, mln::jit_body_flags(*p), rotated), &c->jit_fn,
                                     log);
            else
                log = why;
            if (e != cudaSuccess) {
                c->jit_fn = nullptr;
                c->err = "double-float kernel unavailable: " + log;
                return fail(MLN_EUNSUPPORTED);
            }
            c->df32 = true;
            c->max_threads = mln::df_threads(c->s.D, rotated);
        } else if (ok && want_jit) {
            std::string why, log;
            cudaError_t e = cudaErrorNotSupported;
            if (mln::jit_available(&why))
                e = mln::jit_compile(mln::jit_merged_source(c->s, p->dt, p->precision == MLN_FP32, rotated,
                                                            mln::jit_body_flags(*p)),
                                     &c->jit_fn, log);
            else
                log = why;
            if (e != cudaSuccess) {
                c->jit_fn = nullptr;
                if (p->kernel == MLN_KERNEL_JIT || rotated) {
                    c->err = "run-time compiled kernel unavailable: " + log;
                    return fail(MLN_EUNSUPPORTED);
                }
            }
        }
    }
    if (!ok) {
        c->err = "no kernel for this N";
        return fail(MLN_EUNSUPPORTED);
    }
    pick_launch_shape(c);
    if (cudaMalloc(&c->st[1], std::max<size_t>(c->state_bytes, 16)) != cudaSuccess ||
        cudaMalloc(&c->E[1], c->field_bytes) != cudaSuccess || cudaMalloc(&c->H[1], c->field_bytes) != cudaSuccess ||
        cudaMalloc(&c->flags, 256) != cudaSuccess) {
        cudaGetLastError();
        c->err = "device allocation failed";
        return fail(MLN_ENOMEM);
    }
    if (cudaMemsetAsync(c->flags, 0, 256, c->stream) != cudaSuccess) {
        c->err = "flag reset failed";
        return fail(MLN_ECUDA);
    }
    if (p->maxwell == MLN_MAXWELL_PSTD && (st = mln::pstd_init(c)) != MLN_OK) return fail(st);
    // output tables: rho = rho_c + Z (sd0 + Sd s), populations, d = sd0 + Sd s
    const int D = c->D, n = p->N, nn = n * n;
    std::vector<double> zr((size_t)2 * nn * D, 0.0), zo(2 * nn, 0.0);
    for (int r = 0; r < 2 * nn; ++r) {
        double o = c->s.rho_c[r];
        for (int j = 0; j < D; ++j) o += c->s.Z[r * D + j] * c->s.sd0[j];
        zo[r] = o;
        for (int k = 0; k < D; ++k) {
            double acc = 0;
            for (int j = 0; j < D; ++j) acc += c->s.Z[r * D + j] * c->s.Sd[j * D + k];
            zr[(size_t)r * D + k] = acc;
        }
    }
    std::vector<double> pr((size_t)n * D), po(n);
    for (int l = 0; l < n; ++l) {
        int r = 2 * (l * n + l);
        po[l] = zo[r];
        for (int k = 0; k < D; ++k) pr[(size_t)l * D + k] = zr[(size_t)r * D + k];
    }
    if ((st = upload_table(c, &c->tab_rho, zr, zo)) != MLN_OK) return fail(st);
    if ((st = upload_table(c, &c->tab_pop, pr, po)) != MLN_OK) return fail(st);
    if ((st = upload_table(c, &c->tab_d, c->s.Sd, c->s.sd0)) != MLN_OK) return fail(st);
    if ((st = upload_table(c, &c->tab_in, c->s.Sp, c->s.sp0)) != MLN_OK) return fail(st);
    // initial medium state from rho0: state = sp0 + Sp d0
    if (c->n_med > 0) {
        std::vector<double> v0(D);
        for (int k = 0; k < D; ++k) {
            double acc = c->s.sp0[k];
            for (int j = 0; j < D; ++j) acc += c->s.Sp[k * D + j] * c->s.d0[j];
            v0[k] = acc;
        }
        if ((st = ensure_scratch(c, D * sizeof(double))) != MLN_OK) return fail(st);
        if (cudaMemcpy(c->scratch, v0.data(), D * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            c->err = "upload of the initial state failed";
            return fail(MLN_ECUDA);
        }
        if (p->precision == MLN_FP64)
            fill_state<double><<<grid_for(c->n_med, 256), 256, 0, c->stream>>>(
                static_cast<double *>(c->st[0]), c->stride, c->n_med, D, static_cast<double *>(c->scratch));
        else
            fill_state<float><<<grid_for(c->n_med, 256), 256, 0, c->stream>>>(
                static_cast<float *>(c->st[0]), c->stride, c->n_med, D, static_cast<double *>(c->scratch));
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
            c->err = "initial state kernel failed";
            return fail(MLN_ECUDA);
        }
    }
    *out = c;
    return MLN_OK;
}

mln_status mln_step(mln_ctx *c, int64_t n_steps, const double *src) {
    if (!c || n_steps < 0) return MLN_EINVAL;
    if (n_steps == 0) return MLN_OK;
    mln_status st = c->p.precision == MLN_FP64 ? run_steps<double>(c, n_steps, src) : run_steps<float>(c, n_steps, src);
    if (st == MLN_OK) c->steps += n_steps;
    return st;
}

mln_status mln_sync(mln_ctx *c) {
    if (!c) return MLN_EINVAL;
    MLN_CK(c, cudaStreamSynchronize(c->stream));
    unsigned int f = 0;
    MLN_CK(c, cudaMemcpy(&f, c->flags, sizeof(f), cudaMemcpyDeviceToHost));
    if (f & 2u) {
        c->err = "a tensor-core kernel gave up waiting for an MMA to complete";
        MLN_CK(c, cudaMemset(c->flags, 0, sizeof(unsigned int)));
        return MLN_ETIMEOUT;
    }
    if (f & 4u) {
        c->err = "a persistent batch kernel gave up waiting for a neighbouring tile";
        MLN_CK(c, cudaMemset(c->flags, 0, sizeof(unsigned int)));
        return MLN_ETIMEOUT;
    }
    if (f & 1u) {
        c->err = "non-finite E_z on the device";
        MLN_CK(c, cudaMemset(c->flags, 0, sizeof(unsigned int)));
        return MLN_ENONFINITE;
    }
    return MLN_OK;
}

int64_t mln_step_count(const mln_ctx *c) { return c ? c->steps : -1; }

int64_t mln_launch_count(const mln_ctx *c) { return c ? c->launches : -1; }

int32_t mln_kernel_in_use(const mln_ctx *c) {
    if (!c) return -1;
    if (c->tc) return c->tc;
    if (c->df32) return MLN_KERNEL_DF32;
    return c->jit_fn ? MLN_KERNEL_JIT : c->sparse ? MLN_KERNEL_SPARSE : MLN_KERNEL_REGISTER;
}

mln_status mln_autotune(mln_ctx *c, int32_t trials, int32_t *block_steps, int32_t *tile_cells) {
    if (!c || trials < 1) return MLN_EINVAL;
    MLN_CK(c, cudaStreamSynchronize(c->stream));
    mln_status st = c->p.precision == MLN_FP64 ? autotune_t<double>(c, trials) : autotune_t<float>(c, trials);
    if (block_steps) *block_steps = c->K;
    if (tile_cells) *tile_cells = c->tile;
    return st;
}

mln_status mln_work_per_step(const mln_ctx *c, double *flops_medium, double *flops_cell, double *bytes_medium,
                             double *bytes_cell) {
    if (!c) return MLN_EINVAL;
    const mln::Setup &s = c->s;
    const int D = s.D, q = s.q, N = s.N, P = 2 * q;
    auto nz = [](const std::vector<double> &v, int rows, int cols, int ld, double diag) {
        double n = 0;
        for (int i = 0; i < rows; ++i)
            for (int j = 0; j < cols; ++j) n += (v[i * ld + j] - (i == j ? diag : 0.0)) != 0.0;
        return n;
    };
    // Exact operation counts of the method on this input (FMA = 2 flops): a
    // product row with k non-zero entries is k multiplications and k - 1
    // additions; added onto a vector, k additions; a non-zero offset, one more.
    const double nT = nz(s.T, D, P, D, 0.0);          // T on the plane columns (= T^T on the plane rows)
    double planes_used = 0;                           // plane rows of T^T with a non-zero entry
    for (int k = 0; k < P; ++k) {
        bool any = false;
        for (int i = 0; i < D; ++i) any = any || s.T[i * D + k] != 0.0;
        planes_used += any;
    }
    auto dot = [&](const std::vector<double> &w, double c0) {  // c0 + w . x
        const double k = nz(w, 1, D, D, 0.0);
        return k > 0 ? 2 * k - 1 + (c0 != 0.0) : 0.0;
    };
    // the N - 1 series for (sin, cos - 1), the other planes by the subtraction
    // formulas (10 flops), and 6 flops per plane for the increment
    const double rot = 6.0 * q + 10.0 * (q - (N - 1)) + 8.0 * (N - 1);
    const double tt = 2 * nT - planes_used;           // z = T^T y
    double f;
    if (c->p.form == MLN_FORM_MERGED) {
        // y'' = y + T dz; dP/dt = c' + wm . y''; y = (y'' + b2) + C1 y''
        f = tt + rot + 2 * nT + dot(s.wm, s.cm) + 2 * nz(s.C1, D, D, D, 0.0) + nz(s.b2, 1, D, D, 0.0);
    } else if (c->p.form == MLN_FORM_ROTATED) {
        // z'' = z + dz on the P plane coordinates; dP/dt = cm + wz . z'';
        // z = (z'' + cz) + C1z z''
        f = P + rot + dot(s.wz, s.cm) + 2 * nz(s.C1z, D, D, D, 0.0) + nz(s.cz, 1, D, D, 0.0);
    } else {
        // d' = d + ((A0 - I) d + b), twice per step
        const double half = 2 * nz(s.A0, D, D, D, 1.0) + nz(s.b, 1, D, D, 0.0);
        if (c->p.form == MLN_FORM_RODRIGUES) {
            // per plane: S_k d' and S_k^2 d' (dense, 2 D^2 each) and the two scaled adds (4 D)
            f = 2 * half + dot(s.w, s.c) + q * (4.0 * D * D + 4.0 * D) + (rot - 6.0 * q);
        } else {
            f = 2 * half + tt + rot + 2 * nT + dot(s.w, s.c);
        }
    }
    if (flops_medium) *flops_medium = f;
    if (flops_cell) *flops_cell = 9.0;
    if (bytes_medium) *bytes_medium = 2.0 * (2 + D) * c->rsz;
    if (bytes_cell) *bytes_cell = 2.0 * 2 * c->rsz;
    return MLN_OK;
}

mln_status mln_launch_shape(const mln_ctx *c, int32_t *block_steps, int32_t *tile_cells, int32_t *threads) {
    if (!c) return MLN_EINVAL;
    if (block_steps) *block_steps = c->K;
    if (tile_cells) *tile_cells = c->tile;
    if (threads) *threads = c->threads;
    return MLN_OK;
}

mln_status mln_get_fields(mln_ctx *c, double *Ez_host, double *Hy_host) {
    if (!c) return MLN_EINVAL;
    mln_status st = MLN_OK;
    if (Ez_host && (st = read_field(c, c->E[0], Ez_host)) != MLN_OK) return st;
    if (Hy_host && (st = read_field(c, c->H[0], Hy_host)) != MLN_OK) return st;
    return MLN_OK;
}

mln_status mln_get_rho(mln_ctx *c, int64_t cell0, int64_t count, double *rho_host) {
    if (!c || (!rho_host && count > 0)) return MLN_EINVAL;
    int64_t m0;
    mln_status st = check_cells(c, cell0, count, &m0);
    if (st != MLN_OK) return st;
    return read_rows(c, m0, count, c->tab_rho, 2 * c->p.N * c->p.N, rho_host);
}

mln_status mln_get_populations(mln_ctx *c, int64_t cell0, int64_t count, double *pop_host) {
    if (!c || (!pop_host && count > 0)) return MLN_EINVAL;
    int64_t m0;
    mln_status st = check_cells(c, cell0, count, &m0);
    if (st != MLN_OK) return st;
    return read_rows(c, m0, count, c->tab_pop, c->p.N, pop_host);
}

mln_status mln_save_state(mln_ctx *c, double *d_host, double *Ez_host, double *Hy_host) {
    if (!c) return MLN_EINVAL;
    mln_status st;
    if (d_host && (st = read_rows(c, 0, c->n_med, c->tab_d, c->D, d_host)) != MLN_OK) return st;
    return mln_get_fields(c, Ez_host, Hy_host);
}

mln_status mln_load_state(mln_ctx *c, const double *d_host, const double *Ez_host, const double *Hy_host) {
    if (!c) return MLN_EINVAL;
    mln_status st;
    if (d_host && c->n_med > 0) {
        size_t bytes = static_cast<size_t>(c->n_med) * c->D * sizeof(double);
        if ((st = ensure_scratch(c, bytes)) != MLN_OK) return st;
        MLN_CK(c, cudaMemcpyAsync(c->scratch, d_host, bytes, cudaMemcpyHostToDevice, c->stream));
        if (c->p.precision == MLN_FP64)
            rows_to_state<double><<<grid_for(c->n_med, 128), 128, 0, c->stream>>>(
                static_cast<const double *>(c->scratch), c->n_med, c->D, c->tab_in, static_cast<double *>(c->st[0]),
                c->stride);
        else
            rows_to_state<float><<<grid_for(c->n_med, 128), 128, 0, c->stream>>>(
                static_cast<const double *>(c->scratch), c->n_med, c->D, c->tab_in, static_cast<float *>(c->st[0]),
                c->stride);
        MLN_CK(c, cudaGetLastError());
        MLN_CK(c, cudaStreamSynchronize(c->stream));
    }
    if (Ez_host && (st = write_field(c, c->E[0], Ez_host)) != MLN_OK) return st;
    if (Hy_host && (st = write_field(c, c->H[0], Hy_host)) != MLN_OK) return st;
    return MLN_OK;
}

}  // extern "C"
