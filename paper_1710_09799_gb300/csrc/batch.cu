// Batched solver: many independent grids (any mix of N = 2..4, lengths and
// boundaries, one precision) advanced together. Two launch structures, each
// captured once per mln_batch_step call into a CUDA graph and replayed:
// every K steps one launch per N present covering every tile of every grid
// with that N (MLN_BATCH_CHUNKS), or one persistent launch per N for all the
// call's K-step chunks, tiles waiting on their neighbours' progress counters
// (MLN_BATCH_PERSISTENT, run-time compiled kernels only).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "dispatch.cuh"
#include "jit.h"
#include "mln.h"
#include "setup.h"

namespace mln {

// Merged-form constants of one grid with every row padded to a whole number
// of 16-byte vectors, and T also stored transposed, so that each product
// reads its row with vector loads from shared memory.
template <int N, typename R>
struct PaddedConsts {
    static constexpr int D = Dims<N>::D, V = 16 / static_cast<int>(sizeof(R)), DP = (D + V - 1) / V * V;
    R C1[D * DP];  // C1[i * DP + j] = (A0^2 - I)_ij
    R T[D * DP];   // T[i * DP + j] = T_ij
    R Tt[D * DP];  // Tt[k * DP + i] = T_ik
    R b2[DP];
    R wm[DP];
    R psi_dt[N - 1];
    R cm;
};

template <typename R>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int n = 4;
    __device__ __forceinline__ static void get(const float *p, float (&o)[4]) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
};
template <>
struct Vec<double> {
    static constexpr int n = 2;
    __device__ __forceinline__ static void get(const double *p, double (&o)[2]) {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        o[0] = v.x;
        o[1] = v.y;
    }
};

// sum_j row[j] x[j] in ascending j, as the dense products of the register
// model: starting from row[0] x[0] (first_mul) or as fma's onto acc.
template <int D, bool first_mul, typename R>
__device__ __forceinline__ R dot_row(const R *row, const R (&x)[D], R acc) {
    constexpr int V = Vec<R>::n;
#pragma unroll
    for (int j0 = 0; j0 < D; j0 += V) {
        R c[V];
        Vec<R>::get(row + j0, c);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const int j = j0 + e;
            if (j < D) acc = (first_mul && j == 0) ? c[e] * x[0] : fma(c[e], x[j], acc);
        }
    }
    return acc;
}

// The register cell model's merged step (same operations in the same order,
// hence the same bits) with the constants read from the padded layout.
template <int N, typename R>
struct PaddedCell {
    static constexpr int D = Dims<N>::D;
    using Consts = PaddedConsts<N, R>;
    static constexpr int DP = Consts::DP;
    R s[D];
    __device__ __forceinline__ void setup(unsigned char *, const Consts &) {}
    __device__ __forceinline__ void load(const R *src, int64_t stride, int64_t m) {
#pragma unroll
        for (int i = 0; i < D; ++i) s[i] = src[i * stride + m];
    }
    __device__ __forceinline__ void store(R *dst, int64_t stride, int64_t m) const {
#pragma unroll
        for (int i = 0; i < D; ++i) dst[i * stride + m] = s[i];
    }
    __device__ __forceinline__ R step(R e, const Consts &k) {
        R z[D];
#pragma unroll
        for (int c = 0; c < D; ++c) z[c] = dot_row<D, true>(k.Tt + c * DP, s, R(0));  // z = T^T y
        rotation_increment<N>(z, k.psi_dt, e);
#pragma unroll
        for (int i = 0; i < D; ++i) {  // y + T (R - I) z: onto y in FP64, the increment first in FP32
            if constexpr (sizeof(R) == 8) s[i] = dot_row<D, false>(k.T + i * DP, z, s[i]);
            else s[i] = s[i] + dot_row<D, true>(k.T + i * DP, z, R(0));
        }
        const R dpdt = dot_row<D, false>(k.wm, s, k.cm);
#pragma unroll
        for (int i = 0; i < D; ++i) {  // (y'' + b2) + C1 y'' in FP64; y'' + (C1 y'' + b2) in FP32
            if constexpr (sizeof(R) == 8) z[i] = dot_row<D, false>(k.C1 + i * DP, s, s[i] + k.b2[i]);
            else z[i] = s[i] + dot_row<D, false>(k.C1 + i * DP, s, k.b2[i]);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) s[i] = z[i];
        return dpdt;
    }
    __device__ __forceinline__ void end_step() {}
};

// One block per work item (grid, tile) of the grids with N levels; one kernel
// per N, so that each gets the registers of its own cell size. The grid's
// constants are staged in shared memory (padded rows read with 16-byte
// vector loads; every thread of a warp reads the same entry: broadcasts).
template <int N, typename R>
__global__ void __launch_bounds__(kBatchThreads, 1)
    mln_batch_kernel(const BatchGrid<R> *__restrict__ grids, const BatchItem *__restrict__ items,
                     const unsigned char *__restrict__ consts, int parity, int nsteps, int halo, int tile,
                     int64_t step_offset) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    batch_body<N, R, PaddedCell<N, R>>(grids, items, consts, parity, nsteps, halo, tile, step_offset, smem_raw);
}

}  // namespace mln

struct mln_batch {
    std::vector<mln_ctx *> ctx;
    int precision = MLN_FP32;
    cudaStream_t user = nullptr;     // the caller's stream (may be the legacy default stream)
    cudaStream_t stream = nullptr;   // the batch's own stream: graphs are captured and replayed here
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int K = 16, tile = 256, threads = 288;
    int64_t steps = 0, src_len = 0, launches = 0;
    std::vector<const double *> src;
    void *d_grids = nullptr, *d_items = nullptr, *d_consts = nullptr;
    int64_t n_items = 0;
    int64_t item_off[mln::kBatchMaxN + 1] = {}, item_cnt[mln::kBatchMaxN + 1] = {};  // work items by N
    // per N: run-time compiled kernel over the union sparsity pattern (or
    // nullptr: the padded-constant kernel)
    void *jit[mln::kBatchMaxN + 1] = {};
    void *jitp[mln::kBatchMaxN + 1] = {};  // the persistent kernel of the same module
    mln::BatchPattern pat[mln::kBatchMaxN + 1];
    bool df32 = false;                  // FP64 grids stepped in double-float pairs (MLN_KERNEL_DF32)
    int mode = MLN_BATCH_CHUNKS;
    int wait_limit = 1 << 22;           // polls of a persistent block's wait (about 0.4 s at 100 ns each)
    void *d_work = nullptr;             // persistent: one work counter per N
    void *d_progress = nullptr;         // persistent: chunks completed per work item
    // captured launch sequences, by step count
    std::map<int64_t, cudaGraphExec_t> graphs;
    std::string err;
};

namespace {

#define MLN_BCK(b, call)                                                        \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            (b)->err = std::string(#call) + ": " + cudaGetErrorString(e_);      \
            return MLN_ECUDA;                                                   \
        }                                                                       \
    } while (0)

void drop_graphs(mln_batch *b) {
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// Padded constants of one grid from its context's merged-form constants
// (the same values, rearranged).
template <int N, typename R>
bool pad_consts_t(const std::vector<unsigned char> &merged, std::vector<unsigned char> &out) {
    using M = mln::MergedConsts<N, R>;
    using P = mln::PaddedConsts<N, R>;
    static_assert(sizeof(P) <= mln::kBatchConstsMax, "padded constants exceed the shared-memory room");
    if (merged.size() != sizeof(M)) return false;
    M m;
    std::memcpy(&m, merged.data(), sizeof(M));
    P p;
    std::memset(&p, 0, sizeof(P));
    constexpr int D = P::D, DP = P::DP;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            p.C1[i * DP + j] = m.C1[i * D + j];
            p.T[i * DP + j] = m.T[i * D + j];
            p.Tt[j * DP + i] = m.T[i * D + j];
        }
    for (int i = 0; i < D; ++i) {
        p.b2[i] = m.b2[i];
        p.wm[i] = m.wm[i];
    }
    for (int a = 0; a < N - 1; ++a) p.psi_dt[a] = m.psi_dt[a];
    p.cm = m.cm;
    out.resize(sizeof(P));
    std::memcpy(out.data(), &p, sizeof(P));
    return true;
}

template <typename R>
bool pad_consts(int N, const std::vector<unsigned char> &merged, std::vector<unsigned char> &out) {
    switch (N) {
    case 2: return pad_consts_t<2, R>(merged, out);
    case 3: return pad_consts_t<3, R>(merged, out);
    case 4: return pad_consts_t<4, R>(merged, out);
    default: return false;
    }
}

// Grid table and work list for the current tile size: the tiles of the
// grids with N levels form one contiguous run per N (largest N first), the
// work of one launch of that N's kernel.
template <typename R>
mln_status build_tables(mln_batch *b) {
    std::vector<mln::BatchGrid<R>> grids;
    std::vector<unsigned char> blob;
    std::vector<std::pair<int, mln::BatchItem>> items;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        mln_ctx *c = b->ctx[i];
        mln::BlockArgs<R> a = mln::base_args<R>(c);
        mln::BatchGrid<R> g{};
        for (int s = 0; s < 2; ++s) {
            g.E[s] = static_cast<R *>(c->E[s]);
            g.H[s] = static_cast<R *>(c->H[s]);
            g.S[s] = static_cast<R *>(c->st[s]);
        }
        g.src = (b->src.empty() || c->p.source_kind == MLN_SRC_NONE) ? nullptr : b->src[i];
        g.flags = c->flags;
        g.n_cells = c->p.n_cells;
        g.mb = c->p.medium_begin;
        g.me = c->p.medium_end;
        g.stride = c->stride;
        g.source_cell = c->p.source_cell;
        g.N = c->p.N;
        g.boundary = c->p.boundary;
        g.source_kind = c->p.source_kind;
        std::vector<unsigned char> padded;
        if (b->jit[c->p.N]) {
            mln::batch_pack(b->pat[c->p.N], c->s, c->p.dt, sizeof(R) == 4, padded, b->df32);
        } else if (!pad_consts<R>(c->p.N, c->consts, padded)) {
            b->err = "batch: no padded constants for this N";
            return MLN_EUNSUPPORTED;
        }
        if (padded.size() > static_cast<size_t>(mln::kBatchConstsMax)) {
            b->err = "batch: constants of grid " + std::to_string(i) + " exceed the shared-memory room";
            return MLN_EUNSUPPORTED;
        }
        g.consts_off = static_cast<int32_t>(blob.size());
        g.consts_bytes = static_cast<int32_t>((padded.size() + 15) / 16 * 16);
        g.ch = a.ch;
        g.ca = a.ca;
        g.cb = a.cb;
        g.inv_dx = a.inv_dx;
        g.kappa = a.kappa;
        blob.insert(blob.end(), padded.begin(), padded.end());
        blob.resize((blob.size() + 15) / 16 * 16, 0);
        grids.push_back(g);
        const int64_t nt = (c->p.n_cells + b->tile - 1) / b->tile;
        for (int64_t t = 0; t < nt; ++t)
            items.push_back({c->p.N, mln::BatchItem{static_cast<int32_t>(i), static_cast<int32_t>(t)}});
    }
    std::stable_sort(items.begin(), items.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    std::vector<mln::BatchItem> list;
    for (int N = 0; N <= mln::kBatchMaxN; ++N) b->item_off[N] = b->item_cnt[N] = 0;
    for (size_t k = 0; k < items.size(); ++k) {
        const int N = items[k].first;
        if (b->item_cnt[N] == 0) b->item_off[N] = static_cast<int64_t>(k);
        ++b->item_cnt[N];
        list.push_back(items[k].second);
    }
    cudaFree(b->d_grids);
    cudaFree(b->d_items);
    cudaFree(b->d_consts);
    cudaFree(b->d_progress);
    b->d_grids = b->d_items = b->d_consts = b->d_progress = nullptr;
    MLN_BCK(b, cudaMalloc(&b->d_progress, std::max<size_t>(list.size(), 1) * sizeof(int)));
    if (!b->d_work) MLN_BCK(b, cudaMalloc(&b->d_work, (mln::kBatchMaxN + 1) * sizeof(unsigned long long)));
    MLN_BCK(b, cudaMalloc(&b->d_grids, grids.size() * sizeof(grids[0])));
    MLN_BCK(b, cudaMalloc(&b->d_items, list.size() * sizeof(list[0])));
    MLN_BCK(b, cudaMalloc(&b->d_consts, std::max<size_t>(blob.size(), 16)));
    MLN_BCK(b, cudaMemcpy(b->d_grids, grids.data(), grids.size() * sizeof(grids[0]), cudaMemcpyHostToDevice));
    MLN_BCK(b, cudaMemcpy(b->d_items, list.data(), list.size() * sizeof(list[0]), cudaMemcpyHostToDevice));
    MLN_BCK(b, cudaMemcpy(b->d_consts, blob.data(), blob.size(), cudaMemcpyHostToDevice));
    b->n_items = static_cast<int64_t>(list.size());
    return MLN_OK;
}

template <typename R>
size_t batch_smem(int threads) {
    return mln::kBatchConstsMax + mln::field_smem<R>(threads);
}

template <int N, typename R>
cudaError_t launch_batch_n(mln_batch *b, int parity, int nsteps, int64_t step_offset) {
    if (b->item_cnt[N] == 0) return cudaSuccess;
    // at most 8 KB + 4 x 256 x 8 B = 16 KB: below the 48 KB default, no attribute needed
    const size_t smem = batch_smem<R>(b->threads);
    if (b->jit[N])
        return mln::jit_launch_batch(b->jit[N], b->d_grids, static_cast<const mln::BatchItem *>(b->d_items) + b->item_off[N],
                                     b->d_consts, parity, nsteps, b->K, b->tile, step_offset,
                                     static_cast<unsigned>(b->item_cnt[N]), b->threads, smem, b->stream);
    mln::mln_batch_kernel<N, R><<<static_cast<unsigned>(b->item_cnt[N]), b->threads, smem, b->stream>>>(
        static_cast<const mln::BatchGrid<R> *>(b->d_grids),
        static_cast<const mln::BatchItem *>(b->d_items) + b->item_off[N],
        static_cast<const unsigned char *>(b->d_consts), parity, nsteps, b->K, b->tile, step_offset);
    return cudaGetLastError();
}

// One launch per N present (largest first), all on the batch's stream.
template <typename R>
cudaError_t launch_batch(mln_batch *b, int parity, int nsteps, int64_t step_offset) {
    cudaError_t e = launch_batch_n<4, R>(b, parity, nsteps, step_offset);
    if (e == cudaSuccess) e = launch_batch_n<3, R>(b, parity, nsteps, step_offset);
    if (e == cudaSuccess) e = launch_batch_n<2, R>(b, parity, nsteps, step_offset);
    return e;
}

int batch_kernels(const mln_batch *b) {
    int k = 0;
    for (int N = 2; N <= mln::kBatchMaxN; ++N) k += b->item_cnt[N] > 0;
    return k;
}

// One persistent launch of every chunk of n_steps steps for the items of
// one N: counters reset, then the kernel (blocks beyond what fits on the GPU
// wait to start and take the remaining items).
template <int N, typename R>
cudaError_t launch_persist_n(mln_batch *b, int64_t n_steps) {
    if (b->item_cnt[N] == 0) return cudaSuccess;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    mln::BatchPersist p{};
    p.work = static_cast<unsigned long long *>(b->d_work) + N;
    p.progress = static_cast<int *>(b->d_progress) + b->item_off[N];
    p.n_items = b->item_cnt[N];
    p.n_chunks = static_cast<int32_t>((n_steps + b->K - 1) / b->K);
    p.K = b->K;
    p.last_steps = static_cast<int32_t>(n_steps - static_cast<int64_t>(p.n_chunks - 1) * b->K);
    p.wait_limit = b->wait_limit;
    cudaError_t e = cudaMemsetAsync(p.work, 0, sizeof(unsigned long long), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.progress, 0, p.n_items * sizeof(int), b->stream);
    if (e != cudaSuccess) return e;
    const int64_t total = static_cast<int64_t>(p.n_chunks) * p.n_items;
    const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(total, static_cast<int64_t>(sms) * 8));
    const size_t smem = batch_smem<R>(b->threads);
    return mln::jit_launch_batch_persist(b->jitp[N], b->d_grids,
                                         static_cast<const mln::BatchItem *>(b->d_items) + b->item_off[N],
                                         b->d_consts, b->K, b->tile, b->steps, p, blocks, b->threads, smem, b->stream);
}

// Queue the launches of n_steps steps from the batch's current step count;
// the result ends in buffer set 0 of every grid.
template <typename R>
mln_status queue_steps(mln_batch *b, int64_t n_steps) {
    int parity = 0;
    if (b->mode == MLN_BATCH_PERSISTENT) {
        MLN_BCK(b, (launch_persist_n<4, R>(b, n_steps)));
        MLN_BCK(b, (launch_persist_n<3, R>(b, n_steps)));
        MLN_BCK(b, (launch_persist_n<2, R>(b, n_steps)));
        parity = static_cast<int>(((n_steps + b->K - 1) / b->K) & 1);
    } else {
        for (int64_t done = 0; done < n_steps;) {
            int ns = static_cast<int>(std::min<int64_t>(b->K, n_steps - done));
            MLN_BCK(b, launch_batch<R>(b, parity, ns, b->steps + done));
            parity ^= 1;
            done += ns;
        }
    }
    if (parity == 1) {
        for (mln_ctx *c : b->ctx) {
            MLN_BCK(b, cudaMemcpyAsync(c->st[0], c->st[1], c->state_bytes, cudaMemcpyDeviceToDevice, b->stream));
            MLN_BCK(b, cudaMemcpyAsync(c->E[0], c->E[1], c->field_bytes, cudaMemcpyDeviceToDevice, b->stream));
            MLN_BCK(b, cudaMemcpyAsync(c->H[0], c->H[1], c->field_bytes, cudaMemcpyDeviceToDevice, b->stream));
        }
    }
    return MLN_OK;
}

template <typename R>
mln_status autotune_batch(mln_batch *b, int trials) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int Ks[] = {4, 8, 12, 16, 24, 32, 48, 64};
    const int tiles[] = {64, 128, 192, 256, 320, 384, 448};
    cudaEvent_t e0, e1;
    MLN_BCK(b, cudaEventCreate(&e0));
    MLN_BCK(b, cudaEventCreate(&e1));
    double best = 1e300;
    int bestK = b->K, bestTile = b->tile;
    for (int K : Ks)
        for (int tile : tiles) {
            // tiles longer than their halo (+ 1 for a tile made of a Mur cell): a tile's
            // halo covers only its two neighbours (the persistent launch relies on it)
            if (tile + 2 * K > mln::kBatchThreads || tile < K + 2) continue;
            b->K = K;
            b->tile = tile;
            b->threads = (tile + 2 * K + 31) / 32 * 32;
            mln_status st = build_tables<R>(b);
            if (st != MLN_OK) return st;
            // parity 0 reads the caller's buffers and writes the contexts': no state changes
            if (launch_batch<R>(b, 0, K, 0) != cudaSuccess) continue;
            MLN_BCK(b, cudaEventRecord(e0, b->stream));
            for (int t = 0; t < trials; ++t) MLN_BCK(b, launch_batch<R>(b, 0, K, 0));
            MLN_BCK(b, cudaEventRecord(e1, b->stream));
            MLN_BCK(b, cudaEventSynchronize(e1));
            float ms = 0;
            MLN_BCK(b, cudaEventElapsedTime(&ms, e0, e1));
            const double per_step = ms / (static_cast<double>(trials) * K);
            if (per_step < best) {
                best = per_step;
                bestK = K;
                bestTile = tile;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->K = bestK;
    b->tile = bestTile;
    b->threads = (bestTile + 2 * bestK + 31) / 32 * 32;
    for (mln_ctx *c : b->ctx) MLN_BCK(b, cudaMemsetAsync(c->flags, 0, sizeof(unsigned int), b->stream));
    return build_tables<R>(b);
}

}  // namespace

extern "C" {

void mln_batch_destroy(mln_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaFree(b->d_grids);
    cudaFree(b->d_items);
    cudaFree(b->d_consts);
    cudaFree(b->d_progress);
    cudaFree(b->d_work);
    for (mln_ctx *c : b->ctx) mln_destroy(c);
    delete b;
}

mln_status mln_batch_create(int32_t count, const mln_params *params, void *const *d_state, void *const *Ez,
                            void *const *Hy, const double *const *src, int64_t src_len, void *stream,
                            mln_batch **out) {
    if (out) *out = nullptr;
    if (count < 1 || !params || !d_state || !Ez || !Hy || !out || src_len < 0) {
        mln::create_error() = "invalid batch arguments";
        return MLN_EINVAL;
    }
    const bool df32 = params[0].kernel == MLN_KERNEL_DF32;
    for (int32_t i = 0; i < count; ++i) {
        const mln_params &p = params[i];
        if (p.precision != params[0].precision || p.form != MLN_FORM_MERGED || p.N > mln::kBatchMaxN ||
            p.maxwell != MLN_MAXWELL_FDTD ||
            (df32 ? (p.kernel != MLN_KERNEL_DF32 || p.precision != MLN_FP64)
                  : (p.kernel != MLN_KERNEL_AUTO && p.kernel != MLN_KERNEL_REGISTER && p.kernel != MLN_KERNEL_JIT))) {
            mln::create_error() = "batch grids need one precision, MLN_FORM_MERGED, MLN_MAXWELL_FDTD, N <= 4 and kernel AUTO, "
                                  "REGISTER or JIT, or MLN_KERNEL_DF32 with MLN_FP64 for every grid (grid " +
                                  std::to_string(i) + ")";
            return MLN_EINVAL;
        }
        if (p.source_kind != MLN_SRC_NONE && src_len > 0 && (!src || !src[i])) {
            mln::create_error() = "grid " + std::to_string(i) + " has a source but no samples";
            return MLN_EINVAL;
        }
    }
    mln_batch *b = new (std::nothrow) mln_batch();
    if (!b) return MLN_ENOMEM;
    b->precision = params[0].precision;
    b->df32 = df32;
    b->user = static_cast<cudaStream_t>(stream);
    b->src_len = src_len;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        mln::create_error() = "creating the batch stream failed";
        mln_batch_destroy(b);
        return MLN_ECUDA;
    }
    for (int32_t i = 0; i < count; ++i) {
        mln_params p = params[i];
        p.kernel = MLN_KERNEL_REGISTER;
        mln_ctx *c = nullptr;
        mln_status st = mln_create(&p, d_state[i], Ez[i], Hy[i], stream, &c);
        if (st != MLN_OK) {
            mln::create_error() = "grid " + std::to_string(i) + ": " + mln::create_error();
            mln_batch_destroy(b);
            return st;
        }
        b->ctx.push_back(c);
        b->src.push_back(src && src_len > 0 ? src[i] : nullptr);
    }
    // Cell model per N: the run-time compiled kernel over the union sparsity
    // pattern of that N's grids unless a grid asks for the register model
    // (MLN_KERNEL_REGISTER); MLN_KERNEL_JIT makes its absence an error.
    bool want_jit = true, need_jit = df32;
    for (int32_t i = 0; i < count; ++i) {
        want_jit = want_jit && params[i].kernel != MLN_KERNEL_REGISTER;
        need_jit = need_jit || params[i].kernel == MLN_KERNEL_JIT;
    }
    if (df32)
        for (int32_t i = 0; i < count; ++i)
            if (!mln::df_constants_in_range(b->ctx[i]->s, params[i].dt)) {
                mln::create_error() = "grid " + std::to_string(i) +
                                      ": MLN_KERNEL_DF32: a constant of the step is outside the double-float range";
                mln_batch_destroy(b);
                return MLN_EUNSUPPORTED;
            }
    std::string why;
    if (want_jit && mln::jit_available(&why)) {
        const bool fp32 = b->precision == MLN_FP32;
        for (mln_ctx *c : b->ctx) mln::batch_pattern_add(b->pat[c->p.N], c->s, c->p, fp32);
        for (int N = 2; N <= mln::kBatchMaxN; ++N) {
            if (b->pat[N].N == 0) continue;
            std::string log;
            const std::string src_n = mln::jit_batch_source(b->pat[N], fp32, df32);
            if (mln::jit_compile(src_n, &b->jit[N], log, "mln_jit_batch") != cudaSuccess ||
                mln::jit_compile(src_n, &b->jitp[N], log, "mln_jit_batch_persist") != cudaSuccess) {
                b->jit[N] = b->jitp[N] = nullptr;
                why = log;
            }
        }
    }
    if (need_jit) {
        for (mln_ctx *c : b->ctx)
            if (!b->jit[c->p.N]) {
                mln::create_error() = std::string(df32 ? "double-float" : "run-time compiled") +
                                      " batch kernel unavailable: " + why;
                mln_batch_destroy(b);
                return MLN_EUNSUPPORTED;
            }
    }
    b->K = 16;
    b->tile = mln::kBatchThreads - 2 * b->K;
    b->threads = mln::kBatchThreads;
    mln_status st = b->precision == MLN_FP64 ? build_tables<double>(b) : build_tables<float>(b);
    if (st != MLN_OK) {
        mln::create_error() = b->err;
        mln_batch_destroy(b);
        return st;
    }
    *out = b;
    return MLN_OK;
}

mln_status mln_batch_autotune(mln_batch *b, int32_t trials, int32_t *block_steps, int32_t *tile_cells) {
    if (!b || trials < 1) return MLN_EINVAL;
    MLN_BCK(b, cudaStreamSynchronize(b->user));
    MLN_BCK(b, cudaStreamSynchronize(b->stream));
    drop_graphs(b);
    mln_status st = b->precision == MLN_FP64 ? autotune_batch<double>(b, trials) : autotune_batch<float>(b, trials);
    MLN_BCK(b, cudaStreamSynchronize(b->stream));
    if (block_steps) *block_steps = b->K;
    if (tile_cells) *tile_cells = b->tile;
    return st;
}

mln_status mln_batch_step(mln_batch *b, int64_t n_steps) {
    if (!b || n_steps < 0) return MLN_EINVAL;
    if (n_steps == 0) return MLN_OK;
    if (b->src_len > 0 && b->steps + n_steps > b->src_len) {
        b->err = "source samples exhausted";
        return MLN_EINVAL;
    }
    // The launches depend on the step offset through the source pointers only;
    // a graph captured for one (offset, count) is replayed when both repeat.
    const bool has_src = b->src_len > 0;
    const int64_t key = has_src ? -1 : n_steps;
    cudaGraphExec_t exec = nullptr;
    auto it = b->graphs.find(key);
    if (it != b->graphs.end()) exec = it->second;
    if (!exec || has_src) {
        if (exec) {
            cudaGraphExecDestroy(exec);
            b->graphs.erase(key);
        }
        cudaGraph_t graph = nullptr;
        MLN_BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        mln_status st = b->precision == MLN_FP64 ? queue_steps<double>(b, n_steps) : queue_steps<float>(b, n_steps);
        cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
        if (st != MLN_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        MLN_BCK(b, ce);
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        MLN_BCK(b, ie);
        b->graphs[key] = exec;
    }
    // order the batch's stream after the caller's work, and the caller's after the graph
    MLN_BCK(b, cudaEventRecord(b->ev_in, b->user));
    MLN_BCK(b, cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    MLN_BCK(b, cudaGraphLaunch(exec, b->stream));
    MLN_BCK(b, cudaEventRecord(b->ev_out, b->stream));
    MLN_BCK(b, cudaStreamWaitEvent(b->user, b->ev_out, 0));
    const int64_t per = (n_steps + b->K - 1) / b->K;
    b->launches += (b->mode == MLN_BATCH_PERSISTENT ? 1 : per) * batch_kernels(b);
    b->steps += n_steps;
    for (mln_ctx *c : b->ctx) {
        c->steps += n_steps;
        c->launches += per;
    }
    return MLN_OK;
}

mln_status mln_batch_set_launch(mln_batch *b, int32_t mode, int32_t wait_limit) {
    if (!b || (mode != MLN_BATCH_CHUNKS && mode != MLN_BATCH_PERSISTENT) || wait_limit < 0) return MLN_EINVAL;
    if (mode == MLN_BATCH_PERSISTENT) {
        for (mln_ctx *c : b->ctx)
            if (!b->jitp[c->p.N]) {
                b->err = "the persistent launch needs the run-time compiled batch kernels";
                return MLN_EUNSUPPORTED;
            }
        if (b->tile < b->K + 2) {
            b->err = "the persistent launch needs tiles longer than K + 1 cells";
            return MLN_EUNSUPPORTED;
        }
    }
    MLN_BCK(b, cudaStreamSynchronize(b->stream));
    drop_graphs(b);
    b->mode = mode;
    b->wait_limit = wait_limit;
    return MLN_OK;
}

int32_t mln_batch_launch(const mln_batch *b) { return b ? b->mode : -1; }

mln_status mln_batch_sync(mln_batch *b) {
    if (!b) return MLN_EINVAL;
    MLN_BCK(b, cudaStreamSynchronize(b->stream));
    MLN_BCK(b, cudaStreamSynchronize(b->user));
    // every grid's flag word is read and cleared; the first grid's problem is reported
    mln_status first = MLN_OK;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        mln_status st = mln_sync(b->ctx[i]);
        if (st != MLN_OK && first == MLN_OK) {
            b->err = "grid " + std::to_string(i) + ": " + mln_last_error(b->ctx[i]);
            first = st;
        }
    }
    return first;
}

mln_ctx *mln_batch_context(mln_batch *b, int32_t i) {
    if (!b || i < 0 || i >= static_cast<int32_t>(b->ctx.size())) return nullptr;
    return b->ctx[i];
}

mln_status mln_batch_shape(const mln_batch *b, int32_t *block_steps, int32_t *tile_cells, int64_t *items,
                           int64_t *launches) {
    if (!b) return MLN_EINVAL;
    if (block_steps) *block_steps = b->K;
    if (tile_cells) *tile_cells = b->tile;
    if (items) *items = b->n_items;
    if (launches) *launches = b->launches;
    return MLN_OK;
}

const char *mln_batch_error(const mln_batch *b) { return b ? b->err.c_str() : ""; }

int32_t mln_batch_kernel_in_use(const mln_batch *b, int32_t N) {
    if (!b || N < 2 || N > mln::kBatchMaxN || b->item_cnt[N] == 0) return -1;
    if (b->jit[N] && b->df32) return MLN_KERNEL_DF32;
    return b->jit[N] ? MLN_KERNEL_JIT : MLN_KERNEL_REGISTER;
}

mln_status mln_batch_kernel_source(int32_t count, const mln_params *params, int32_t N, char *buf, size_t cap,
                                   size_t *len) {
    if (count < 1 || !params || N < 2 || N > mln::kBatchMaxN) {
        mln::create_error() = "invalid arguments";
        return MLN_EINVAL;
    }
    mln::BatchPattern pat;
    bool fp32 = params[0].precision == MLN_FP32;
    for (int32_t i = 0; i < count; ++i) {
        if (params[i].N != N) continue;
        std::string err;
        mln::Setup s;
        mln_status st = mln::validate(params[i], err);
        if (st == MLN_OK) st = mln::build_setup(params[i], s, err);
        if (st != MLN_OK) {
            mln::create_error() = "grid " + std::to_string(i) + ": " + err;
            return st;
        }
        mln::batch_pattern_add(pat, s, params[i], fp32);
    }
    if (pat.N == 0) {
        mln::create_error() = "no grid with this N";
        return MLN_EINVAL;
    }
    const std::string src = mln::jit_batch_source(pat, fp32, params[0].kernel == MLN_KERNEL_DF32);
    if (len) *len = src.size();
    if (buf && cap > 0) {
        const size_t k = std::min(cap - 1, src.size());
        std::memcpy(buf, src.data(), k);
        buf[k] = '\0';
    }
    return MLN_OK;
}

}  // extern "C"
