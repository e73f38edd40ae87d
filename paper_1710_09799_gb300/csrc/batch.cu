// Batched solver: many independent grids (any mix of N = 2..4, lengths and
// boundaries, one precision) advanced together, each launch covering every
// tile of every grid. The sequence of launches of one mln_batch_step call is
// captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "dispatch.cuh"
#include "mln.h"
#include "setup.h"

namespace mln {

// Shared-memory room for one grid's constants (the merged-form constants of
// N = 4 in FP64 are 3.9 KB).
constexpr int kBatchConstsMax = 4096;
constexpr int kBatchMaxN = 4;

template <typename R>
struct BatchGrid {
    R *E[2], *H[2], *S[2];   // buffer set 0 (caller's) and 1 (context's)
    const double *src;       // source samples from the batch's step 0, or nullptr
    unsigned int *flags;
    int64_t n_cells, mb, me, stride, source_cell;
    int32_t N, boundary, source_kind, consts_off, consts_bytes, pad_;
    R ch, ca, cb, inv_dx, kappa;
};

struct BatchItem {
    int32_t grid, tile;
};

template <int N, typename R>
__device__ __forceinline__ void batch_tile(const BlockArgs<R> &a, const unsigned char *consts, int64_t tile,
                                           unsigned char *rest) {
    using K = MergedConsts<N, R>;
    block_body<N, R, RegisterCell<N, R, K>>(a, *reinterpret_cast<const K *>(consts), tile, rest);
}

// One block per work item (grid, tile). The grid's constants are staged in
// shared memory (every thread of a warp reads the same entry: broadcasts).
template <typename R>
__global__ void __launch_bounds__(kMaxThreads, 1)
    mln_batch_kernel(const BatchGrid<R> *__restrict__ grids, const BatchItem *__restrict__ items,
                     const unsigned char *__restrict__ consts, int parity, int nsteps, int halo, int tile,
                     int64_t step_offset) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchItem it = items[blockIdx.x];
    const BatchGrid<R> &g = grids[it.grid];
    for (int o = threadIdx.x * 16; o < g.consts_bytes; o += blockDim.x * 16)
        *reinterpret_cast<uint4 *>(smem_raw + o) = *reinterpret_cast<const uint4 *>(consts + g.consts_off + o);
    __syncthreads();
    BlockArgs<R> a;
    a.E_in = g.E[parity];
    a.H_in = g.H[parity];
    a.s_in = g.S[parity];
    a.E_out = g.E[parity ^ 1];
    a.H_out = g.H[parity ^ 1];
    a.s_out = g.S[parity ^ 1];
    a.src = g.src ? g.src + step_offset : nullptr;
    a.flags = g.flags;
    a.n_cells = g.n_cells;
    a.mb = g.mb;
    a.me = g.me;
    a.stride = g.stride;
    a.source_cell = g.source_cell;
    a.nsteps = nsteps;
    a.halo = halo;
    a.tile = tile;
    a.boundary = g.boundary;
    a.source_kind = g.source_kind;
    a.pad_ = 0;
    a.ch = g.ch;
    a.ca = g.ca;
    a.cb = g.cb;
    a.inv_dx = g.inv_dx;
    a.kappa = g.kappa;
    unsigned char *rest = smem_raw + kBatchConstsMax;
    switch (g.N) {
    case 2: batch_tile<2, R>(a, smem_raw, it.tile, rest); break;
    case 3: batch_tile<3, R>(a, smem_raw, it.tile, rest); break;
    case 4: batch_tile<4, R>(a, smem_raw, it.tile, rest); break;
    default: break;
    }
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

// Grid table and work list for the current tile size (tiles sorted by
// decreasing cost, D^2 per cell, so the largest start first).
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
        g.consts_off = static_cast<int32_t>(blob.size());
        g.consts_bytes = static_cast<int32_t>((c->consts.size() + 15) / 16 * 16);
        g.ch = a.ch;
        g.ca = a.ca;
        g.cb = a.cb;
        g.inv_dx = a.inv_dx;
        g.kappa = a.kappa;
        blob.insert(blob.end(), c->consts.begin(), c->consts.end());
        blob.resize((blob.size() + 15) / 16 * 16, 0);
        grids.push_back(g);
        const int64_t nt = (c->p.n_cells + b->tile - 1) / b->tile;
        const int cost = c->D * c->D;
        for (int64_t t = 0; t < nt; ++t) items.push_back({cost, mln::BatchItem{static_cast<int32_t>(i), static_cast<int32_t>(t)}});
    }
    std::stable_sort(items.begin(), items.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    std::vector<mln::BatchItem> list;
    for (auto &x : items) list.push_back(x.second);
    cudaFree(b->d_grids);
    cudaFree(b->d_items);
    cudaFree(b->d_consts);
    b->d_grids = b->d_items = b->d_consts = nullptr;
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
    return mln::kBatchConstsMax + 2 * static_cast<size_t>(threads) * sizeof(R);
}

template <typename R>
cudaError_t launch_batch(mln_batch *b, int parity, int nsteps, int64_t step_offset) {
    // at most 4 KB + 2 x 512 x 8 B = 12 KB: below the 48 KB default, no attribute needed
    const size_t smem = batch_smem<R>(b->threads);
    auto kern = mln::mln_batch_kernel<R>;
    kern<<<static_cast<unsigned>(b->n_items), b->threads, smem, b->stream>>>(
        static_cast<const mln::BatchGrid<R> *>(b->d_grids), static_cast<const mln::BatchItem *>(b->d_items),
        static_cast<const unsigned char *>(b->d_consts), parity, nsteps, b->K, b->tile, step_offset);
    return cudaGetLastError();
}

// Queue the launches of n_steps steps from the batch's current step count;
// the result ends in buffer set 0 of every grid.
template <typename R>
mln_status queue_steps(mln_batch *b, int64_t n_steps) {
    int parity = 0;
    for (int64_t done = 0; done < n_steps;) {
        int ns = static_cast<int>(std::min<int64_t>(b->K, n_steps - done));
        MLN_BCK(b, launch_batch<R>(b, parity, ns, b->steps + done));
        parity ^= 1;
        done += ns;
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
            if (tile + 2 * K > mln::kMaxThreads) continue;
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
    for (int32_t i = 0; i < count; ++i) {
        const mln_params &p = params[i];
        if (p.precision != params[0].precision || p.form != MLN_FORM_MERGED || p.N > mln::kBatchMaxN ||
            p.kernel == MLN_KERNEL_SPARSE) {
            mln::create_error() = "batch grids need one precision, MLN_FORM_MERGED, N <= 4 and the register kernel "
                                  "(grid " + std::to_string(i) + ")";
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
    b->K = 16;
    b->tile = 256;
    b->threads = (b->tile + 2 * b->K + 31) / 32 * 32;
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
    b->launches += per;
    b->steps += n_steps;
    for (mln_ctx *c : b->ctx) {
        c->steps += n_steps;
        c->launches += per;
    }
    return MLN_OK;
}

mln_status mln_batch_sync(mln_batch *b) {
    if (!b) return MLN_EINVAL;
    MLN_BCK(b, cudaStreamSynchronize(b->stream));
    MLN_BCK(b, cudaStreamSynchronize(b->user));
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        mln_status st = mln_sync(b->ctx[i]);
        if (st != MLN_OK) {
            b->err = "grid " + std::to_string(i) + ": " + mln_last_error(b->ctx[i]);
            return st;
        }
    }
    return MLN_OK;
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

}  // extern "C"
