// mln_adjoint: gradients of a probe-field objective by the discrete adjoint
// (reverse-time) method with checkpointing and recomputation.
//
// The reverse sweep reads, for every step, a recorded "set": the step's
// state, fields and the intermediates of its medium step, written by the
// tracing kernel (the literal Strang step). Where the sets of all segments
// of `every` steps fit the memory limit, a Strang-form context on the
// register model records them in its forward pass and any other context
// recomputes all segments side by side from its checkpoints (mapped to the
// adjoint vector d, which all forms share up to rounding: the merged and
// rotated forms hold an affine image of d); the backward pass is then
// replayed from one CUDA graph. Otherwise segment s - 1 is recomputed while
// the reverse sweep of segment s runs. The reverse sweep runs from each
// segment's last step to its first, carrying the adjoint of (E, H, d) and
// accumulating the gradients of the step's constants; the host maps those
// to the dipole operator and the relaxation superoperator (exact Frechet
// derivatives, see adjoint_chain).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "adjoint.cuh"
#include "ctx.h"
#include "dispatch.cuh"
#include "mln.h"
#include "setup.h"

namespace {

#define MLN_ACK(c, call)                                                        \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            (c)->err = std::string(#call) + ": " + cudaGetErrorString(e_);      \
            st = MLN_ECUDA;                                                     \
            goto done;                                                          \
        }                                                                       \
    } while (0)

template <int N, typename R>
mln::AdjConsts<N, R> adj_consts(const mln::Setup &s, double dt) {
    constexpr int D = mln::Dims<N>::D, Q = mln::Dims<N>::Q;
    mln::AdjConsts<N, R> k;
    std::memset(&k, 0, sizeof(k));
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            k.Dl[i * D + j] = static_cast<R>(s.A0[i * D + j] - (i == j ? 1.0 : 0.0));
            k.T[i * D + j] = static_cast<R>(s.T[i * D + j]);
        }
    for (int i = 0; i < D; ++i) {
        k.b[i] = static_cast<R>(s.b[i]);
        k.w[i] = static_cast<R>(s.w[i]);
    }
    for (int a = 0; a < N - 1; ++a) k.psi_dt[a] = static_cast<R>(s.psi[a] * dt);
    for (int p = 0; p < Q; ++p) k.theta_dt[p] = static_cast<R>(s.theta[p] * dt);
    return k;
}

// d = sd0 + Sd s for every medium cell, SoA in and out (tab = [Sd | sd0] in FP64).
template <typename R>
__global__ void state_to_d(const R *__restrict__ s, R *__restrict__ d, int64_t stride, int64_t count, int D,
                           const double *__restrict__ tab) {
    const int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (c >= count) return;
    for (int k = 0; k < D; ++k) {
        double acc = tab[D * D + k];
        for (int j = 0; j < D; ++j) acc += tab[k * D + j] * static_cast<double>(s[j * stride + c]);
        d[k * stride + c] = static_cast<R>(acc);
    }
}

// Buffers of one (state, E, H) set inside a larger allocation.
template <typename R>
struct Set {
    R *E, *H, *S;
    R *I;  // traced intermediates of the step that starts from this set
};

template <int N, typename R>
mln_status adjoint_t(mln_ctx *c, int64_t n_steps, const double *src, int64_t probe, int every, mln_adjoint_out *out) {
    using L = mln::AccLayout<N>;
    // a segment never spans more than the run (the slots are sized by it)
    if (every > n_steps) every = static_cast<int>(n_steps);
    mln_status st = MLN_OK;
    const int64_t n = c->p.n_cells;
    const size_t sb = c->state_bytes, fb = c->field_bytes;
    // a set: state, E, H, then the intermediates of the step from it
    // (2 D + 2 q rows of `stride`, 2 q more in FP64: see StrangTraceCell)
    const size_t ib = static_cast<size_t>(2 * mln::Dims<N>::D + (sizeof(R) == 8 ? 4 : 2) * mln::Dims<N>::Q) *
                      c->stride * sizeof(R);
    const size_t off_I = (sb + 2 * fb + 255) / 256 * 256;
    const size_t set_bytes = (off_I + ib + 255) / 256 * 256;
    const int64_t nseg = (n_steps + every - 1) / every;
    unsigned char *ckpt = nullptr, *slots = nullptr, *adj = nullptr;
    double *dsrc = nullptr, *acc = nullptr, *accsum = nullptr;
    std::vector<double> hacc(L::size, 0.0);
    const mln::AdjConsts<N, R> k = adj_consts<N, R>(c->s, c->p.dt);
    auto set_at = [&](unsigned char *base, int64_t i) {
        unsigned char *p = base + i * set_bytes;
        return Set<R>{reinterpret_cast<R *>(p + sb), reinterpret_cast<R *>(p + sb + fb), reinterpret_cast<R *>(p),
                      reinterpret_cast<R *>(p + off_I)};
    };
    auto copy_set = [&](Set<R> dst, Set<R> from, cudaStream_t strm) {
        cudaError_t e = cudaMemcpyAsync(dst.S, from.S, sb, cudaMemcpyDeviceToDevice, strm);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst.E, from.E, fb, cudaMemcpyDeviceToDevice, strm);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst.H, from.H, fb, cudaMemcpyDeviceToDevice, strm);
        return e;
    };
    const Set<R> user{static_cast<R *>(c->E[0]), static_cast<R *>(c->H[0]), static_cast<R *>(c->st[0]), nullptr};
    mln::BlockArgs<R> fa = mln::base_args<R>(c);
    // Reverse sweep: K steps per launch over tiles with K-cell halos (one more
    // on the right of an open grid), cells of AdjLanes lanes; tiles of about
    // n / SMs cells, so that a small grid fills every SM with one block (one
    // wave), up to the block's thread limit. FP64 is bound by its arithmetic
    // and takes K = 4 (the halo costs flops); FP32 is bound by each launch's
    // fixed latency and takes K = 12 (a third of the launches) in blocks of up
    // to 640 threads. Measured on the 8192-cell gradient workload (FP32
    // gradient at K = 4, 8, 10, 12: 1.44e9, 1.70e9, 1.76e9, 1.78e9 cell-updates/s).
    constexpr int LN = mln::AdjLanes<N>::value;
    const int open1 = c->p.boundary == MLN_BC_PERIODIC ? 0 : 1;
    const int bK = sizeof(R) == 4 ? 12 : 4;
    const int max_cells = mln::AdjThreads<R>::kMax / LN;
    const int cell_step = LN < 32 ? 32 / LN : 1;  // whole warps
    const int btile = static_cast<int>(std::max<int64_t>(
        1, std::min<int64_t>((n + std::max(c->sms, 1) - 1) / std::max(c->sms, 1), max_cells - 2 * bK - open1)));
    const int bcells = (btile + 2 * bK + open1 + cell_step - 1) / cell_step * cell_step;
    const unsigned bthreads = static_cast<unsigned>(bcells * LN);
    const unsigned bgrid = static_cast<unsigned>((n + btile - 1) / btile);
    const size_t bsmem = mln::adj_block_smem<N, R>(bcells);
    // the recompute runs the literal Strang form whatever the context's form
    std::vector<unsigned char> strang;
    const bool convert = c->p.form != MLN_FORM_STRANG;  // checkpoints hold another form's state
    if (!mln::pack_consts(c->s, MLN_FORM_STRANG, c->p.dt, static_cast<R>(0), strang)) return MLN_EUNSUPPORTED;
    // Recompute: the context's fused steps per launch (autotuned if the
    // caller did), at most 256 threads a block (the tracing kernel's bound);
    // every step recorded into its slot. One segment at a time runs the
    // context's tile (its latency-bound shape); segments side by side run the
    // longest tile (least halo: the launch has work for every SM).
    const int rK = std::min(c->K, 64);
    const int tile_one = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->tile, 256 - 2 * rK)));
    const int tile_many = std::max(tile_one, 256 - 2 * rK);
    mln::AdjBlockArgs<R> aa{};
    Set<R> A0s, A1s;
    // Two ways to schedule the recomputation (segments are independent given
    // their checkpoints; a ring of a few thousand cells leaves most of the GPU
    // idle in one segment's launches):
    // - all at once, when every segment's slot fits the memory limit (by
    //   default half the free device memory): the forward pass records them
    //   (Strang contexts on the register model), or after it each launch
    //   advances the same steps of all full segments side by side (grid y =
    //   segment); then the reverse sweeps run segment after segment;
    // - otherwise two slot buffers: segment s - 1 is recomputed on a second
    //   stream while the reverse sweep of segment s runs; events order the
    //   recompute after the sweep that last used its buffer, and each sweep
    //   after its recompute.
    cudaStream_t rs = nullptr;
    // All at once: the backward pass (the side-by-side recomputation, the
    // reverse sweep, the reduction) is captured on the second stream and
    // replayed as one graph: one host call instead of ~1000 launches, and
    // shorter gaps between them. The forward pass stays on the context's
    // stream with programmatic launches (measured faster than inside the
    // graph: FP32 gradient 1.47e9 against 1.32e9 cell-updates/s).
    cudaStream_t ws = nullptr;  // the stream that work is issued to
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool capturing = false;
    cudaEvent_t ev_fwd = nullptr, ev_rec[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
    unsigned char *slot_buf[2] = {nullptr, nullptr};
    const size_t slot_bytes = static_cast<size_t>(every + 1) * set_bytes;
    const int64_t nfull = n_steps / every;  // segments of `every` steps
    int64_t launches = 0;
    bool all_at_once = false;
    {
        size_t free_b = 0, total_b = 0;
        if (nfull <= 65535 && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            // the workspace this context already holds counts as free
            const double avail = static_cast<double>(free_b) + static_cast<double>(c->adj_buf_bytes);
            const double limit = c->adj_mem > 0 ? static_cast<double>(c->adj_mem) : 0.5 * avail;
            all_at_once = static_cast<double>(nseg) * static_cast<double>(slot_bytes) <= limit;
        }
    }
    // the workspace's parts: offsets of the slots, the adjoint sets, the
    // accumulators, their sums and dJ/dsrc from its base (the checkpoints)
    auto up256 = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t ws_off[5];
    ws_off[0] = up256(static_cast<size_t>(nseg) * set_bytes);
    ws_off[1] = ws_off[0] + up256(static_cast<size_t>(all_at_once ? nseg : 2) * slot_bytes);
    ws_off[2] = ws_off[1] + up256(2 * set_bytes);
    ws_off[3] = ws_off[2] + up256(static_cast<size_t>(L::size) * n * sizeof(double));
    ws_off[4] = ws_off[3] + up256(static_cast<size_t>(L::size) * sizeof(double));
    const size_t ws_need = ws_off[4] + (src ? up256(static_cast<size_t>(n_steps) * sizeof(double)) : 0);
    auto slot_of = [&](int64_t sg) { return all_at_once ? slots + sg * slot_bytes : slot_buf[sg & 1]; };
    // A Strang-form context whose step is the register model (the tracing
    // kernel's arithmetic) and whose segments all fit: its forward pass can
    // record the segments itself, so nothing is recomputed.
    const bool traced_forward = all_at_once && c->p.form == MLN_FORM_STRANG && !c->jit_fn && !c->sparse && !c->tc &&
                                !c->pstd;
    // the segment's checkpoint into set 0 of its slot (as d), on stream strm
    auto prepare = [&](int64_t sg, unsigned char *sl, cudaStream_t strm) -> cudaError_t {
        cudaError_t e = copy_set(set_at(sl, 0), set_at(ckpt, sg), strm);
        if (e == cudaSuccess && convert && c->n_med > 0) {
            state_to_d<R><<<static_cast<unsigned>((c->n_med + 127) / 128), 128, 0, strm>>>(
                set_at(ckpt, sg).S, set_at(sl, 0).S, c->stride, c->n_med, c->D, c->tab_d);
            e = cudaGetLastError();
        }
        return e;
    };
    // steps of `segs` segments side by side from the slot sl of the first
    // (the others seg_bytes apart), every step recorded, on stream strm
    auto run_segments = [&](int64_t sg, int64_t segs, int64_t glen, unsigned char *sl, cudaStream_t strm,
                            bool programmatic = false) -> cudaError_t {
        const int64_t g0 = sg * every;
        const int rtile = segs > 1 ? tile_many : tile_one;
        const int rthreads = (rtile + 2 * rK + 31) / 32 * 32;
        cudaError_t e = cudaSuccess;
        fa.seg_bytes = static_cast<int64_t>(slot_bytes);
        fa.seg_src = every;
        for (int64_t j = 0; e == cudaSuccess && j < glen; j += rK) {
            const int ns = static_cast<int>(std::min<int64_t>(rK, glen - j));
            const Set<R> in = set_at(sl, j), o = set_at(sl, j + ns), r1 = set_at(sl, j + 1);
            fa.E_in = in.E;
            fa.H_in = in.H;
            fa.s_in = in.S;
            fa.E_out = o.E;
            fa.H_out = o.H;
            fa.s_out = o.S;
            fa.rec_E = r1.E;
            fa.rec_H = r1.H;
            fa.rec_S = r1.S;
            fa.rec_I = in.I;
            fa.rec_set = static_cast<int64_t>(set_bytes);
            fa.nsteps = ns;
            fa.src = (src && c->p.source_kind != MLN_SRC_NONE) ? src + g0 + j : nullptr;
            // plain launches: the recompute runs beside the reverse sweep, and
            // blocks placed early by programmatic launches took SM resources
            // from it (FP64 gradient 1.77e8 -> 1.56e8 cell-updates/s)
            fa.halo = rK;
            fa.tile = rtile;
            e = mln::launch_block_trace(c->p.N, fa, strang,
                                        dim3(static_cast<unsigned>((n + rtile - 1) / rtile),
                                             static_cast<unsigned>(segs)),
                                        dim3(rthreads), mln::field_smem<R>(rthreads), strm, programmatic);
            ++launches;
        }
        return e;
    };
    // segment sg from its checkpoint into slot sl, on stream strm
    auto recompute = [&](int64_t sg, unsigned char *sl, cudaStream_t strm) -> cudaError_t {
        cudaError_t e = prepare(sg, sl, strm);
        if (e == cudaSuccess) e = run_segments(sg, 1, std::min<int64_t>(every, n_steps - sg * every), sl, strm);
        return e;
    };

    // One workspace, kept by the context for its next call (an optimisation
    // loop evaluates the gradient again and again; allocating and freeing
    // 5-13 GB took 4-8 ms a call): checkpoints | slots | adjoint sets |
    // accumulators | their sums | dJ/dsrc, each on a 256-byte boundary.
    if (c->adj_buf_bytes < ws_need) {
        cudaFree(c->adj_buf);  // synchronises with the device first
        c->adj_buf = nullptr;
        c->adj_buf_bytes = 0;
        MLN_ACK(c, cudaMalloc(&c->adj_buf, ws_need));
        c->adj_buf_bytes = ws_need;
    }
    ckpt = c->adj_buf;
    slots = ckpt + ws_off[0];
    adj = ckpt + ws_off[1];
    acc = reinterpret_cast<double *>(ckpt + ws_off[2]);
    accsum = reinterpret_cast<double *>(ckpt + ws_off[3]);
    dsrc = src ? reinterpret_cast<double *>(ckpt + ws_off[4]) : nullptr;
    slot_buf[0] = slots;
    slot_buf[1] = slots + slot_bytes;
    MLN_ACK(c, cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking));
    MLN_ACK(c, cudaEventCreateWithFlags(&ev_fwd, cudaEventDisableTiming));
    for (int b = 0; b < 2; ++b) {
        MLN_ACK(c, cudaEventCreateWithFlags(&ev_rec[b], cudaEventDisableTiming));
        MLN_ACK(c, cudaEventCreateWithFlags(&ev_rev[b], cudaEventDisableTiming));
    }

    if (!traced_forward) {
        // forward with checkpoints, the context's own step on its stream
        for (int64_t s = 0; s < nseg; ++s) {
            const int64_t len = std::min<int64_t>(every, n_steps - s * every);
            MLN_ACK(c, copy_set(set_at(ckpt, s), user, c->stream));
            mln_status r = mln_step(c, len, src ? src + s * every : nullptr);
            if (r != MLN_OK) {
                st = r;
                goto done;
            }
        }
    }
    ws = c->stream;
    if (traced_forward) {
        // The forward pass is the recomputation: each segment from the end of
        // the one before, every step traced (the same arithmetic as the
        // context's own Strang step), then the context takes the last state.
        for (int64_t s = 0; s < nseg; ++s) {
            const int64_t len = std::min<int64_t>(every, n_steps - s * every);
            MLN_ACK(c, copy_set(set_at(slot_of(s), 0), s == 0 ? user : set_at(slot_of(s - 1), every), ws));
            MLN_ACK(c, run_segments(s, 1, len, slot_of(s), ws, true));
        }
        MLN_ACK(c, copy_set(user, set_at(slot_of(nseg - 1), n_steps - (nseg - 1) * every), ws));
        c->steps += n_steps;
        c->launches += launches;
    }
    if (all_at_once) {
        MLN_ACK(c, cudaEventRecord(ev_fwd, c->stream));
        MLN_ACK(c, cudaStreamWaitEvent(rs, ev_fwd, 0));
        MLN_ACK(c, cudaStreamBeginCapture(rs, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        ws = rs;
    }
    // backward
    MLN_ACK(c, cudaMemsetAsync(adj, 0, 2 * set_bytes, ws));
    MLN_ACK(c, cudaMemsetAsync(acc, 0, L::size * n * sizeof(double), ws));
    A0s = set_at(adj, 0);
    A1s = set_at(adj, 1);
    aa.acc = acc;
    aa.n_cells = n;
    aa.mb = c->p.medium_begin;
    aa.me = c->p.medium_end;
    aa.stride = c->stride;
    aa.source_cell = c->p.source_cell;
    aa.probe_cell = probe;
    aa.source_kind = c->p.source_kind;
    aa.boundary = c->p.boundary;
    aa.kappa = fa.kappa;
    aa.dt = c->p.dt;
    aa.ch = fa.ch;
    aa.ca = fa.ca;
    aa.cb = fa.cb;
    aa.inv_dx = fa.inv_dx;
    if (traced_forward) {
        // every segment recorded by the forward pass
    } else if (all_at_once) {
        for (int64_t s = 0; s < nseg; ++s) MLN_ACK(c, prepare(s, slot_of(s), ws));
        if (nfull > 0) MLN_ACK(c, run_segments(0, nfull, every, slot_of(0), ws));
        if (nfull < nseg) MLN_ACK(c, run_segments(nfull, 1, n_steps - nfull * every, slot_of(nfull), ws));
    } else {
        MLN_ACK(c, cudaEventRecord(ev_fwd, c->stream));
        MLN_ACK(c, cudaStreamWaitEvent(rs, ev_fwd, 0));
        MLN_ACK(c, recompute(nseg - 1, slot_buf[(nseg - 1) & 1], rs));
        MLN_ACK(c, cudaEventRecord(ev_rec[(nseg - 1) & 1], rs));
    }
    for (int64_t s = nseg - 1; s >= 0; --s) {
        const int64_t s0 = s * every, len = std::min<int64_t>(every, n_steps - s0);
        unsigned char *sl = slot_of(s);
        if (!all_at_once) MLN_ACK(c, cudaStreamWaitEvent(c->stream, ev_rec[s & 1], 0));
        if (s >= 1 && !all_at_once) {
            // the buffer of segment s - 1 was last read by the sweep of segment s + 1
            MLN_ACK(c, cudaStreamWaitEvent(rs, ev_rev[(s - 1) & 1], 0));
            MLN_ACK(c, recompute(s - 1, slot_buf[(s - 1) & 1], rs));
            MLN_ACK(c, cudaEventRecord(ev_rec[(s - 1) & 1], rs));
        }
        for (int64_t j_hi = len - 1; j_hi >= 0; j_hi -= bK) {
            aa.rec = sl;
            aa.rec_set = static_cast<int64_t>(set_bytes);
            aa.off_E = static_cast<int64_t>(sb);
            aa.off_I = static_cast<int64_t>(off_I);
            aa.j_hi = static_cast<int32_t>(j_hi);
            aa.nsteps = static_cast<int32_t>(std::min<int64_t>(bK, j_hi + 1));
            aa.halo = bK;
            aa.tile = btile;
            aa.Ea = A0s.E;
            aa.Ha = A0s.H;
            aa.Sa = A0s.S;
            aa.Eb = A1s.E;
            aa.Hb = A1s.H;
            aa.Sb = A1s.S;
            aa.dsrc = (src && c->p.source_kind != MLN_SRC_NONE) ? dsrc + s0 : nullptr;
            mln::mln_adjoint_block<N, R><<<bgrid, bthreads, bsmem, ws>>>(aa, k);
            MLN_ACK(c, cudaGetLastError());
            std::swap(A0s, A1s);
        }
        if (!all_at_once) MLN_ACK(c, cudaEventRecord(ev_rev[s & 1], c->stream));
    }
    if (sizeof(R) == 8) mln::mln_adjoint_reduce<<<L::size, 256, 0, ws>>>(acc, n, accsum);
    else mln::mln_adjoint_reduce_pairs<<<L::size, 256, 0, ws>>>(reinterpret_cast<const float2 *>(acc), n, accsum);
    MLN_ACK(c, cudaGetLastError());
    if (capturing) {
        capturing = false;
        MLN_ACK(c, cudaStreamEndCapture(rs, &graph));
        MLN_ACK(c, cudaGraphInstantiate(&graph_exec, graph, 0));
        MLN_ACK(c, cudaGraphLaunch(graph_exec, rs));
        MLN_ACK(c, cudaEventRecord(ev_rev[0], rs));
        MLN_ACK(c, cudaStreamWaitEvent(c->stream, ev_rev[0], 0));
    }
    MLN_ACK(c, cudaMemcpyAsync(hacc.data(), accsum, L::size * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (out->dJ_dsrc) {
        if (src && c->p.source_kind != MLN_SRC_NONE)
            MLN_ACK(c, cudaMemcpyAsync(out->dJ_dsrc, dsrc, n_steps * sizeof(double), cudaMemcpyDeviceToHost,
                                       c->stream));
        else
            std::fill(out->dJ_dsrc, out->dJ_dsrc + n_steps, 0.0);
    }
    MLN_ACK(c, cudaStreamSynchronize(c->stream));
    out->J = hacc[L::J];
    {
        std::string err;
        st = mln::adjoint_chain(c->p, c->s, hacc.data(), out->dJ_dmu, out->dJ_dG, err);
        if (st != MLN_OK) c->err = err;
    }
done:
    if (capturing) {  // a failure while capturing: end the capture, drop its graph
        cudaGraph_t partial = nullptr;
        cudaStreamEndCapture(rs, &partial);
        if (partial) cudaGraphDestroy(partial);
    }
    cudaStreamSynchronize(c->stream);
    if (rs) {
        cudaStreamSynchronize(rs);
        cudaStreamDestroy(rs);
    }
    if (ev_fwd) cudaEventDestroy(ev_fwd);
    for (int b = 0; b < 2; ++b) {
        if (ev_rec[b]) cudaEventDestroy(ev_rec[b]);
        if (ev_rev[b]) cudaEventDestroy(ev_rev[b]);
    }
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph) cudaGraphDestroy(graph);
    return st;
}

}  // namespace

extern "C" {

mln_status mln_set_adjoint_memory(mln_ctx *c, int64_t bytes) {
    if (!c || bytes < 0) return MLN_EINVAL;
    c->adj_mem = bytes;
    return MLN_OK;
}

mln_status mln_adjoint_release(mln_ctx *c) {
    if (!c) return MLN_EINVAL;
    if (c->adj_buf) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) e = cudaFree(c->adj_buf);
        c->adj_buf = nullptr;
        c->adj_buf_bytes = 0;
        if (e != cudaSuccess) {
            c->err = std::string("adjoint workspace release: ") + cudaGetErrorString(e);
            return MLN_ECUDA;
        }
    }
    return MLN_OK;
}

mln_status mln_adjoint(mln_ctx *c, int64_t n_steps, const double *src, int64_t probe_cell, int32_t every,
                       mln_adjoint_out *out) {
    if (!c || !out || n_steps < 1 || every < 1 || probe_cell < 0 || probe_cell >= c->p.n_cells) {
        if (c) c->err = "invalid adjoint arguments";
        return MLN_EINVAL;
    }
    if (c->p.N > 4 || c->p.maxwell != MLN_MAXWELL_FDTD || c->pstd) {
        c->err = "mln_adjoint needs MLN_MAXWELL_FDTD and N <= 4";
        return MLN_EUNSUPPORTED;
    }
    switch (c->p.N) {
    case 2: return c->p.precision == MLN_FP64 ? adjoint_t<2, double>(c, n_steps, src, probe_cell, every, out)
                                              : adjoint_t<2, float>(c, n_steps, src, probe_cell, every, out);
    case 3: return c->p.precision == MLN_FP64 ? adjoint_t<3, double>(c, n_steps, src, probe_cell, every, out)
                                              : adjoint_t<3, float>(c, n_steps, src, probe_cell, every, out);
    case 4: return c->p.precision == MLN_FP64 ? adjoint_t<4, double>(c, n_steps, src, probe_cell, every, out)
                                              : adjoint_t<4, float>(c, n_steps, src, probe_cell, every, out);
    default: return MLN_EUNSUPPORTED;
    }
}

}  // extern "C"
