// The solver context (internal; shared by the single-grid and batched entry points).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "mln.h"
#include "setup.h"

struct mln_ctx {
    mln_params p{};
    mln::Setup s;
    int D = 0;
    int64_t n_med = 0, stride = 0;
    size_t rsz = 8;                 // bytes per device real
    size_t state_bytes = 0, field_bytes = 0;
    void *st[2] = {nullptr, nullptr};  // [0] caller's buffer, [1] context-owned alternate
    void *E[2] = {nullptr, nullptr};
    void *H[2] = {nullptr, nullptr};
    cudaStream_t stream = nullptr;
    unsigned int *flags = nullptr;
    std::vector<unsigned char> consts;
    int K = 16, tile = 0, threads = 0, max_threads = mln::kMaxThreads;
    int64_t steps = 0, launches = 0;
    bool sparse = false;               // shared-memory sparse cell model (FP64 merged)
    void *jit_fn = nullptr;            // run-time compiled step kernel (CUfunction), or nullptr
    bool df32 = false;                 // ... whose cell update is double-float (MLN_KERNEL_DF32)
    void *prog = nullptr;              // its program: rowptr | cols | vals
    int tc = 0;                        // tensor-core cell model: 0 none, MLN_KERNEL_TENSOR(_SMEM)
    bool tcr = false;                  // ... for the rotated basis (MLN_FORM_ROTATED)
    int64_t adj_mem = 0;               // mln_adjoint's limit for the recorded segments (0: half the free memory)
    unsigned char *adj_buf = nullptr;  // mln_adjoint's device workspace, kept between calls
    size_t adj_buf_bytes = 0;
    int sms = 152;                     // SMs of the context's device
    void *tc_img = nullptr;            // its B-operand image (device)
    std::vector<unsigned char> tc_scal;  // and scalar constants
    void *pstd = nullptr;              // PSTD field solver: tables and work arrays (nullptr: FDTD)
    void *pstd_host = nullptr;         // and its stream, events and captured step graphs
    int nnz = 0, nrowptr = 0;
    // output tables (FP64, device): rows x D matrix followed by rows offsets
    double *tab_rho = nullptr, *tab_pop = nullptr, *tab_d = nullptr, *tab_in = nullptr;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    std::string err;
};

namespace mln {

// Launch arguments of a context that do not change between launches.
template <typename R>
inline BlockArgs<R> base_args(const mln_ctx *c) {
    const double eps = kEps0 * c->p.eps_r, mu = kMu0 * c->p.mu_r;
    const double sg = c->p.sigma * c->p.dt / (2.0 * eps);
    const double cv = 1.0 / std::sqrt(eps * mu);
    BlockArgs<R> a{};
    a.flags = c->flags;
    a.n_cells = c->p.n_cells;
    a.mb = c->p.medium_begin;
    a.me = c->p.medium_end;
    a.stride = c->stride;
    a.source_cell = c->p.source_cell;
    a.halo = c->K;
    a.tile = c->tile;
    a.boundary = c->p.boundary;
    a.source_kind = c->p.source_kind;
    a.ch = static_cast<R>(c->p.dt / (mu * c->p.dx));
    a.ca = static_cast<R>((1.0 - sg) / (1.0 + sg));
    a.cb = static_cast<R>((c->p.dt / eps) / (1.0 + sg));
    a.inv_dx = static_cast<R>(1.0 / c->p.dx);
    a.kappa = static_cast<R>((cv * c->p.dt - c->p.dx) / (cv * c->p.dt + c->p.dx));
    return a;
}

}  // namespace mln
