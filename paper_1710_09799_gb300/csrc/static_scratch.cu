// mln_step_noalloc: the fused step without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code that runs where the CUDA
// allocator is off limits (inside a framework that owns all device memory
// through its own pool, a plug-in that must not change the process's memory
// footprint, a real-time loop that forbids allocation after start-up). For
// them this entry point runs the same register-model step kernel as
// mln_step, but its second (ping-pong) copy of the state and fields and its
// flag word live in one file-scope __device__ array of fixed size, instead of
// in memory that mln_create allocates. The caller passes the state and field
// buffers; nothing else is allocated on the device.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "dispatch.cuh"
#include "mln.h"
#include "setup.h"

namespace {

// Every device that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[MLN_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};
CUcontext g_scratch_ctx[kMaxDevices] = {nullptr};  // the context the address belongs to

// The current driver context (through the runtime's entry-point query, so the
// library does not link libcuda); nullptr if that query is unavailable.
CUcontext current_context() {
    static CUresult (*get)(CUcontext *) = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get = reinterpret_cast<CUresult (*)(CUcontext *)>(fn);
    }
    CUcontext ctx = nullptr;
    if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    return ctx;
}

// Device address of the array on the current device, looked up with that
// device current at its first use and kept; looked up again when the
// device's context has changed since (after cudaDeviceReset the module is
// loaded anew and the array may sit elsewhere).
mln_status scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        mln::create_error() = "no current CUDA device";
        return MLN_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    const CUcontext ctx = current_context();  // nullptr before the runtime has made one current
    if (!g_scratch_addr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
            mln::create_error() = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return MLN_ECUDA;
        }
        g_scratch_addr[dev] = ptr;
        g_scratch_ctx[dev] = current_context();  // the lookup has made the device's context current
    }
    *out = g_scratch_addr[dev];
    return MLN_OK;
}

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Every medium cell starts from the same state vector, passed by value.
template <typename R>
struct InitVec {
    R v[MLN_MAX_N * MLN_MAX_N - 1];
};

template <typename R>
__global__ void fill_state_static(R *__restrict__ state, int64_t stride, int64_t count, int D,
                                  const __grid_constant__ InitVec<R> v) {
    int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (c >= count) return;
    for (int k = 0; k < D; ++k) state[k * stride + c] = v.v[k];
}

template <typename R>
mln_status run_static(const mln_params &p, const mln::Setup &s, void *d_state, void *Ez, void *Hy, int init_state,
                      int64_t n_steps, const double *src, cudaStream_t stream, void *scratch) {
    const int64_t n = p.n_cells, n_med = p.medium_end - p.medium_begin;
    const int64_t stride = mln::state_stride(p);
    const int D = s.D;
    const size_t state_bytes = static_cast<size_t>(D) * stride * sizeof(R);
    const size_t field_bytes = static_cast<size_t>(n) * sizeof(R);
    // layout: flags | state | E | H, each 256-byte aligned
    unsigned char *base = static_cast<unsigned char *>(scratch);
    unsigned int *flags = reinterpret_cast<unsigned int *>(base);
    R *st_alt = reinterpret_cast<R *>(base + 256);
    R *E_alt = reinterpret_cast<R *>(base + 256 + align256(state_bytes));
    R *H_alt = reinterpret_cast<R *>(base + 256 + align256(state_bytes) + align256(field_bytes));

    std::vector<unsigned char> consts;
    if (!mln::pack_consts(s, p.form, p.dt, R(0), consts)) {
        mln::create_error() = "no kernel for this N";
        return MLN_EUNSUPPORTED;
    }
    // the flag word keeps the previous call's value: clear it
    if (cudaMemsetAsync(flags, 0, sizeof(unsigned int), stream) != cudaSuccess) {
        mln::create_error() = "clearing the flag word failed";
        return MLN_ECUDA;
    }
    if (init_state && n_med > 0) {
        // the state of rho0 by the set-up's d -> state map, state = sp0 + Sp d0
        // (as mln_create builds it)
        InitVec<R> v{};
        for (int k = 0; k < D; ++k) {
            double acc = s.sp0[k];
            for (int j = 0; j < D; ++j) acc += s.Sp[k * D + j] * s.d0[j];
            v.v[k] = static_cast<R>(acc);
        }
        fill_state_static<R><<<static_cast<unsigned>((n_med + 255) / 256), 256, 0, stream>>>(
            static_cast<R *>(d_state), stride, n_med, D, v);
        if (cudaGetLastError() != cudaSuccess) {
            mln::create_error() = "initial state kernel launch failed";
            return MLN_ECUDA;
        }
    }
    // launch shape as mln_create's default, register model
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int K = p.block_steps > 0 ? p.block_steps : 16;
    if (2 * K > mln::kMaxThreads - 32) K = (mln::kMaxThreads - 32) / 2;
    int tile = p.tile_cells;
    if (tile <= 0) {
        int64_t ntiles = sms;
        tile = static_cast<int>((n + ntiles - 1) / ntiles);
        while (tile + 2 * K > mln::kMaxThreads) {
            ntiles += sms;
            tile = static_cast<int>((n + ntiles - 1) / ntiles);
        }
        tile = tile < 1 ? 1 : tile;
    }
    if (tile > n) tile = static_cast<int>(n);
    if (tile + 2 * K > mln::kMaxThreads) tile = mln::kMaxThreads - 2 * K;
    const int threads = (tile + 2 * K + 31) / 32 * 32;
    const int64_t ntiles = (n + tile - 1) / tile;

    const double eps = mln::kEps0 * p.eps_r, mu = mln::kMu0 * p.mu_r;
    const double sg = p.sigma * p.dt / (2.0 * eps);
    const double cv = 1.0 / std::sqrt(eps * mu);
    mln::BlockArgs<R> a{};
    a.flags = flags;
    a.n_cells = n;
    a.mb = p.medium_begin;
    a.me = p.medium_end;
    a.stride = stride;
    a.source_cell = p.source_cell;
    a.halo = K;
    a.tile = tile;
    a.boundary = p.boundary;
    a.source_kind = p.source_kind;
    a.ch = static_cast<R>(p.dt / (mu * p.dx));
    a.ca = static_cast<R>((1.0 - sg) / (1.0 + sg));
    a.cb = static_cast<R>((p.dt / eps) / (1.0 + sg));
    a.inv_dx = static_cast<R>(1.0 / p.dx);
    a.kappa = static_cast<R>((cv * p.dt - p.dx) / (cv * p.dt + p.dx));
    void *st[2] = {d_state, st_alt}, *E[2] = {Ez, E_alt}, *H[2] = {Hy, H_alt};
    const size_t smem = mln::field_smem<R>(threads);
    int cur = 0;
    for (int64_t done = 0; done < n_steps;) {
        int ns = static_cast<int>(n_steps - done < K ? n_steps - done : K);
        a.E_in = static_cast<const R *>(E[cur]);
        a.H_in = static_cast<const R *>(H[cur]);
        a.s_in = static_cast<const R *>(st[cur]);
        a.E_out = static_cast<R *>(E[cur ^ 1]);
        a.H_out = static_cast<R *>(H[cur ^ 1]);
        a.s_out = static_cast<R *>(st[cur ^ 1]);
        a.src = (src && p.source_kind != MLN_SRC_NONE) ? src + done : nullptr;
        a.nsteps = ns;
        cudaError_t e = mln::launch_block(p.N, p.form, a, consts, dim3(static_cast<unsigned>(ntiles)), dim3(threads),
                                          smem, stream);
        if (e != cudaSuccess) {
            mln::create_error() = std::string("step kernel launch: ") + cudaGetErrorString(e);
            return MLN_ECUDA;
        }
        cur ^= 1;
        done += ns;
    }
    if (cur == 1) {
        if (cudaMemcpyAsync(d_state, st_alt, state_bytes, cudaMemcpyDeviceToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(Ez, E_alt, field_bytes, cudaMemcpyDeviceToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(Hy, H_alt, field_bytes, cudaMemcpyDeviceToDevice, stream) != cudaSuccess) {
            mln::create_error() = "copy back from the static scratch failed";
            return MLN_ECUDA;
        }
    }
    return MLN_OK;
}


// Bytes of scratch a problem needs: flag word, alternate state, alternate E and H.
size_t scratch_bytes_for(const mln_params *p) {
    if (!p || p->N < 2 || p->N > MLN_MAX_N || p->n_cells < 0) return 0;
    const size_t r = p->precision == MLN_FP64 ? 8 : 4;
    const size_t D = static_cast<size_t>(p->N) * p->N - 1;
    const size_t state = D * static_cast<size_t>(mln::state_stride(*p)) * r;
    const size_t field = static_cast<size_t>(p->n_cells) * r;
    return 256 + align256(state) + 2 * align256(field);
}

}  // namespace

extern "C" {

mln_status mln_step_noalloc(const mln_params *p, void *d_state, void *Ez, void *Hy, int32_t init_state,
                            int64_t n_steps, const double *src, void *stream) {
    if (!p || !d_state || !Ez || !Hy || n_steps < 0) {
        mln::create_error() = "null argument or negative step count";
        return MLN_EINVAL;
    }
    std::string err;
    mln_status st = mln::validate(*p, err);
    if (st != MLN_OK) {
        mln::create_error() = err;
        return st;
    }
    if ((p->kernel != MLN_KERNEL_AUTO && p->kernel != MLN_KERNEL_REGISTER) || p->maxwell != MLN_MAXWELL_FDTD ||
        p->form == MLN_FORM_ROTATED) {
        mln::create_error() = "mln_step_noalloc runs the register cell model (kernel MLN_KERNEL_AUTO or "
                              "MLN_KERNEL_REGISTER; not the rotated form) with the FDTD field solver only";
        return MLN_EINVAL;
    }
    const size_t need = scratch_bytes_for(p);
    if (need > MLN_STATIC_SCRATCH_BYTES) {
        mln::create_error() = "problem needs " + std::to_string(need) + " bytes of scratch, above the static maximum of " +
                       std::to_string(static_cast<size_t>(MLN_STATIC_SCRATCH_BYTES)) + " bytes";
        return MLN_EINVAL;
    }
    mln::Setup s;
    st = mln::build_setup(*p, s, err);
    if (st != MLN_OK) {
        mln::create_error() = err;
        return st;
    }
    void *scratch = nullptr;
    if ((st = scratch_address(&scratch)) != MLN_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    return p->precision == MLN_FP64
               ? run_static<double>(*p, s, d_state, Ez, Hy, init_state, n_steps, src, cs, scratch)
               : run_static<float>(*p, s, d_state, Ez, Hy, init_state, n_steps, src, cs, scratch);
}

}  // extern "C"
