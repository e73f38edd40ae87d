// Pseudo-spectral (PSTD) field solver: the Maxwell part of a step with the
// spatial derivatives of Eq. 1 taken from the trigonometric interpolant of
// the periodic samples (the variant the paper's Secs. 1 and 3 say the method
// carries over to), and the unchanged Strang step of the medium (Eq. 23).
//
// One time step n -> n+1 on a ring of n_cells = 2^m cells:
//   1. medium cells: d^{n-1/2} -> d^{n+1/2} with E^n and dP/dt^{n+1/2}
//      (the cell models of the fused FDTD kernel, one step per launch);
//   2. H^{n+1/2} = H^{n-1/2} + dt/mu D+ E^n, D+ = F^-1 diag(i k e^{+i k dx/2}) F;
//   3. E^{n+1} = ca E^n + cb (D- H^{n+1/2} - dP/dt^{n+1/2}) + source,
//      D- = F^-1 diag(i k e^{-i k dx/2}) F,
// with k = 2 pi m / (n dx) for m <= n/2 and 2 pi (m - n) / (n dx) above (the
// Nyquist multiplier is the same real number for either sign of k).
//
// F is a four-step FFT, n = N1 N2 (N1, N2 powers of two up to 4096): a
// length-N1 transform of every stride-N2 column, the twiddle W_n^(i2 k1), a
// length-N2 transform of every row, output index k1 + N1 k2. Each of the two
// kernels gives one block to one column (row) and transforms it in shared
// memory with radix-4 (and one radix-2) Stockham stages, twiddles from an
// FP64-built table of e^{-2 pi i t / n}; the first forward kernel reads the
// real field, the first inverse kernel multiplies by the spectral multiplier
// (which carries 1/n and dt/mu), and the last inverse kernel applies the H or
// E update to the real part in place. A step is the medium kernel on a forked
// branch (it needs only E^n, like dE/dx) and the four kernels of each
// derivative; its launches are captured once into a CUDA graph (one step, and
// kGraphSteps steps) and replayed on the context's own stream, ordered after
// and before the caller's stream by events; in FP32 each transform kernel
// carries a programmatic dependency on the one before it, so it loads its
// tables while that one drains. The source sample of each step is
// read through a device-side cursor (base pointer and index) that the source
// cell's thread advances, so the captured launches do not change from step to
// step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "kernels.cuh"
#include "pstd.h"
#include "setup.h"

namespace mln {
namespace {

template <typename R>
struct Cx2;
template <>
struct Cx2<double> {
    using T = double2;
};
template <>
struct Cx2<float> {
    using T = float2;
};

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
    return {a.x + b.x, a.y + b.y};
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
    return {a.x - b.x, a.y - b.y};
}

// Programmatic dependent launch: the transform kernels may be launched so
// that they start while the kernel before them in the stream finishes. Each
// first loads its constant tables (twiddles and multipliers, written once at
// set-up), then waits for the grids it depends on to complete and their
// writes to be visible (a no-op when the launch carries no programmatic
// dependency), and only then reads or writes the work buffers and fields.
// Once its inputs are loaded, it lets the next kernel in the stream launch.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Source samples of an mln_step call and the index of the next one.
struct SrcCursor {
    const double *base;
    int64_t idx;
};

__global__ void set_cursor(SrcCursor *c, const double *base) {
    c->base = base;
    c->idx = 0;
}

enum { kEpiComplex = 0, kEpiH = 1, kEpiE = 2 };

template <typename R>
struct FsArgs {
    using C = typename Cx2<R>::T;
    const C *in;       // fs_cols: Z (nullptr: no update, only the forward transform of field)
                       // fs_rows_mid: Y
    C *out;            // fs_cols: Y of the updated field (nullptr: none); fs_rows_mid: Z
    const C *mult;     // fs_rows_mid: spectral multiplier of X[k1 + N1 k2]
    const C *tw;       // tw[t] = e^{-2 pi i t / n}, t < n
    int64_t n;
    int32_t N1, N2;
    int32_t epi;       // fs_cols with in: kEpiH (field += re) or kEpiE
    R *field;
    const R *dpdt;     // kEpiE: dP/dt^{n+1/2} (zero in vacuum cells)
    R ca, cb;
    SrcCursor *cursor;  // kEpiE: source samples (nullptr: no source)
    int64_t source_cell;
    int32_t source_kind;
    unsigned int *flags;
};

// 4-point DFT in place, natural order; the fourth root of unity is -i
// (forward) or +i (inverse).
template <typename C>
__device__ __forceinline__ void dft4(C &x0, C &x1, C &x2, C &x3, bool inverse) {
    const C a0 = cadd(x0, x2), a1 = csub(x0, x2);
    const C b0 = cadd(x1, x3), b1 = csub(x1, x3);
    const C ib1 = inverse ? C{-b1.y, b1.x} : C{b1.y, -b1.x};
    x0 = cadd(a0, b0);
    x2 = csub(a0, b0);
    x1 = cadd(a1, ib1);
    x3 = csub(a1, ib1);
}

// Length-L transform of s0 in shared memory (L a power of two), Stockham
// stages between s0 and s1: in a stage of radix R after sub-transforms of
// length Ns, butterfly b reads b + r L/R, applies W_L^(r k L/(R Ns)) (k = b
// mod Ns; wL[m] = W_L^m, in shared memory) and writes (b - k) R + k + q Ns.
// Returns the buffer that holds the result. All threads of the block call it.
template <typename C>
__device__ C *block_fft(C *s0, C *s1, int L, bool inv, const C *wL) {
    C *cur = s0, *nxt = s1;
    int Ns = 1;
    for (int m = L; m > 1;) {
        const int R = (m % 4 == 0) ? 4 : 2;
        const int q = L / R;
        const int step = L / (R * Ns);
        for (int b = threadIdx.x; b < q; b += blockDim.x) {
            const int k = b & (Ns - 1);
            const int base = (b - k) * R + k;
            if (R == 4) {
                C v0 = cur[b], v1 = cur[b + q], v2 = cur[b + 2 * q], v3 = cur[b + 3 * q];
                if (Ns > 1) {
                    C w1 = wL[k * step], w2 = wL[2 * k * step], w3 = wL[3 * k * step];
                    if (inv) {
                        w1.y = -w1.y;
                        w2.y = -w2.y;
                        w3.y = -w3.y;
                    }
                    v1 = cmul(v1, w1);
                    v2 = cmul(v2, w2);
                    v3 = cmul(v3, w3);
                }
                dft4(v0, v1, v2, v3, inv);
                nxt[base] = v0;
                nxt[base + Ns] = v1;
                nxt[base + 2 * Ns] = v2;
                nxt[base + 3 * Ns] = v3;
            } else {
                C v0 = cur[b], v1 = cur[b + q];
                if (Ns > 1) {
                    C w = wL[k * step];
                    if (inv) w.y = -w.y;
                    v1 = cmul(v1, w);
                }
                nxt[base] = cadd(v0, v1);
                nxt[base + Ns] = csub(v0, v1);
            }
        }
        __syncthreads();
        C *t = cur;
        cur = nxt;
        nxt = t;
        Ns *= R;
        m /= R;
    }
    return cur;
}

// Elements per thread of a transform kernel: L / blockDim.x <= kMaxPer.
constexpr int kMaxPer = 16;

// A derivative is three steps of the four-step transform (n = N1 N2, x at
// N2 i1 + i2, X at k1 + N1 k2):
//   forward columns:  Y[k1 N2 + i2] = W_n^(i2 k1) sum_i1 x[N2 i1 + i2] W_N1^(i1 k1)
//   rows (fs_rows_mid): X[k1 + N1 k2] = sum_i2 Y[k1 N2 + i2] W_N2^(i2 k2), times the
//                     multiplier, then Z[k1 N2 + i2] = W_n^(-i2 k1) sum_k2 X[k1 + N1 k2] W_N2^(-i2 k2)
//   inverse columns:  x'[N2 i1 + i2] = sum_k1 Z[k1 N2 + i2] W_N1^(-i1 k1)
// The inverse column pass of one derivative and the forward column pass of
// the next work on the same column, so fs_cols does both: it updates the
// field from x' and transforms the updated column.

// Column kernel, block i2: (if in) the inverse transform of column i2 of Z
// and the update of the field there; (if out) the forward transform of the
// field's column i2, twiddled, into Y. Global loads are issued before the
// first stage.
template <typename R>
__global__ void __launch_bounds__(256) fs_cols(const __grid_constant__ FsArgs<R> a) {
    using C = typename Cx2<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = a.N1;
    C *s0 = reinterpret_cast<C *>(smem), *s1 = s0 + L, *wL = s1 + L;
    const int64_t i2 = blockIdx.x;
    const int64_t tstep = a.n / L;
    C wo[kMaxPer];
    R fv[kMaxPer];
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
        const int i = threadIdx.x + j * blockDim.x;
        if (i < L) {
            wL[i] = a.tw[i * tstep];
            if (a.out) wo[j] = a.tw[i2 * i];
        }
    }
    grid_dep_wait();
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
        const int i = threadIdx.x + j * blockDim.x;
        if (i < L) {
            const int64_t idx = static_cast<int64_t>(a.N2) * i + i2;
            fv[j] = a.field[idx];
            if (a.in) s0[i] = a.in[idx];
        }
    }
    grid_dep_launch();
    C *x = s0, *scratch = s1;
    if (a.in) {
        __syncthreads();
        const C *f = block_fft(s0, s1, L, true, wL);
        C *g = (f == s0) ? s1 : s0;
#pragma unroll
        for (int j = 0; j < kMaxPer; ++j) {
            const int i1 = threadIdx.x + j * blockDim.x;
            if (i1 < L) {
                const int64_t idx = static_cast<int64_t>(a.N2) * i1 + i2;
                const R d = f[i1].x;
                R v;
                if (a.epi == kEpiH) {
                    v = fv[j] + d;
                } else {
                    v = a.ca * fv[j] + a.cb * (d - a.dpdt[idx]);
                    if (a.cursor != nullptr && idx == a.source_cell) {
                        const SrcCursor cur = *a.cursor;
                        if (cur.base != nullptr) {
                            const R s = static_cast<R>(cur.base[cur.idx]);
                            v = (a.source_kind == MLN_SRC_HARD) ? s : v + s;
                        }
                        a.cursor->idx = cur.idx + 1;  // the one reader of this step; the next step reads after this launch
                    }
                    if (!isfinite(v)) atomicOr(a.flags, 1u);
                }
                a.field[idx] = v;
                fv[j] = v;
            }
        }
        x = g;
        scratch = const_cast<C *>(f);
    }
    if (!a.out) return;
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
        const int i1 = threadIdx.x + j * blockDim.x;
        if (i1 < L) x[i1] = C{fv[j], R(0)};
    }
    __syncthreads();
    const C *f = block_fft(x, scratch, L, false, wL);
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
        const int k1 = threadIdx.x + j * blockDim.x;
        if (k1 < L) a.out[static_cast<int64_t>(k1) * a.N2 + i2] = cmul(f[k1], wo[j]);
    }
}

// Row kernel, block k1: forward transform of row k1 of Y (output k2 is
// X[k1 + N1 k2]), times the multiplier, inverse transform over k2, twiddle
// W_n^(-i2 k1), into row k1 of Z.
template <typename R>
__global__ void __launch_bounds__(256) fs_rows_mid(const __grid_constant__ FsArgs<R> a) {
    using C = typename Cx2<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = a.N2;
    C *s0 = reinterpret_cast<C *>(smem), *s1 = s0 + L, *wL = s1 + L;
    const int64_t k1 = blockIdx.x;
    const int64_t tstep = a.n / L;
    C mu[kMaxPer], wo[kMaxPer];
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
        const int i = threadIdx.x + j * blockDim.x;
        if (i < L) {
            wL[i] = a.tw[i * tstep];
            mu[j] = a.mult[k1 + static_cast<int64_t>(a.N1) * i];
            C w = a.tw[i * k1];
            w.y = -w.y;
            wo[j] = w;
        }
    }
    grid_dep_wait();
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
        const int i = threadIdx.x + j * blockDim.x;
        if (i < L) s0[i] = a.in[k1 * L + i];
    }
    grid_dep_launch();
    __syncthreads();
    C *f = block_fft(s0, s1, L, false, wL);
    C *g = (f == s0) ? s1 : s0;
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
        const int k2 = threadIdx.x + j * blockDim.x;
        if (k2 < L) f[k2] = cmul(f[k2], mu[j]);
    }
    __syncthreads();
    const C *z = block_fft(f, g, L, true, wL);
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
        const int i2 = threadIdx.x + j * blockDim.x;
        if (i2 < L) a.out[k1 * L + i2] = cmul(z[i2], wo[j]);
    }
}

template <typename R>
struct CellArgs {
    R *state;
    const R *E;
    R *dpdt;
    int64_t stride, n_med, mb;
};

// One Strang step of every medium cell with the field E^n of its cell;
// dP/dt^{n+1/2} goes to dpdt at the cell's grid index.
template <int N, typename R, typename Cell>
__global__ void __launch_bounds__(256)
    pstd_cell_kernel(const __grid_constant__ CellArgs<R> a, const __grid_constant__ typename Cell::Consts k) {
    extern __shared__ __align__(16) unsigned char smem[];
    Cell cell;
    cell.setup(smem, k);
    __syncthreads();
    const int64_t m = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (m >= a.n_med) return;
    cell.load(a.state, a.stride, m);
    const R dpdt = cell.step(a.E[a.mb + m], k);
    cell.end_step();
    cell.store(a.state, a.stride, m);
    a.dpdt[a.mb + m] = dpdt;
}

template <int N, typename R, typename K>
cudaError_t launch_cell_register(const CellArgs<R> &a, const std::vector<unsigned char> &consts, cudaStream_t st) {
    K k;
    if (consts.size() != sizeof(K)) return cudaErrorInvalidValue;
    std::memcpy(&k, consts.data(), sizeof(K));
    const unsigned grid = static_cast<unsigned>((a.n_med + 255) / 256);
    pstd_cell_kernel<N, R, RegisterCell<N, R, K>><<<grid, 256, 0, st>>>(a, k);
    return cudaGetLastError();
}

constexpr int kSparseThreads = 128;

template <int N>
size_t sparse_cell_smem(const mln_ctx *c) {
    return SharedSparseCell<N>::smem_bytes(kSparseThreads, c->nnz, c->nrowptr);
}

// The sparse cell kernel's shared memory can exceed the 48 KB default: raise
// its limit once, before any launch is captured.
template <int N>
cudaError_t prepare_sparse(const mln_ctx *c) {
    return cudaFuncSetAttribute(pstd_cell_kernel<N, double, SharedSparseCell<N>>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sparse_cell_smem<N>(c)));
}

template <int N>
cudaError_t launch_cell_sparse(const mln_ctx *c, const CellArgs<double> &a, cudaStream_t st) {
    SparseConsts<N> k;
    if (c->consts.size() != sizeof(k)) return cudaErrorInvalidValue;
    std::memcpy(&k, c->consts.data(), sizeof(k));
    const unsigned grid = static_cast<unsigned>((a.n_med + kSparseThreads - 1) / kSparseThreads);
    pstd_cell_kernel<N, double, SharedSparseCell<N>><<<grid, kSparseThreads, sparse_cell_smem<N>(c), st>>>(a, k);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cells(const mln_ctx *c, const CellArgs<R> &a, cudaStream_t st) {
    const int N = c->p.N, form = c->p.form;
    if constexpr (sizeof(R) == 8) {
        if (c->sparse) {
            switch (N) {
            case 2: return launch_cell_sparse<2>(c, a, st);
            case 3: return launch_cell_sparse<3>(c, a, st);
            case 4: return launch_cell_sparse<4>(c, a, st);
            case 5: return launch_cell_sparse<5>(c, a, st);
            case 6: return launch_cell_sparse<6>(c, a, st);
            default: return cudaErrorInvalidValue;
            }
        }
    }
    if (form == MLN_FORM_RODRIGUES) {
        switch (N) {
        case 2: return launch_cell_register<2, R, RodriguesConsts<2, R>>(a, c->consts, st);
        case 3: return launch_cell_register<3, R, RodriguesConsts<3, R>>(a, c->consts, st);
        case 4: return launch_cell_register<4, R, RodriguesConsts<4, R>>(a, c->consts, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (N) {
#define MLN_PSTD_CASE(NN)                                                                     \
    case NN:                                                                                  \
        if (form == MLN_FORM_STRANG)                                                          \
            return launch_cell_register<NN, R, StrangConsts<NN, R>>(a, c->consts, st);        \
        return launch_cell_register<NN, R, MergedConsts<NN, R>>(a, c->consts, st);
        MLN_PSTD_CASE(2)
        MLN_PSTD_CASE(3)
        MLN_PSTD_CASE(4)
        MLN_PSTD_CASE(5)
        MLN_PSTD_CASE(6)
#undef MLN_PSTD_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

// Device layout of the one allocation: work0 | work1 | tw | mult_h | mult_e
// (n complex each), dpdt (n reals), the source cursor.
template <typename R>
struct Layout {
    using C = typename Cx2<R>::T;
    C *work0, *work1, *tw, *mh, *me;
    R *dpdt;
    SrcCursor *cursor;
    static size_t cursor_off(int64_t n) { return (5 * n * sizeof(C) + n * sizeof(R) + 15) / 16 * 16; }
    static size_t bytes(int64_t n) { return cursor_off(n) + sizeof(SrcCursor); }
    Layout(void *base, int64_t n) {
        C *p = static_cast<C *>(base);
        work0 = p;
        work1 = p + n;
        tw = p + 2 * n;
        mh = p + 3 * n;
        me = p + 4 * n;
        dpdt = reinterpret_cast<R *>(p + 5 * n);
        cursor = reinterpret_cast<SrcCursor *>(static_cast<unsigned char *>(base) + cursor_off(n));
    }
};

// n = N1 N2 with N1 <= N2 <= 2 N1 (powers of two).
void split(int64_t n, int *N1, int *N2) {
    int m = 0;
    while ((int64_t(1) << m) < n) ++m;
    *N1 = 1 << (m / 2);
    *N2 = 1 << (m - m / 2);
}

// at most kMaxPer elements per thread
int block_threads(int L) { return std::min(256, std::max(32, L / 4)); }

// two buffers and the W_L table
template <typename R>
size_t fs_smem(int L) {
    return 3 * static_cast<size_t>(L) * sizeof(typename Cx2<R>::T);
}

template <typename R>
FsArgs<R> fs_base(const mln_ctx *c, const Layout<R> &L) {
    FsArgs<R> a{};
    int N1, N2;
    split(c->p.n_cells, &N1, &N2);
    a.n = c->p.n_cells;
    a.N1 = N1;
    a.N2 = N2;
    a.tw = L.tw;
    a.flags = c->flags;
    return a;
}

// A transform kernel; in FP32 launched with a programmatic dependency on the
// kernel before it in the stream (captured as a programmatic graph edge).
// FP32 transforms are latency-bound, and starting each while the previous
// one drains shortens the step (28.6 -> 20.8 us at 65536 cells). The FP64
// transforms run about one warp per SM sub-partition, limited by the latency
// of dependent FP64 operations; blocks placed early leave SMs unevenly loaded
// beside the overlapping medium kernel, and the FP64 step took longer
// (76 -> 87 us), so FP64 launches carry no such dependency.
template <typename R>
cudaError_t launch_fs(void (*kernel)(FsArgs<R>), const FsArgs<R> &a, int blocks, int L, cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(static_cast<unsigned>(block_threads(L)));
    cfg.dynamicSmemBytes = fs_smem<R>(L);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = sizeof(R) == 4 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <typename R>
cudaError_t launch_cols(const FsArgs<R> &a, cudaStream_t st) {
    return launch_fs<R>(fs_cols<R>, a, a.N2, a.N1, st);
}

template <typename R>
cudaError_t launch_rows(const FsArgs<R> &a, cudaStream_t st) {
    return launch_fs<R>(fs_rows_mid<R>, a, a.N1, a.N2, st);
}

// Y of E^n into work0 (the first kernel of every mln_step call).
template <typename R>
cudaError_t enqueue_prologue(const mln_ctx *c, cudaStream_t st) {
    Layout<R> L(c->pstd, c->p.n_cells);
    FsArgs<R> a = fs_base<R>(c, L);
    a.field = static_cast<R *>(c->E[0]);
    a.out = L.work0;
    return launch_cols<R>(a, st);
}

struct Host {
    cudaStream_t stream = nullptr, side = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t one = nullptr, many = nullptr;  // 1 step, kGraphSteps steps
};

// One step on h->stream, entered with Y of E^n in work0: the medium kernel on
// the side branch (it reads E^n); rows of the E derivative (work0 -> work1);
// H update and Y of H^{n+1/2} (work1 -> work0); rows of the H derivative;
// after the medium kernel, E update and Y of E^{n+1} (work1 -> work0).
template <typename R>
cudaError_t enqueue_step(const mln_ctx *c, Host *h) {
    Layout<R> L(c->pstd, c->p.n_cells);
    const BlockArgs<R> b = base_args<R>(c);
    R *E = static_cast<R *>(c->E[0]);
    R *H = static_cast<R *>(c->H[0]);
    cudaError_t e = cudaSuccess;
    const bool medium = c->n_med > 0;
    if (medium) {
        e = cudaEventRecord(h->ev_fork, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
        const CellArgs<R> ca{static_cast<R *>(c->st[0]), E, L.dpdt, c->stride, c->n_med, c->p.medium_begin};
        if (e == cudaSuccess) e = launch_cells<R>(c, ca, h->side);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->side);
    }
    FsArgs<R> r = fs_base<R>(c, L);
    r.in = L.work0;
    r.out = L.work1;
    r.mult = L.mh;
    if (e == cudaSuccess) e = launch_rows<R>(r, h->stream);
    FsArgs<R> ch = fs_base<R>(c, L);
    ch.in = L.work1;
    ch.out = L.work0;
    ch.epi = kEpiH;
    ch.field = H;
    if (e == cudaSuccess) e = launch_cols<R>(ch, h->stream);
    r.mult = L.me;
    if (e == cudaSuccess) e = launch_rows<R>(r, h->stream);
    if (e == cudaSuccess && medium) e = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
    FsArgs<R> ce = fs_base<R>(c, L);
    ce.in = L.work1;
    ce.out = L.work0;
    ce.epi = kEpiE;
    ce.field = E;
    ce.dpdt = L.dpdt;
    ce.ca = b.ca;
    ce.cb = b.cb;
    ce.cursor = c->p.source_kind != MLN_SRC_NONE ? L.cursor : nullptr;
    ce.source_cell = c->p.source_cell;
    ce.source_kind = c->p.source_kind;
    if (e == cudaSuccess) e = launch_cols<R>(ce, h->stream);
    return e;
}

constexpr int kGraphSteps = 16;

template <typename R>
cudaError_t capture(const mln_ctx *c, Host *h, int steps, cudaGraphExec_t *out) {
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (int s = 0; s < steps && le == cudaSuccess; ++s) le = enqueue_step<R>(c, h);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->stream, &g);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

template <typename R>
mln_status init_t(mln_ctx *c) {
    using C = typename Cx2<R>::T;
    const int64_t n = c->p.n_cells;
    if (cudaMalloc(&c->pstd, Layout<R>::bytes(n)) != cudaSuccess) {
        cudaGetLastError();
        c->pstd = nullptr;
        c->err = "PSTD tables: device allocation failed";
        return MLN_ENOMEM;
    }
    Layout<R> L(c->pstd, n);
    const double two_pi = 6.283185307179586476925286766559;
    const double mu = kMu0 * c->p.mu_r, dx = c->p.dx, dt = c->p.dt;
    std::vector<C> tw(n), mh(n), me(n);
    for (int64_t t = 0; t < n; ++t) {
        const double ang = two_pi * static_cast<double>(t) / static_cast<double>(n);
        tw[t] = {static_cast<R>(std::cos(ang)), static_cast<R>(-std::sin(ang))};
        const int64_t ms = (t <= n / 2) ? t : t - n;
        const double kk = two_pi * static_cast<double>(ms) / (static_cast<double>(n) * dx);
        const double th = 0.5 * kk * dx;
        // i k e^{+-i th} = (-+k sin th, k cos th); 1/n of the inverse transform, dt/mu for H
        const double sh = dt / mu / static_cast<double>(n), se = 1.0 / static_cast<double>(n);
        mh[t] = {static_cast<R>(-kk * std::sin(th) * sh), static_cast<R>(kk * std::cos(th) * sh)};
        me[t] = {static_cast<R>(kk * std::sin(th) * se), static_cast<R>(kk * std::cos(th) * se)};
    }
    cudaError_t e = cudaMemcpy(L.tw, tw.data(), n * sizeof(C), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.mh, mh.data(), n * sizeof(C), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.me, me.data(), n * sizeof(C), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(L.dpdt, 0, n * sizeof(R));
    if (e == cudaSuccess) e = cudaMemset(L.cursor, 0, sizeof(SrcCursor));
    if (e == cudaSuccess && sizeof(R) == 8 && c->sparse) {
        switch (c->p.N) {
        case 2: e = prepare_sparse<2>(c); break;
        case 3: e = prepare_sparse<3>(c); break;
        case 4: e = prepare_sparse<4>(c); break;
        case 5: e = prepare_sparse<5>(c); break;
        case 6: e = prepare_sparse<6>(c); break;
        default: e = cudaErrorInvalidValue;
        }
    }
    Host *h = new (std::nothrow) Host();
    c->pstd_host = h;
    if (!h) return MLN_ENOMEM;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    // the transforms' shared memory (two buffers of the longer side) can exceed the 48 KB default
    int N1, N2;
    split(n, &N1, &N2);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fs_cols<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(fs_smem<R>(N1)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fs_rows_mid<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(fs_smem<R>(N2)));
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("PSTD set-up: ") + cudaGetErrorString(e);
        return MLN_ECUDA;
    }
    return MLN_OK;
}

template <typename R>
mln_status steps_t(mln_ctx *c, int64_t n_steps, const double *src) {
    Host *h = static_cast<Host *>(c->pstd_host);
    Layout<R> L(c->pstd, c->p.n_cells);
    cudaError_t e = cudaSuccess;
    if (!h->one) e = capture<R>(c, h, 1, &h->one);
    if (e == cudaSuccess && !h->many && n_steps >= kGraphSteps) e = capture<R>(c, h, kGraphSteps, &h->many);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_in, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_in, 0);
    if (e == cudaSuccess) {
        set_cursor<<<1, 1, 0, h->stream>>>(L.cursor, c->p.source_kind != MLN_SRC_NONE ? src : nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = enqueue_prologue<R>(c, h->stream);
        c->launches += 2;
    }
    const int64_t per_step = pstd_launches_per_step(c->p.n_cells, c->n_med);
    int64_t done = 0;
    for (; e == cudaSuccess && done + kGraphSteps <= n_steps; done += kGraphSteps) e = cudaGraphLaunch(h->many, h->stream);
    for (; e == cudaSuccess && done < n_steps; ++done) e = cudaGraphLaunch(h->one, h->stream);
    c->launches += done * per_step;
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_out, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, h->ev_out, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("PSTD step: ") + cudaGetErrorString(e);
        return MLN_ECUDA;
    }
    return MLN_OK;
}

}  // namespace

mln_status pstd_init(mln_ctx *c) { return c->p.precision == MLN_FP64 ? init_t<double>(c) : init_t<float>(c); }

void pstd_free(mln_ctx *c) {
    if (Host *h = static_cast<Host *>(c->pstd_host)) {
        if (h->stream) cudaStreamSynchronize(h->stream);
        if (h->one) cudaGraphExecDestroy(h->one);
        if (h->many) cudaGraphExecDestroy(h->many);
        if (h->ev_in) cudaEventDestroy(h->ev_in);
        if (h->ev_out) cudaEventDestroy(h->ev_out);
        if (h->ev_fork) cudaEventDestroy(h->ev_fork);
        if (h->ev_join) cudaEventDestroy(h->ev_join);
        if (h->side) cudaStreamDestroy(h->side);
        if (h->stream) cudaStreamDestroy(h->stream);
        delete h;
    }
    c->pstd_host = nullptr;
    if (c->pstd) cudaFree(c->pstd);
    c->pstd = nullptr;
}

mln_status pstd_steps(mln_ctx *c, int64_t n_steps, const double *src) {
    if (!c->pstd || !c->pstd_host) return MLN_EINVAL;
    return c->p.precision == MLN_FP64 ? steps_t<double>(c, n_steps, src) : steps_t<float>(c, n_steps, src);
}

int pstd_launches_per_step(int64_t n_cells, int64_t n_medium) {
    (void)n_cells;
    return (n_medium > 0 ? 1 : 0) + 4;
}

}  // namespace mln
