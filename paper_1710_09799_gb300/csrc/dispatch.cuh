// Packing of the per-context constants and launch of the fused step kernel
// for one precision (internal; included by kernels_fp64.cu / kernels_fp32.cu).
#pragma once

#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "setup.h"

namespace mln {

template <int N, typename R>
void pack_strang(const Setup &s, double dt, std::vector<unsigned char> &out) {
    constexpr int D = Dims<N>::D;
    StrangConsts<N, R> k;
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
    k.c = static_cast<R>(s.c);
    out.resize(sizeof(k));
    std::memcpy(out.data(), &k, sizeof(k));
}

template <int N, typename R>
void pack_merged(const Setup &s, double dt, std::vector<unsigned char> &out) {
    constexpr int D = Dims<N>::D;
    MergedConsts<N, R> k;
    std::memset(&k, 0, sizeof(k));
    for (int i = 0; i < D * D; ++i) {
        k.C1[i] = static_cast<R>(s.C1[i]);
        k.T[i] = static_cast<R>(s.T[i]);
    }
    for (int i = 0; i < D; ++i) {
        k.b2[i] = static_cast<R>(s.b2[i]);
        k.wm[i] = static_cast<R>(s.wm[i]);
    }
    for (int a = 0; a < N - 1; ++a) k.psi_dt[a] = static_cast<R>(s.psi[a] * dt);
    k.cm = static_cast<R>(s.cm);
    out.resize(sizeof(k));
    std::memcpy(out.data(), &k, sizeof(k));
}

// S_k = T Theta_k T^T (Theta_k: -1 at (2k, 2k+1), +1 at (2k+1, 2k)) and S_k^2, in FP64.
template <int N, typename R>
void pack_rodrigues(const Setup &s, double dt, std::vector<unsigned char> &out) {
    constexpr int D = Dims<N>::D, Q = Dims<N>::Q;
    RodriguesConsts<N, R> k;
    std::memset(&k, 0, sizeof(k));
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) k.Dl[i * D + j] = static_cast<R>(s.A0[i * D + j] - (i == j ? 1.0 : 0.0));
    std::vector<double> S(D * D), S2(D * D);
    for (int p = 0; p < Q; ++p) {
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j)
                S[i * D + j] = -s.T[i * D + 2 * p] * s.T[j * D + 2 * p + 1] + s.T[i * D + 2 * p + 1] * s.T[j * D + 2 * p];
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                double acc = 0;
                for (int l = 0; l < D; ++l) acc += S[i * D + l] * S[l * D + j];
                S2[i * D + j] = acc;
            }
        for (int i = 0; i < D * D; ++i) {
            k.S[p * D * D + i] = static_cast<R>(S[i]);
            k.S2[p * D * D + i] = static_cast<R>(S2[i]);
        }
    }
    for (int i = 0; i < D; ++i) {
        k.b[i] = static_cast<R>(s.b[i]);
        k.w[i] = static_cast<R>(s.w[i]);
    }
    for (int a = 0; a < N - 1; ++a) k.psi_dt[a] = static_cast<R>(s.psi[a] * dt);
    k.c = static_cast<R>(s.c);
    out.resize(sizeof(k));
    std::memcpy(out.data(), &k, sizeof(k));
}

template <typename R>
bool pack_consts_t(const Setup &s, int form, double dt, std::vector<unsigned char> &out) {
    if (form == MLN_FORM_RODRIGUES) {
        switch (s.N) {
        case 2: pack_rodrigues<2, R>(s, dt, out); return true;
        case 3: pack_rodrigues<3, R>(s, dt, out); return true;
        case 4: pack_rodrigues<4, R>(s, dt, out); return true;
        default: return false;
        }
    }
    switch (s.N) {
#define MLN_PACK_CASE(NN)                                        \
    case NN:                                                     \
        if (form == MLN_FORM_STRANG) pack_strang<NN, R>(s, dt, out); \
        else pack_merged<NN, R>(s, dt, out);                        \
        return true;
        MLN_PACK_CASE(2)
        MLN_PACK_CASE(3)
        MLN_PACK_CASE(4)
        MLN_PACK_CASE(5)
        MLN_PACK_CASE(6)
#undef MLN_PACK_CASE
    default:
        return false;
    }
}

// A step kernel launch, with (programmatic) or without a programmatic
// dependency on the kernel before it in the stream (mln_block_kernel waits for
// that grid before it touches the fields): with one, the launch is prepared
// while the previous grid runs and its blocks start as soon as that grid
// completes. Launches beside concurrent work on another stream go without:
// blocks placed early hold SM resources that work needs.
template <typename... P, typename... A>
cudaError_t launch_dependent(bool programmatic, void (*kern)(P...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t st, const A &...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = programmatic ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int N, typename R, typename K>
cudaError_t launch_one(const BlockArgs<R> &a, const std::vector<unsigned char> &consts, dim3 grid,
                       dim3 block, size_t smem, cudaStream_t st, bool programmatic) {
    K k;
    if (consts.size() != sizeof(K)) return cudaErrorInvalidValue;
    std::memcpy(&k, consts.data(), sizeof(K));
    return launch_dependent(programmatic, mln_block_kernel<N, R, RegisterCell<N, R, K>>, grid, block, smem, st, a,
                            k);
}

// The sparse program of the merged FP64 step (see SparseConsts): entries of
// T^T on the plane rows, T on the plane columns, A0^2 - I and A0^T w whose
// FP64 value is not exactly zero.
inline void build_sparse_program(const Setup &s, std::vector<int32_t> &rowptr, std::vector<int32_t> &cols,
                                 std::vector<double> &vals) {
    const int D = s.D, P = 2 * s.q;
    rowptr.clear();
    cols.clear();
    vals.clear();
    auto put = [&](int c, double v) {
        if (v != 0.0) {
            cols.push_back(c);
            vals.push_back(v);
        }
    };
    for (int r = 0; r < P; ++r) {  // z_r = sum_i T[i][r] y_i
        rowptr.push_back(static_cast<int32_t>(vals.size()));
        for (int i = 0; i < D; ++i) put(i, s.T[i * D + r]);
    }
    rowptr.push_back(static_cast<int32_t>(vals.size()));
    for (int r = 0; r < D; ++r) {  // y_r += sum_k T[r][k] z_k
        for (int k = 0; k < P; ++k) put(k, s.T[r * D + k]);
        rowptr.push_back(static_cast<int32_t>(vals.size()));
    }
    for (int r = 0; r < D; ++r) {  // (C1 y)_r
        for (int j = 0; j < D; ++j) put(j, s.C1[r * D + j]);
        rowptr.push_back(static_cast<int32_t>(vals.size()));
    }
    for (int i = 0; i < D; ++i) put(i, s.wm[i]);  // wm . y
    rowptr.push_back(static_cast<int32_t>(vals.size()));
}

template <int N>
void pack_sparse(const Setup &s, double dt, const int32_t *rowptr, const int32_t *cols, const double *vals,
                 int nnz, int nrowptr, std::vector<unsigned char> &out) {
    SparseConsts<N> k;
    std::memset(&k, 0, sizeof(k));
    for (int i = 0; i < Dims<N>::D; ++i) k.b2[i] = s.b2[i];
    for (int a = 0; a < N - 1; ++a) k.psi_dt[a] = s.psi[a] * dt;
    k.cm = s.cm;
    k.rowptr = rowptr;
    k.cols = cols;
    k.vals = vals;
    k.nnz = nnz;
    k.nrowptr = nrowptr;
    out.resize(sizeof(k));
    std::memcpy(out.data(), &k, sizeof(k));
}

template <int N>
cudaError_t launch_sparse_one(const BlockArgs<double> &a, const std::vector<unsigned char> &consts, dim3 grid,
                              dim3 block, size_t smem, cudaStream_t st) {
    SparseConsts<N> k;
    if (consts.size() != sizeof(k)) return cudaErrorInvalidValue;
    std::memcpy(&k, consts.data(), sizeof(k));
    auto kern = mln_block_kernel<N, double, SharedSparseCell<N>>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return launch_dependent(true, kern, grid, block, smem, st, a, k);
}

// The Strang step with its intermediates traced (mln_trace_kernel), N <= 4,
// at most 256 threads a block: the adjoint's recomputation.
template <typename R>
cudaError_t launch_block_trace_t(int N, const BlockArgs<R> &a, const std::vector<unsigned char> &consts, dim3 grid,
                                 dim3 block, size_t smem, cudaStream_t st, bool programmatic) {
    switch (N) {
#define MLN_TRACE_CASE(NN)                                                                                  \
    case NN: {                                                                                              \
        StrangConsts<NN, R> k;                                                                              \
        if (consts.size() != sizeof(k)) return cudaErrorInvalidValue;                                       \
        std::memcpy(&k, consts.data(), sizeof(k));                                                          \
        if (block.x > 256) return cudaErrorInvalidValue;                                                   \
        return launch_dependent(programmatic, mln_trace_kernel<NN, R>, grid, block, smem, st, a, k);       \
    }
        MLN_TRACE_CASE(2)
        MLN_TRACE_CASE(3)
        MLN_TRACE_CASE(4)
#undef MLN_TRACE_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

template <typename R>
cudaError_t launch_block_t(int N, int form, const BlockArgs<R> &a, const std::vector<unsigned char> &consts,
                           dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool programmatic) {
    if (form == MLN_FORM_RODRIGUES) {
        switch (N) {
        case 2: return launch_one<2, R, RodriguesConsts<2, R>>(a, consts, grid, block, smem, st, programmatic);
        case 3: return launch_one<3, R, RodriguesConsts<3, R>>(a, consts, grid, block, smem, st, programmatic);
        case 4: return launch_one<4, R, RodriguesConsts<4, R>>(a, consts, grid, block, smem, st, programmatic);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (N) {
#define MLN_LAUNCH_CASE(NN)                                                                     \
    case NN:                                                                                    \
        if (form == MLN_FORM_STRANG)                                                            \
            return launch_one<NN, R, StrangConsts<NN, R>>(a, consts, grid, block, smem, st, programmatic);    \
        return launch_one<NN, R, MergedConsts<NN, R>>(a, consts, grid, block, smem, st, programmatic);
        MLN_LAUNCH_CASE(2)
        MLN_LAUNCH_CASE(3)
        MLN_LAUNCH_CASE(4)
        MLN_LAUNCH_CASE(5)
        MLN_LAUNCH_CASE(6)
#undef MLN_LAUNCH_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

// Entry points defined once per precision.
bool pack_consts(const Setup &s, int form, double dt, double tag, std::vector<unsigned char> &out);
bool pack_consts(const Setup &s, int form, double dt, float tag, std::vector<unsigned char> &out);
// programmatic: launch with a programmatic dependency on the kernel before it
cudaError_t launch_block(int N, int form, const BlockArgs<double> &a, const std::vector<unsigned char> &consts,
                         dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool programmatic = true);
cudaError_t launch_block(int N, int form, const BlockArgs<float> &a, const std::vector<unsigned char> &consts,
                         dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool programmatic = true);
cudaError_t launch_block_trace(int N, const BlockArgs<double> &a, const std::vector<unsigned char> &consts,
                               dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool programmatic);
cudaError_t launch_block_trace(int N, const BlockArgs<float> &a, const std::vector<unsigned char> &consts,
                               dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool programmatic);
cudaError_t launch_sin_cosm1(int precision, const double *x, int64_t n, double *s, double *c1, cudaStream_t st);
bool pack_sparse_consts(const Setup &s, double dt, const int32_t *rowptr, const int32_t *cols, const double *vals,
                        int nnz, int nrowptr, std::vector<unsigned char> &out);
cudaError_t launch_block_sparse(int N, const BlockArgs<double> &a, const std::vector<unsigned char> &consts,
                                dim3 grid, dim3 block, size_t smem, cudaStream_t st);
size_t sparse_smem_bytes(int N, int threads, int nnz, int nrowptr);

}  // namespace mln
