// Instantiation of the fused step kernels for double (N = 2..6, both forms).
#include "dispatch.cuh"

namespace mln {

bool pack_consts(const Setup &s, int form, double dt, double, std::vector<unsigned char> &out) {
    return pack_consts_t<double>(s, form, dt, out);
}

cudaError_t launch_block_trace(int N, const BlockArgs<double> &a, const std::vector<unsigned char> &consts,
                               dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool programmatic) {
    return launch_block_trace_t<double>(N, a, consts, grid, block, smem, st, programmatic);
}

cudaError_t launch_block(int N, int form, const BlockArgs<double> &a, const std::vector<unsigned char> &consts,
                         dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool programmatic) {
    return launch_block_t<double>(N, form, a, consts, grid, block, smem, st, programmatic);
}

cudaError_t launch_sin_cosm1(int precision, const double *x, int64_t n, double *s, double *c1, cudaStream_t st) {
    const unsigned grid = static_cast<unsigned>((n + 255) / 256);
    if (n <= 0) return cudaSuccess;
    if (precision == MLN_FP64) sin_cosm1_kernel<double><<<grid, 256, 0, st>>>(x, n, s, c1);
    else sin_cosm1_kernel<float><<<grid, 256, 0, st>>>(x, n, s, c1);
    return cudaGetLastError();
}

bool pack_sparse_consts(const Setup &s, double dt, const int32_t *rowptr, const int32_t *cols, const double *vals,
                        int nnz, int nrowptr, std::vector<unsigned char> &out) {
    switch (s.N) {
    case 2: pack_sparse<2>(s, dt, rowptr, cols, vals, nnz, nrowptr, out); return true;
    case 3: pack_sparse<3>(s, dt, rowptr, cols, vals, nnz, nrowptr, out); return true;
    case 4: pack_sparse<4>(s, dt, rowptr, cols, vals, nnz, nrowptr, out); return true;
    case 5: pack_sparse<5>(s, dt, rowptr, cols, vals, nnz, nrowptr, out); return true;
    case 6: pack_sparse<6>(s, dt, rowptr, cols, vals, nnz, nrowptr, out); return true;
    default: return false;
    }
}

cudaError_t launch_block_sparse(int N, const BlockArgs<double> &a, const std::vector<unsigned char> &consts,
                                dim3 grid, dim3 block, size_t smem, cudaStream_t st) {
    switch (N) {
    case 2: return launch_sparse_one<2>(a, consts, grid, block, smem, st);
    case 3: return launch_sparse_one<3>(a, consts, grid, block, smem, st);
    case 4: return launch_sparse_one<4>(a, consts, grid, block, smem, st);
    case 5: return launch_sparse_one<5>(a, consts, grid, block, smem, st);
    case 6: return launch_sparse_one<6>(a, consts, grid, block, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

size_t sparse_smem_bytes(int N, int threads, int nnz, int nrowptr) {
    switch (N) {
    case 2: return SharedSparseCell<2>::smem_bytes(threads, nnz, nrowptr);
    case 3: return SharedSparseCell<3>::smem_bytes(threads, nnz, nrowptr);
    case 4: return SharedSparseCell<4>::smem_bytes(threads, nnz, nrowptr);
    case 5: return SharedSparseCell<5>::smem_bytes(threads, nnz, nrowptr);
    case 6: return SharedSparseCell<6>::smem_bytes(threads, nnz, nrowptr);
    default: return 0;
    }
}

}  // namespace mln
