// Instantiation of the fused step kernels for double (N = 2..6, both forms).
#include "dispatch.cuh"

namespace mln {

bool pack_consts(const Setup &s, int form, double dt, double, std::vector<unsigned char> &out) {
    return pack_consts_t<double>(s, form, dt, out);
}

cudaError_t launch_block(int N, int form, const BlockArgs<double> &a, const std::vector<unsigned char> &consts,
                         dim3 grid, dim3 block, size_t smem, cudaStream_t st) {
    return launch_block_t<double>(N, form, a, consts, grid, block, smem, st);
}

cudaError_t launch_sin_cosm1(int precision, const double *x, int64_t n, double *s, double *c1, cudaStream_t st) {
    const unsigned grid = static_cast<unsigned>((n + 255) / 256);
    if (n <= 0) return cudaSuccess;
    if (precision == MLN_FP64) sin_cosm1_kernel<double><<<grid, 256, 0, st>>>(x, n, s, c1);
    else sin_cosm1_kernel<float><<<grid, 256, 0, st>>>(x, n, s, c1);
    return cudaGetLastError();
}

}  // namespace mln
