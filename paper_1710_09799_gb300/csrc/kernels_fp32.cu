// Instantiation of the fused step kernels for float (N = 2..6, both forms).
#include "dispatch.cuh"

namespace mln {

bool pack_consts(const Setup &s, int form, double dt, float, std::vector<unsigned char> &out) {
    return pack_consts_t<float>(s, form, dt, out);
}

cudaError_t launch_block_trace(int N, const BlockArgs<float> &a, const std::vector<unsigned char> &consts,
                               dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool programmatic) {
    return launch_block_trace_t<float>(N, a, consts, grid, block, smem, st, programmatic);
}

cudaError_t launch_block(int N, int form, const BlockArgs<float> &a, const std::vector<unsigned char> &consts,
                         dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool programmatic) {
    return launch_block_t<float>(N, form, a, consts, grid, block, smem, st, programmatic);
}

}  // namespace mln
