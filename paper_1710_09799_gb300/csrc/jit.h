// Per-problem kernels compiled at run time (internal header).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "kernels.cuh"
#include "setup.h"

namespace mln {

// CUDA source of the merged-form step kernel of one context (constants inlined,
// exact zeros left out), kernel name mln_jit_step.
// rotated: the state is z = T^T y (MLN_FORM_ROTATED), else y (MLN_FORM_MERGED)
std::string jit_merged_source(const Setup &s, double dt, bool fp32, bool rotated = false, unsigned body_flags = 0u);
// The same step (merged or rotated form, FP64 context) in double-float
// arithmetic (MLN_KERNEL_DF32); kernel name mln_jit_step.
std::string jit_df_source(const Setup &s, double dt, unsigned body_flags = 0u, bool rotated = false);
// Threads per block that kernel is compiled for: 256 for the dense rotated
// form (D > 15: its pair vectors need up to 255 registers), else kMaxThreads.
int df_threads(int D, bool rotated);
// Whether every constant of that kernel is an FP32 pair without overflow and
// with a normal low word (zero, or 1e-30 < |v| < 1e37).
bool df_constants_in_range(const Setup &s, double dt, bool rotated = false);
// Flags of the fused step's block body (kBody* of kernels.cuh) for a problem:
// its boundary, whether it has a source; the compiled kernels never record.
unsigned jit_body_flags(const mln_params &p);

// Whether NVRTC and the driver entry points could be loaded (reason if not).
bool jit_available(std::string *why);

// Compile (or reuse from the cache) a source for the current device; the
// kernel is looked up by name.
cudaError_t jit_compile(const std::string &src, void **fn, std::string &log, const char *name = "mln_jit_step");

// Union sparsity pattern of the merged-form constants of the grids of a
// batch that have the same N: an entry is kept when it is non-zero (in the
// batch's precision) for at least one of them.
struct BatchPattern {
    int N = 0;
    std::vector<char> tt;  // 2q x D: T^T plane rows
    std::vector<char> t;   // D x 2q: T plane columns
    std::vector<char> wm;  // D
    std::vector<char> c1;  // D x D
    unsigned flags = ~0u;  // block-body flags that hold for every grid of the pattern
};
void batch_pattern_add(BatchPattern &pat, const Setup &s, const mln_params &p, bool fp32);
// Number of constants of one grid in the pattern's compacted order.
int batch_consts_count(const BatchPattern &pat);
// One grid's constants in that order (precision's reals, padded to 16 bytes).
// df: each constant as the (hi, lo) FP32 pair of double-float arithmetic (8 bytes).
void batch_pack(const BatchPattern &pat, const Setup &s, double dt, bool fp32, std::vector<unsigned char> &out,
                bool df = false);
// Source of the batched step kernel for the pattern's N (kernel mln_jit_batch):
// the products over the pattern's entries only, same order as the register
// model; each grid's constants are staged in shared memory and, when they
// fit, held in registers for the launch.
// df: the FP64 grids' step in double-float pairs (MLN_KERNEL_DF32), constants as pairs.
std::string jit_batch_source(const BatchPattern &pat, bool fp32, bool df = false);
cudaError_t jit_launch_batch(void *fn, const void *grids, const void *items, const void *consts, int parity,
                             int nsteps, int halo, int tile, int64_t step_offset, unsigned nblocks, unsigned threads,
                             size_t smem, cudaStream_t st);

// The persistent batch kernel of the same module (compiled as "mln_jit_batch_persist").
cudaError_t jit_launch_batch_persist(void *fn, const void *grids, const void *items, const void *consts, int halo,
                                     int tile, int64_t step_offset, const BatchPersist &p, unsigned nblocks,
                                     unsigned threads, size_t smem, cudaStream_t st);
cudaError_t jit_launch(void *fn, const BlockArgs<double> &a, dim3 g, dim3 b, size_t smem, cudaStream_t st);
cudaError_t jit_launch(void *fn, const BlockArgs<float> &a, dim3 g, dim3 b, size_t smem, cudaStream_t st);

}  // namespace mln
