// Per-problem kernels compiled at run time (internal header).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "kernels.cuh"
#include "setup.h"

namespace mln {

// CUDA source of the merged-form step kernel of one context (constants inlined,
// exact zeros left out), kernel name mln_jit_step.
std::string jit_merged_source(const Setup &s, double dt, bool fp32);

// Whether NVRTC and the driver entry points could be loaded (reason if not).
bool jit_available(std::string *why);

// Compile (or reuse from the cache) a source for the current device.
cudaError_t jit_compile(const std::string &src, void **fn, std::string &log);

cudaError_t jit_launch(void *fn, const BlockArgs<double> &a, dim3 g, dim3 b, size_t smem, cudaStream_t st);
cudaError_t jit_launch(void *fn, const BlockArgs<float> &a, dim3 g, dim3 b, size_t smem, cudaStream_t st);

}  // namespace mln
