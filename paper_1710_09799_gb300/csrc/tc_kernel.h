// Host interface of the tensor-core cell model (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "kernels.cuh"
#include "setup.h"

namespace mln {

// N values with a tensor-core kernel.
bool tc_supported(int N);
// Rows (cells incl. halo) of one tile: the MMA M.
int tc_rows();
// Dynamic shared memory of one CTA.
int tc_smem_bytes(int N);
// B-operand image (uploaded to the device once) and the scalar constants.
bool pack_tc(const Setup &s, double dt, std::vector<unsigned char> &img, std::vector<unsigned char> &scal);
// One launch of a.nsteps steps; a.tile + 2 a.halo must equal tc_rows().
cudaError_t launch_tc(int N, const BlockArgs<float> &a, const std::vector<unsigned char> &scal, const void *bimg,
                      int sms, cudaStream_t st);
// C (128 x nc) = A (128 x kc) B (nc x kc)^T through the kernel's product
// path, with A staged in tensor memory (tmem_a) or in shared memory.
cudaError_t tc_product(int nc, int kc, bool tmem_a, const float *A, const double *B, float *C, std::string &err);
// Rotated basis (MLN_FORM_ROTATED) on tensor cores, kind::f16 with FP16
// hi/lo operands: constant-operand image and scalars, one launch, the
// diagnostic product (A scaled and split on the device, B's rows scaled by
// powers of two and split on the host; (nc, kc) = (48, 48), (32, 32), (16, 16)).
bool pack_tcr(const Setup &s, double dt, std::vector<unsigned char> &img, std::vector<unsigned char> &scal);
cudaError_t launch_tcr(int N, const BlockArgs<float> &a, const std::vector<unsigned char> &scal, const void *bimg,
                       int sms, cudaStream_t st);
cudaError_t tcr_product(int nc, int kc, const float *A, const double *B, float *C, std::string &err);
int tcr_smem_bytes(int N);
// The product kernel with its MMA left out: the bounded completion wait runs
// out; err is set when it did.
cudaError_t tc_wait_selftest(std::string &err);

}  // namespace mln
