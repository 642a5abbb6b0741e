// The paper's comparison strategies (Section 3) on this library's data: the
// library route (cuBLAS strided-batched SGEMMs for the operator products) and
// the plain multi-kernel route (volume, surface and update kernels).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "dg_args.h"

namespace dgk {

// Front half of the library route for (model, N): the fused kernel's stages
// 1-3 writing X[tile][row][NE] (FP32); gemm_ne / gemm_kx / gemm_mp2 /
// gemm_xtile describe X and the row-padded operator blob.
const KernelCfg* front_cfg(int model, int N);
// Number of library-route GEMM products of the model (acoustic 8, elastic 24).
int library_products(int model);
// The operator products of every column tile: cuBLAS strided-batched SGEMMs
// on the handle's stream (cublas: a cublasHandle_t) into
// Y[product][K padded to tiles][Np], product stride yprod floats.  Returns
// the first non-zero cublasStatus_t, or 0.
int library_gemms(void* cublas, int model, int N, const StepArgs& a, float* Y, size_t yprod);
// Geometric combination, source and AB3 update (a.mode 0) or RHS (mode 1)
// from the products.
cudaError_t launch_library_epilogue(int model, int N, const StepArgs& a, const float* Y, size_t yprod,
                                    cudaStream_t s);
// Volume, surface and (a.mode 0) update kernels of the plain route; R0 is a
// state-sized device buffer for the partial RHS.
cudaError_t launch_plain_step(int model, int N, const StepArgs& a, float* R0, cudaStream_t s);

}  // namespace dgk
