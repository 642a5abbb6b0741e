// Kernel table and launch of the fused step kernel.
#include <cstdio>
#include <mutex>

#include "dg_kernels.cuh"

namespace dgk {

const KernelCfg* kernel_cfg_acoustic(int N);
const KernelCfg* kernel_cfg_elastic(int N);

const KernelCfg* kernel_cfg(int model, int N) {
  return model == 0 ? kernel_cfg_acoustic(N) : kernel_cfg_elastic(N);
}

// Opt every instantiation into its dynamic shared-memory size once per device.
static cudaError_t prepare(const KernelCfg* c) {
  static std::mutex mu;
  static bool done[2][8][64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  // index by table position: find it
  for (int m = 0; m < 2; ++m)
    for (int n = 1; n <= 8; ++n)
      if (kernel_cfg(m, n) == c) {
        if (!done[m][n - 1][dev]) {
          e = cudaFuncSetAttribute(reinterpret_cast<const void*>(c->fn),
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(c->smem));
          if (e != cudaSuccess) return e;
          done[m][n - 1][dev] = true;
        }
        return cudaSuccess;
      }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step(int model, int N, const StepArgs& args, cudaStream_t stream) {
  const KernelCfg* c = kernel_cfg(model, N);
  if (!c) return cudaErrorInvalidValue;
  cudaError_t e = prepare(c);
  if (e != cudaSuccess) return e;
  const int nblk = (args.K + c->EB - 1) / c->EB;
  if (nblk == 0) return cudaSuccess;
  StepArgs a = args;
  void* params[] = {&a};
  return cudaLaunchKernel(reinterpret_cast<const void*>(c->fn), dim3(nblk), dim3(c->NT), params,
                          c->smem, stream);
}

}  // namespace dgk
