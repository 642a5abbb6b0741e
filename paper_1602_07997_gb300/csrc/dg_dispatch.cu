// Kernel table and launch of the persistent fused step kernel.
#include <mutex>

#include "dg_kernels.cuh"

namespace dgk {

const KernelCfg* kernel_cfg_acoustic(int N);
const KernelCfg* kernel_cfg_elastic(int N);

const KernelCfg* kernel_cfg(int model, int N) {
  return model == 0 ? kernel_cfg_acoustic(N) : kernel_cfg_elastic(N);
}

namespace {
constexpr int kMaxDev = 64;
struct DevInfo {
  bool init = false;
  int sms = 0;
  int occ[2][8] = {};  // resident CTAs per SM for each instantiation
};
std::mutex g_mu;
DevInfo g_dev[kMaxDev];

// Opt the instantiation into its dynamic shared memory and read its occupancy.
cudaError_t prepare(int model, int N, const KernelCfg* c, int* grid_cap) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  DevInfo& d = g_dev[dev];
  if (!d.init) {
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    d.init = true;
  }
  int& occ = d.occ[model][N - 1];
  if (occ == 0) {
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(c->fn),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(c->smem));
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, reinterpret_cast<const void*>(c->fn), c->NT,
                                                      c->smem);
    if (e != cudaSuccess) return e;
    occ = n > 0 ? n : 1;
  }
  *grid_cap = d.sms * occ;
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_step(int model, int N, const StepArgs& args, cudaStream_t stream) {
  const KernelCfg* c = kernel_cfg(model, N);
  if (!c) return cudaErrorInvalidValue;
  int cap = 0;
  cudaError_t e = prepare(model, N, c, &cap);
  if (e != cudaSuccess) return e;
  const int nblk = (args.K + c->EB - 1) / c->EB;
  if (nblk == 0) return cudaSuccess;
  const int grid = nblk < cap ? nblk : cap;
  StepArgs a = args;
  void* params[] = {&a};
  return cudaLaunchKernel(reinterpret_cast<const void*>(c->fn), dim3(grid), dim3(c->NT), params, c->smem,
                          stream);
}

}  // namespace dgk
