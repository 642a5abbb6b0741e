// Right-hand side to host memory without any device allocation.
//
// dg_rhs(h, r_out, on_device = 0) stages the RHS in a device buffer it
// allocates for the call.  dg_rhs_host_noalloc stages it instead in a
// file-scope device array of fixed size that is created when the library is
// loaded, so that callers who must not allocate device memory at call time
// can still read the RHS into host memory.
#include <cuda_runtime.h>

#include <mutex>

#include "dg_args.h"
#include "dg_handle.h"

namespace {

// 4 Mi floats (16 MiB) on every device that loads the library, held until exit.
constexpr size_t kNoAllocMaxFloats = size_t(1) << 22;
static __device__ __align__(256) float g_rhs_scratch[kNoAllocMaxFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per
// device; the device must be current).
int scratch_for_device(int dev, float** out) {
  if (dev < 0 || dev >= kMaxDevices) return dg::fail(DG_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_scratch);
    if (e != cudaSuccess) return dg::cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_scratch[dev] = static_cast<float*>(p);
  }
  *out = g_scratch[dev];
  return DG_OK;
}

}  // namespace

extern "C" int dg_rhs_host_noalloc(dg_handle* h, float* r_out) {
  if (!h || !r_out) return dg::fail(DG_EINVAL, "NULL handle or output");
  const size_t n = size_t(h->K) * h->Nf * h->Np;
  if (n > kNoAllocMaxFloats)
    return dg::fail(DG_EINVAL, "K*Nf*Np = " + std::to_string(n) + " exceeds the allocation-free scratch of " +
                                   std::to_string(kNoAllocMaxFloats) + " floats; use dg_rhs");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dg::cuda_fail(e, "cudaGetDevice");
  if (dev != h->device) return dg::fail(DG_EINVAL, "the handle's device must be current");
  float* scratch = nullptr;
  int rc = scratch_for_device(dev, &scratch);
  if (rc) return rc;
  // the RHS kernel writes every value that is read back: nothing to clear.
  // A fused FP32 variant is used (the handle's own if it is one): a split
  // variant would need its input buffer, which is allocated on first use.
  const dgk::KernelCfg* cfg = h->cfg;
  if (cfg->split || h->opts.strategy != DG_STRATEGY_FUSED) {
    int n = 0;
    const dgk::KernelCfg* v = dgk::kernel_variants(h->model, h->N, &n, 0);
    cfg = nullptr;
    for (int i = 0; i < n && !cfg; ++i)
      if (!v[i].split) cfg = &v[i];
    if (!cfg) return dg::fail(DG_EINVAL, "no fused variant for this degree");
  }
  dgk::StepArgs a = h->args(1);
  a.rout = scratch;
  e = dgk::launch_step(cfg, a, h->stream);
  if (e != cudaSuccess) return dg::cuda_fail(e, "launch");
  e = dgk::launch_xsrc(h->xs, h->step, h->Nf * h->Np, a, h->stream);  // sources beyond the first
  if (e != cudaSuccess) return dg::cuda_fail(e, "launch");
  e = cudaMemcpyAsync(r_out, scratch, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return dg::cuda_fail(e, "copy to host");
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return dg::cuda_fail(e, "synchronize");
  return DG_OK;
}
