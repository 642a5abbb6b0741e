// Right-hand side to host memory without any device allocation.
//
// dg_rhs(h, r_out, on_device = 0) stages the RHS in a device buffer it
// allocates for the call.  dg_rhs_host_noalloc stages it instead in a
// file-scope device array of fixed size, so that callers who must not
// allocate device memory at call time can still read the RHS into host
// memory.  Everything that could allocate is done once per handle by
// dg_setup (Handle::noalloc_prepare, with the handle's device current):
// the lookup of the array's device address, which loads this file's module
// and with it the array on that device, and the first-use set-up of the
// kernels the call launches.
#include <cuda_runtime.h>

#include "dg_args.h"
#include "dg_handle.h"

namespace {

// 4 Mi floats (16 MiB) on every device where a handle has been set up, held
// until the process exits.
constexpr size_t kNoAllocMaxFloats = size_t(1) << 22;
static __device__ __align__(256) float g_rhs_scratch[kNoAllocMaxFloats];

}  // namespace

namespace dg {

int Handle::noalloc_prepare() {
  noalloc_scratch = nullptr;
  noalloc_cfg = nullptr;
  if (size_t(K) * Nf * Np > kNoAllocMaxFloats) return DG_OK;  // the call will refuse this mesh
  // the fused FP32 variant: the handle's own if it is one, else the process's
  // FP32 choice for (model, N) if that is fused, else the first fused variant
  // compiled for N (a split variant would need its input buffer, which is
  // allocated on first use)
  const dgk::KernelCfg* c = nullptr;
  if (opts.strategy == DG_STRATEGY_FUSED && opts.precision == DG_FP32 && !cfg->split) {
    c = cfg;
  } else {
    c = select_variant(model, N, 0, device, DG_FP32);
    if (c && c->split) {
      int n = 0;
      const dgk::KernelCfg* v = dgk::kernel_variants(model, N, &n, 0);
      c = nullptr;
      for (int i = 0; i < n && !c; ++i)
        if (!v[i].split) c = &v[i];
    }
  }
  if (!c) return fail(DG_EINVAL, "no fused FP32 variant for this degree");
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(allocation-free RHS scratch)");
  e = dgk::prepare_step(c);
  if (e != cudaSuccess) return cuda_fail(e, "set-up of the allocation-free RHS kernel");
  noalloc_scratch = static_cast<float*>(p);
  noalloc_cfg = c;
  return DG_OK;
}

}  // namespace dg

extern "C" int dg_rhs_host_noalloc(dg_handle* h, float* r_out) {
  if (!h || !r_out) return dg::fail(DG_EINVAL, "NULL handle or output");
  const size_t n = size_t(h->K) * h->Nf * h->Np;
  if (n > kNoAllocMaxFloats || !h->noalloc_scratch)
    return dg::fail(DG_EINVAL, "K*Nf*Np = " + std::to_string(n) + " exceeds the allocation-free scratch of " +
                                   std::to_string(kNoAllocMaxFloats) + " floats; use dg_rhs");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dg::cuda_fail(e, "cudaGetDevice");
  if (dev != h->device) return dg::fail(DG_EINVAL, "the handle's device must be current");
  // the RHS kernel writes every value that is read back: nothing to clear
  dgk::StepArgs a = h->args(1);
  a.rout = h->noalloc_scratch;
  e = dgk::launch_step(h->noalloc_cfg, a, h->stream);
  if (e != cudaSuccess) return dg::cuda_fail(e, "launch");
  e = dgk::launch_xsrc(h->xs, h->step, h->Nf * h->Np, a, h->stream);  // sources beyond the first
  if (e != cudaSuccess) return dg::cuda_fail(e, "launch");
  e = cudaMemcpyAsync(r_out, h->noalloc_scratch, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return dg::cuda_fail(e, "copy to host");
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return dg::cuda_fail(e, "synchronize");
  return DG_OK;
}
