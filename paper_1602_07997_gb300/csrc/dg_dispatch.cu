// Kernel variant tables and launch of the persistent fused step kernel.
#include <map>
#include <mutex>

#include "dg_kernels.cuh"

namespace dgk {

const KernelCfg* kernel_variants_acoustic(int N, int* count);
const KernelCfg* kernel_variants_elastic(int N, int* count);
const KernelCfg* kernel_variants_tc(int model, int N, int nsplit, int* count);

const KernelCfg* kernel_variants(int model, int N, int* count, int precision) {
  int c = 0;
  const KernelCfg* v = nullptr;
  if (precision == 0)
    v = model == 0 ? kernel_variants_acoustic(N, &c) : kernel_variants_elastic(N, &c);
  else if (precision == 1 || precision == 2)
    v = kernel_variants_tc(model, N, precision + 1, &c);
  if (count) *count = v ? c : 0;
  return v;
}

const KernelCfg* kernel_cfg(int model, int N) { return kernel_variants(model, N, nullptr); }

namespace {
std::mutex g_mu;
std::map<std::pair<int, const void*>, int> g_cap;  // (device, kernel) -> max resident CTAs

// Opt the kernel into its dynamic shared memory and read its occupancy (once per device).
cudaError_t prepare_fn(const KernelCfg* c, const void* fn, int* grid_cap) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mu);
  auto key = std::make_pair(dev, fn);
  auto it = g_cap.find(key);
  if (it != g_cap.end()) {
    *grid_cap = it->second;
    return cudaSuccess;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(c->smem));
  if (e != cudaSuccess) return e;
  int n = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, c->NT, c->smem);
  if (e != cudaSuccess) return e;
  const int cap = sms * (n > 0 ? n : 1);
  g_cap[key] = cap;
  *grid_cap = cap;
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_step(const KernelCfg* c, const StepArgs& args, cudaStream_t stream) {
  if (!c) return cudaErrorInvalidValue;
  if (c->split == 1 && (!args.xg || !args.ops2)) return cudaErrorInvalidValue;
  if (c->split == 2 && (!args.xg || !args.opstc)) return cudaErrorInvalidValue;
  int cap = 0;
  cudaError_t e = prepare_fn(c, reinterpret_cast<const void*>(c->fn), &cap);
  if (e != cudaSuccess) return e;
  const int nblk = (args.K + c->EB - 1) / c->EB;
  if (nblk == 0) return cudaSuccess;
  const int grid = nblk < cap ? nblk : cap;
  StepArgs a = args;
  void* params[] = {&a};
  e = cudaLaunchKernel(reinterpret_cast<const void*>(c->fn), dim3(grid), dim3(c->NT), params, c->smem, stream);
  if (e != cudaSuccess || !c->split) return e;
  // the GEMM kernel: column tiles of gemm_ne elements x row tiles of gemm_mt
  KernelCfg g = *c;
  g.NT = c->gemm_threads;
  g.smem = c->smem_gemm;
  int gcap = 0;
  e = prepare_fn(&g, reinterpret_cast<const void*>(c->fn_gemm), &gcap);
  if (e != cudaSuccess) return e;
  const unsigned tiles = unsigned(c->gemm_mtiles) * unsigned((args.K + c->gemm_ne - 1) / c->gemm_ne);
  const unsigned ggrid = c->gemm_persistent && tiles > unsigned(gcap) ? unsigned(gcap) : tiles;
  return cudaLaunchKernel(reinterpret_cast<const void*>(c->fn_gemm), dim3(ggrid), dim3(c->gemm_threads), params,
                          c->smem_gemm, stream);
}

// Non-finite = exponent bits all ones (NaN or +-Inf).  Grid-stride float4
// loads (q is 256-byte aligned), then one vote per CTA.
__device__ __forceinline__ bool nonfinite(float x) { return (__float_as_uint(x) & 0x7f800000u) == 0x7f800000u; }

__global__ void __launch_bounds__(256) finite_kernel(const float* __restrict__ q, long long n, int* err) {
  bool bad = false;
  const long long n4 = n >> 2, stride = (long long)gridDim.x * 256;
  const float4* q4 = reinterpret_cast<const float4*>(q);
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n4; i += stride) {
    const float4 v = __ldg(q4 + i);
    bad |= nonfinite(v.x) | nonfinite(v.y) | nonfinite(v.z) | nonfinite(v.w);
  }
  for (long long i = 4 * n4 + (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += stride) bad |= nonfinite(q[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, 2);
}

cudaError_t launch_finite_check(const float* q, long long n, int* err, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = ((n >> 2) + 255) / 256;
  const int grid = int(blocks < 1 ? 1 : (blocks > 152 * 8 ? 152 * 8 : blocks));
  finite_kernel<<<grid, 256, 0, stream>>>(q, n, err);
  return cudaGetLastError();
}

// one warp per (receiver, field): lanes over the nodes, then a warp sum
__global__ void sample_kernel(const float* __restrict__ q, const int* __restrict__ elem,
                              const float* __restrict__ vec, int nrec, int Nf, int Np, float* __restrict__ out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= nrec * Nf) return;
  const int r = w / Nf, f = w - r * Nf;
  const float* qk = q + (size_t(elem[r]) * Nf + f) * Np;
  const float* l = vec + size_t(r) * Np;
  float acc = 0.f;
  for (int i = lane; i < Np; i += 32) acc = fmaf(l[i], qk[i], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[w] = acc;
}

cudaError_t launch_sample(const float* q, const int* elem, const float* vec, int nrec, int Nf, int Np, float* out,
                          cudaStream_t stream) {
  if (nrec <= 0) return cudaSuccess;
  const int warps = nrec * Nf;
  sample_kernel<<<(warps * 32 + 255) / 256, 256, 0, stream>>>(q, elem, vec, nrec, Nf, Np, out);
  return cudaGetLastError();
}

// Thread i owns field-node i of every source element, so sources that share
// an element add up in order without races.
__device__ __forceinline__ void add_xsrc(const XSrc& xs, long long m, int NfNp, int mode, float dta1, float* qn,
                                         float* r, float* rout) {
  for (int i = threadIdx.x; i < NfNp; i += blockDim.x)
    for (int s = 0; s < xs.n; ++s) {
      const float am = (m >= 0 && m < xs.namp) ? xs.amp[size_t(s) * xs.namp + m] : 0.f;
      const float v = am * xs.vec[size_t(s) * NfNp + i];
      const size_t idx = size_t(xs.elem[s]) * NfNp + i;
      if (mode == 0) {
        r[idx] += v;
        qn[idx] = fmaf(dta1, v, qn[idx]);
      } else {
        rout[idx] += v;
      }
    }
}

__global__ void __launch_bounds__(256) xsrc_kernel(const XSrc xs, long long m, int NfNp, int mode, float dta1,
                                                   float* qn, float* r, float* rout) {
  add_xsrc(xs, m, NfNp, mode, dta1, qn, r, rout);
}

// one CTA per solve of the batch, with the buffers and step of its step kernel
__global__ void __launch_bounds__(256) xsrc_batched_kernel(const BatchArgs b, int NfNp) {
  const SolveDev& d = b.solves[blockIdx.x];
  if (d.xs.n == 0 || d.steps_left <= 0) return;
  StepArgs a;
  solve_args(b, d, a);
  add_xsrc(d.xs, d.step, NfNp, 0, a.dt * a.a1, a.qn, a.r2, nullptr);
}

cudaError_t prepare_step(const KernelCfg* c) {
  if (!c) return cudaErrorInvalidValue;
  int cap = 0;
  cudaError_t e = prepare_fn(c, reinterpret_cast<const void*>(c->fn), &cap);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(xsrc_kernel));
}

cudaError_t launch_xsrc(const XSrc& xs, long long step, int NfNp, const StepArgs& a, cudaStream_t stream) {
  if (xs.n <= 0) return cudaSuccess;
  xsrc_kernel<<<1, 256, 0, stream>>>(xs, step, NfNp, a.mode, a.dt * a.a1, a.qn, a.r2, a.rout);
  return cudaGetLastError();
}

cudaError_t launch_xsrc_batched(const BatchArgs& b, int NfNp, cudaStream_t stream) {
  if (b.nsolves <= 0) return cudaSuccess;
  xsrc_batched_kernel<<<b.nsolves, 256, 0, stream>>>(b, NfNp);
  return cudaGetLastError();
}

__global__ void advance_kernel(SolveDev* s, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || s[i].steps_left <= 0) return;
  s[i].step += 1;
  s[i].have = s[i].have < 2 ? s[i].have + 1 : 2;
  s[i].qcur ^= 1;
  s[i].r1slot ^= 1;  // r^m was written into the r^{m-2} slot
  s[i].steps_left -= 1;
}

cudaError_t launch_step_batched(const KernelCfg* c, const BatchArgs& args, cudaStream_t stream) {
  if (!c || !c->fn_batched) return cudaErrorInvalidValue;
  if (c->split && (!c->fn_gemm_batched || (args.total_blocks > 0 && (!args.ops2 || !args.tile_solve))))
    return cudaErrorInvalidValue;
  int cap = 0;
  cudaError_t e = prepare_fn(c, reinterpret_cast<const void*>(c->fn_batched), &cap);
  if (e != cudaSuccess) return e;
  int gcap = 0;
  if (c->split) {
    KernelCfg g = *c;
    g.NT = c->gemm_threads;
    g.smem = c->smem_gemm;
    e = prepare_fn(&g, reinterpret_cast<const void*>(c->fn_gemm_batched), &gcap);
    if (e != cudaSuccess) return e;
  }
  if (args.total_blocks == 0) return cudaSuccess;
  const int grid = args.total_blocks < cap ? args.total_blocks : cap;
  BatchArgs a = args;
  void* params[] = {&a};
  e = cudaLaunchKernel(reinterpret_cast<const void*>(c->fn_batched), dim3(grid), dim3(c->NT), params, c->smem,
                       stream);
  if (e != cudaSuccess || !c->split || args.total_tiles == 0) return e;
  const unsigned tiles = unsigned(args.total_tiles);
  const unsigned ggrid = c->gemm_persistent && tiles > unsigned(gcap) ? unsigned(gcap) : tiles;
  return cudaLaunchKernel(reinterpret_cast<const void*>(c->fn_gemm_batched), dim3(ggrid), dim3(c->gemm_threads),
                          params, c->smem_gemm, stream);
}

cudaError_t launch_advance(SolveDev* solves, int nsolves, cudaStream_t stream) {
  if (nsolves <= 0) return cudaSuccess;
  advance_kernel<<<(nsolves + 127) / 128, 128, 0, stream>>>(solves, nsolves);
  return cudaGetLastError();
}

}  // namespace dgk
