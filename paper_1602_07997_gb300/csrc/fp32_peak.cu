// FP32 fused multiply-add throughput of the current device: the measured
// denominator of the ALU roofline of the high-degree steps.
//
// Every thread runs CH independent FMA chains x <- x a + b (a and b are
// kernel arguments, so nothing folds at compile time) for `iters` x 16
// rounds; the grid fills every SM to its occupancy limit.  Two instruction
// forms are timed: the scalar FP32 FMA and the packed two-lane form
// fma.rn.f32x2 (one instruction, two FP32 FMAs).  A flop is one add or one
// multiply, so one FMA counts 2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dg_internal.h"
#include "dg_handle.h"

namespace {

__device__ float g_peak_sink;  // written only when the chains reach an impossible value

constexpr int kChains = 8;   // independent chains per thread
constexpr int kUnroll = 16;  // rounds per loop iteration

__global__ void __launch_bounds__(256) ffma_scalar_kernel(int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * float(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.2345e30f) g_peak_sink = s;
}

// the same work with half the instructions: kChains / 2 register pairs
__global__ void __launch_bounds__(256) ffma_packed_kernel(int iters, float a, float b) {
  uint64_t x[kChains / 2], av, bv;
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) {
    const float x0 = 1e-3f * float(threadIdx.x + 2 * c), x1 = 1e-3f * float(threadIdx.x + 2 * c + 1);
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(x0), "f"(x1));
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains / 2; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) {
    float y0, y1;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(y0), "=f"(y1) : "l"(x[c]));
    s += y0 + y1;
  }
  if (s == -1.2345e30f) g_peak_sink = s;
}

// Best TFLOP/s of `reps` timed launches of kernel `fn` sized to about
// `target_ms` each (one untimed launch first sizes the loop).
int time_form(const void* fn, cudaStream_t st, int reps, double target_ms, double* tflops, double* ms) {
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, 0);
  if (e != cudaSuccess) return dg::cuda_fail(e, "fp32 peak: device query");
  const int grid = sms * std::max(occ, 1);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return dg::cuda_fail(e, "fp32 peak: events");
  }
  const float a = 0.9999999f, b = 1e-7f;
  int iters = 256;
  double best = 0.0, best_ms = 0.0;
  for (int r = -1; r < reps && e == cudaSuccess; ++r) {
    void* params[] = {&iters, (void*)&a, (void*)&b};
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = cudaLaunchKernel(fn, dim3(grid), dim3(256), params, 0, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) break;
    const double flop = 2.0 * double(grid) * 256.0 * double(iters) * kUnroll * kChains;
    if (r < 0) {  // sizing launch
      iters = int(std::min(4.0e6, std::max(256.0, iters * target_ms / std::max(1e-3, double(t)))));
      continue;
    }
    const double tf = flop / (double(t) * 1e-3) / 1e12;
    if (tf > best) {
      best = tf;
      best_ms = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return dg::cuda_fail(e, "fp32 peak: launch");
  *tflops = best;
  if (ms) *ms = best_ms;
  return DG_OK;
}

}  // namespace

extern "C" int dg_fp32_peak(void* stream, int reps, double target_ms, double* scalar_tflops,
                            double* packed_tflops, double* ms_per_launch) {
  if (reps < 1 || !(target_ms > 0.0) || target_ms > 10000.0)
    return dg::fail(DG_EINVAL, "dg_fp32_peak: reps >= 1 and 0 < target_ms <= 10000");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double s = 0.0, p = 0.0, ms_s = 0.0, ms_p = 0.0;
  int rc = time_form(reinterpret_cast<const void*>(ffma_scalar_kernel), st, reps, target_ms, &s, &ms_s);
  if (rc) return rc;
  rc = time_form(reinterpret_cast<const void*>(ffma_packed_kernel), st, reps, target_ms, &p, &ms_p);
  if (rc) return rc;
  if (scalar_tflops) *scalar_tflops = s;
  if (packed_tflops) *packed_tflops = p;
  if (ms_per_launch) *ms_per_launch = std::max(ms_s, ms_p);
  return DG_OK;
}
