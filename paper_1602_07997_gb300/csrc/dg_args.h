// Kernel argument block and launch table of the fused step kernel
// (plain C++; shared by the host library and the CUDA units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dgk {

// Element record, floats per element (odd length: element-strided reads of
// the records in shared memory are then free of bank conflicts):
//   acoustic (17): g[9] (row-major g[c][d] = dr_d/dx_c), kappa, 1/rho, Z,
//                  Z+ of the element across each face [4] (own Z on the boundary), pad
//   elastic  (25): g[9], lambda, mu, 1/rho, Zp, Zs, cp, cs,
//                  Zp+ per face [4], Zs+ per face [4], pad
template <int MODEL>
struct Rec {
  static constexpr int size = MODEL == 0 ? 17 : 25;
};
// Neighbour word per face: -1 on the outer boundary, otherwise
// (k' << 5) | (rotation << 2) | f' with k' the neighbour element, f' its
// face and rotation one of the 6 face-node permutations.
constexpr int kNbrShift = 5;

// Point sources of a solve beyond the first (which the step kernels add):
// source s adds amp[s][m] vec[s] to r^m of element elem[s] at step m.
struct XSrc {
  int n;                 // number of sources (0: none)
  int namp;              // amplitudes per source (zero past a source's own count)
  const int* elem;       // [n]
  const float* vec;      // [n][Nf Np]
  const float* amp;      // [n][namp]
};

struct StepArgs {
  const float* q;        // q^m   [Kpad][Nf][Np]
  float* qn;             // q^m+1 [Kpad][Nf][Np]            (mode 0)
  const float* r1;       // r^m-1                            (mode 0)
  float* r2;             // in r^m-2, out r^m                (mode 0)
  float* rout;           // r^m [K][Nf][Np]                  (mode 1)
  const float* rec;      // [Kpad][Rec::size]
  const int4* nbr;       // [Kpad] neighbour words
  const float* ops;      // [KD][Mpad]: rows d*Np+j -> D_d[i][j]; rows 3Np+c -> LIFT[i][c]
  const int* ftab;       // [4][Nfp] face masks, then [6][Nfp] rotations
  const float* srcvec;   // [Nf][Np] source shape or null
  float src_amp;
  int src_elem;          // element holding the source, -1 = none
  int K;
  int mode;              // 0 = AB3 step, 1 = RHS only
  int flux;              // 0 upwind, 1 centred
  int bc;                // acoustic: rigid; elastic: 0 free, 1 rigid
  float dt, a1, a2, a3;
  int* err;              // device error word (bounded-wait expiry)
  float* xg;             // split step: GEMM inputs X[tile][row][NE]
  const float* ops2;     // split step (FP32): operator blob [3Np + 4Nfp][rows padded to 32]
  const void* opstc;     // split step (tensor cores): BF16 operator pieces, core-matrix layout
  long long wait_limit;  // bounded device waits: cycles before giving up (0 = 2^31; < 0 = at once, a test hook)
};

// Per-solve device state of a batched launch (served mode).  The step index,
// AB3 start-up phase and buffer parities advance on the device (advance kernel).
struct SolveDev {
  float* q[2];           // ping-pong fields
  float* r[2];           // AB3 history slots
  const float* rec;
  const int4* nbr;
  const float* srcvec;   // [Nf][Np] or null
  const float* amp;      // source amplitude per step (device) or null
  long long step;        // time-step index m
  int namp;
  int src_elem;
  int K;
  int flux, bc;
  float dt;
  int have;              // stored RHS levels (0, 1, 2)
  int qcur;              // q[qcur] holds q^m
  int r1slot;            // r[r1slot] holds r^{m-1}
  int steps_left;        // the advance kernel stops moving a solve at 0
  float* xg;             // split step: the solve's GEMM input buffer
  XSrc xs;               // its point sources beyond the first
};

struct BatchArgs {
  SolveDev* solves;      // [nsolves]
  const int* block_start;  // [nsolves + 1] first global block of each solve
  const int* block_solve;  // [total_blocks] solve of each global block
  int nsolves;
  int total_blocks;
  const float* ops;      // operators of the batch's (model, N)
  const int* ftab;
  int* err;
  // split step: row-padded operators and the GEMM tiles of every solve
  const float* ops2;
  const int* tile_start;   // [nsolves + 1] first global tile of each solve
  const int* tile_solve;   // [total_tiles] solve of each global tile
  int total_tiles;
  long long wait_limit;    // as StepArgs::wait_limit
};

// Host-visible launch configuration of one (model, N) instantiation.  A
// split variant launches fn (front half, writes X) and then fn_gemm:
// split = 1 FP32 CUDA-core GEMM, split = 2 tensor-core GEMM in split-BF16
// arithmetic with gemm_nsplit pieces per operand.
struct KernelCfg {
  int EB, TN, NT;
  bool ops_smem, r_smem;
  size_t smem;
  void (*fn)(StepArgs);
  void (*fn_batched)(BatchArgs);
  int split;
  void (*fn_gemm)(StepArgs);
  void (*fn_gemm_batched)(BatchArgs);  // split step of a batch (FP32 GEMM only)
  size_t smem_gemm;
  int gemm_threads, gemm_ne, gemm_mt, gemm_mtiles, gemm_kx, gemm_mp2, gemm_nsplit;
  size_t gemm_xtile;     // bytes of X per column tile of gemm_ne elements
  bool gemm_persistent;  // grid = min(tiles, SMs x resident CTAs) instead of one CTA per tile
};

// Compiled variants of one (model, N): different elements per block (EB) and
// threads per CTA.  Variant 0 is the default.  precision: 0 FP32 (fused and
// FP32 split kernels), 1 bf16x3 and 2 bf16x6 tensor-core split kernels.
const KernelCfg* kernel_variants(int model, int N, int* count, int precision = 0);
const KernelCfg* kernel_cfg(int model, int N);

// Fused step with one element per thread (acoustic N = 1, 2; elastic N =
// 1): variant `which` (0, 1, 2 (acoustic N = 1 only): elements per CTA), and
// the upload of the operator blob ([3 Np + 4 Nfp][Mpad] as the block
// kernel's) to its constant memory on the current device (once per device
// and N).
KernelCfg ept_variant(int model, int N, int which);
cudaError_t ept_upload_ops(int N, const float* ops, size_t n);
// Opt the step kernel of `cfg` into its shared memory and read its occupancy
// on the current device, and load the small source kernel: everything
// launch_step (non-split cfg) and launch_xsrc set up on their first call.
cudaError_t prepare_step(const KernelCfg* cfg);
// Launch the persistent step kernel on `stream` (grid = min(blocks, SMs x occupancy)).
cudaError_t launch_step(const KernelCfg* cfg, const StepArgs& args, cudaStream_t stream);
// One batched step over every solve of `args` (same model and N); a split
// variant launches the batched front half and then the batched GEMM.
cudaError_t launch_step_batched(const KernelCfg* cfg, const BatchArgs& args, cudaStream_t stream);
// Advance the device-side step state of the solves (one thread per solve).
cudaError_t launch_advance(SolveDev* solves, int nsolves, cudaStream_t stream);
// Point sources beyond the first, after the step's kernels (same stream):
// mode 0 adds a v to r^m (a.r2) and dt a1 a v to q^{m+1} (a.qn) -- the AB3
// update is linear in r^m; mode 1 adds a v to a.rout (a = amp[s][m]).
cudaError_t launch_xsrc(const XSrc& xs, long long step, int NfNp, const StepArgs& a, cudaStream_t stream);
// The same for every solve of a batch with sources, before its advance.
cudaError_t launch_xsrc_batched(const BatchArgs& b, int NfNp, cudaStream_t stream);
// Finite-state check: sets bit 1 of *err if any of q[0..n) is NaN or +-Inf.
cudaError_t launch_finite_check(const float* q, long long n, int* err, cudaStream_t stream);
// Receiver sample: out[r][f] = sum_i vec[r][i] q[elem[r]][f][i].
cudaError_t launch_sample(const float* q, const int* elem, const float* vec, int nrec, int Nf, int Np, float* out,
                          cudaStream_t stream);

}  // namespace dgk
