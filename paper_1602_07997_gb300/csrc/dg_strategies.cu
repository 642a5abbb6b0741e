// The paper's comparison strategies (Section 3), on this library's data:
//
//   library route (Section 3.3, "SGEMM" strategy): the fused kernel's front
//     half writes the operator-product inputs X[tile][row][NE] (volume inputs,
//     surface streams, face normals); cuBLAS strided-batched SGEMMs over the column
//     tiles compute every operator product (D_r/D_s/D_t products and the LIFT
//     products, one GEMM per product and input block) into Y[product][K][Np];
//     a streaming kernel does the geometric combination, the source and the
//     AB3 update.  TF32 tensor-core math can be requested for the GEMMs.
//   plain multi-kernel route (Section 3.2, one node per thread): a volume
//     kernel (the D_r/D_s/D_t products and their geometric combination into a
//     partial RHS), a surface kernel (traces, numerical flux, LIFT added to
//     the partial RHS) and an AB3 update kernel, with the partial RHS in HBM
//     between them.
//
// Both exist to compare against the fused step; they follow the same
// formulas (see the fused kernel's header) in FP32.
#include <cublas_v2.h>

#include "dg_launch.cuh"
#include "dg_strategies.h"

namespace dgk {

// ---------------------------------------------------------------- library route
template <int MODEL, int N>
constexpr int front_eb() {
  return (MODEL == 1 && N >= 5) ? 4 : 8;
}

// The fused kernel's front half writing X in the FP32 GEMM layout (tiles of
// SplitShape::NE elements); split = 0 so that launch_step launches it alone.
template <int MODEL, int N>
KernelCfg make_front_cfg() {
  constexpr int EB = front_eb<MODEL, N>();
  constexpr int NT = threads_for<N, EB, 1>();
  using SS = SplitShape<MODEL, N>;
  static_assert(Plan<MODEL, N, EB, false, false, MODEL == 0, true>::bytes <= 227 * 1024, "shared memory budget");
  KernelCfg c{};
  c.EB = EB;
  c.TN = 1;
  c.NT = NT;
  c.smem = Plan<MODEL, N, EB, false, false, MODEL == 0, true>::bytes;
  c.fn = dg_step_kernel<MODEL, N, EB, 1, NT, false, false, SS::NE, 0>;
  c.split = 0;
  c.gemm_ne = SS::NE;
  c.gemm_kx = SS::KX;
  c.gemm_mp2 = SS::OPP;
  c.gemm_xtile = size_t(SS::KX) * SS::NE * 4;
  return c;
}

const KernelCfg* front_cfg(int model, int N) {
  static const KernelCfg ac[8] = {make_front_cfg<0, 1>(), make_front_cfg<0, 2>(), make_front_cfg<0, 3>(),
                                  make_front_cfg<0, 4>(), make_front_cfg<0, 5>(), make_front_cfg<0, 6>(),
                                  make_front_cfg<0, 7>(), make_front_cfg<0, 8>()};
  static const KernelCfg el[8] = {make_front_cfg<1, 1>(), make_front_cfg<1, 2>(), make_front_cfg<1, 3>(),
                                  make_front_cfg<1, 4>(), make_front_cfg<1, 5>(), make_front_cfg<1, 6>(),
                                  make_front_cfg<1, 7>(), make_front_cfg<1, 8>()};
  if (N < 1 || N > 8) return nullptr;
  return model == 0 ? &ac[N - 1] : &el[N - 1];
}

int library_products(int model) { return model == 0 ? 8 : 24; }

// One strided-batched GEMM per (product, input block): for every column tile t
//   Y_p[t NE + e][i] (+)= sum_r ops2[(arow + r) MP2 + i] X_t[brow + r][e],
// r < klen: column-major C = A op(B) with A = ops2 (lda = MP2), B = the
// tile's X rows read transposed (ldb = NE), C = Y_p (ldc = Np).
static cublasStatus_t gemm(cublasHandle_t h, int Np, int NE, int KX, int MP2, int ntiles, const float* ops2,
                           const float* X, float* Yp, int arow, int brow, int klen, float beta) {
  const float one = 1.0f;
  return cublasSgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_T, Np, NE, klen, &one, ops2 + size_t(arow) * MP2, MP2,
                                   0, X + size_t(brow) * NE, NE, static_cast<long long>(KX) * NE, &beta, Yp, Np,
                                   static_cast<long long>(NE) * Np, ntiles);
}

int library_gemms(void* cublas, int model, int N, const StepArgs& a, float* Y, size_t yprod) {
  cublasHandle_t h = static_cast<cublasHandle_t>(cublas);
  const KernelCfg* f = front_cfg(model, N);
  if (!f) return -1;
  const int Nfp = (N + 1) * (N + 2) / 2, Np = (N + 1) * (N + 2) * (N + 3) / 6, NFN = 4 * Nfp;
  const int NE = f->gemm_ne, KX = f->gemm_kx, MP2 = f->gemm_mp2;
  const int nt = (a.K + NE - 1) / NE;
  auto Yp = [&](int p) { return Y + size_t(p) * yprod; };
  cublasStatus_t s = CUBLAS_STATUS_SUCCESS;
  auto G = [&](int p, int arow, int brow, int klen, float beta) {
    if (s == CUBLAS_STATUS_SUCCESS) s = gemm(h, Np, NE, KX, MP2, nt, a.ops2, a.xg, Yp(p), arow, brow, klen, beta);
  };
  if (model == 0) {
    // X rows: p, w_0..2 (Np each), P_p, psi (4 Nfp each), face normals
    for (int d = 0; d < 3; ++d) G(d, d * Np, 0, Np, 0.f);              // G_d = D_d p
    G(3, 0, Np, 3 * Np + NFN, 0.f);                                    // R = [D_r D_s D_t LIFT] [w; P_p]
    for (int f = 0; f < 4; ++f)                                        // L_f = LIFT_f psi_f
      G(4 + f, 3 * Np + f * Nfp, 4 * Np + NFN + f * Nfp, Nfp, 0.f);
  } else {
    // X rows: v_0..2, s_cd (3 + 3c + d) (Np each), Fscale p_v,0..2 and
    // Fscale dv_0..2 (4 Nfp each), face normals
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) G(3 * c + d, d * Np, c * Np, Np, 0.f);  // U_cd = D_d v_c
    for (int c = 0; c < 3; ++c) {
      G(9 + c, 0, (3 + 3 * c) * Np, 3 * Np, 0.f);                          // sum_d D_d s_cd
      G(9 + c, 3 * Np, 12 * Np + c * NFN, NFN, 1.f);                       // + LIFT (Fscale p_v,c)
    }
    for (int f = 0; f < 4; ++f)                                            // W_f,c = LIFT_f (Fscale dv_c)
      for (int c = 0; c < 3; ++c)
        G(12 + 3 * f + c, 3 * Np + f * Nfp, 12 * Np + (3 + c) * NFN + f * Nfp, Nfp, 0.f);
  }
  return int(s);
}

// Geometric combination, source and AB3 update from the GEMM products, one
// thread per (element, node), nodes across lanes.
template <int MODEL, int N>
__global__ void __launch_bounds__(256) library_epilogue_kernel(const StepArgs a, const float* __restrict__ Y,
                                                                size_t yprod) {
  constexpr int Np = Sz<N>::Np, Nf = MODEL == 0 ? 4 : 9, REC = Rec<MODEL>::size;
  const size_t total = size_t(a.K) * Np;
  for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
    const int k = int(t / Np), i = int(t - size_t(k) * Np);
    const float* gk = a.rec + size_t(k) * REC;
    float g[9];
#pragma unroll
    for (int x = 0; x < 9; ++x) g[x] = __ldg(gk + x);
    auto y = [&](int p) { return __ldg(Y + size_t(p) * yprod + t); };
    float r[Nf];
    if constexpr (MODEL == 0) {
      // velocity lift sum_f n_f L_f, the normals from the X rows of element k
      using XR = XRows<MODEL, N>;
      constexpr int NE = SplitShape<MODEL, N>::NE;
      const float* nk = a.xg + (size_t(k / NE) * XR::KX + XR::KXM) * NE + k % NE;
      const float rinv = __ldg(gk + 10);
      const float G0 = y(0), G1 = y(1), G2 = y(2);
      r[0] = y(3);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float lv = 0.f;
#pragma unroll
        for (int f = 0; f < 4; ++f) lv = fmaf(__ldg(nk + (3 * f + c) * NE), y(4 + f), lv);
        r[1 + c] = lv - rinv * (g[3 * c] * G0 + g[3 * c + 1] * G1 + g[3 * c + 2] * G2);
      }
    } else {
      const float lam = __ldg(gk + 9), mu = __ldg(gk + 10);
      float U[9];
#pragma unroll
      for (int p = 0; p < 9; ++p) U[p] = y(p);
      float gv[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int x = 0; x < 3; ++x) gv[c][x] = g[3 * x] * U[3 * c] + g[3 * x + 1] * U[3 * c + 1] + g[3 * x + 2] * U[3 * c + 2];
      const float div = gv[0][0] + gv[1][1] + gv[2][2];
#pragma unroll
      for (int c = 0; c < 3; ++c) r[c] = y(9 + c);
      r[3] = lam * div + 2.f * mu * gv[0][0];
      r[4] = lam * div + 2.f * mu * gv[1][1];
      r[5] = lam * div + 2.f * mu * gv[2][2];
      r[6] = mu * (gv[0][1] + gv[1][0]);
      r[7] = mu * (gv[0][2] + gv[2][0]);
      r[8] = mu * (gv[1][2] + gv[2][1]);
      // stress LIFT: lambda (n_f.W_f) I + mu (n_f W_f^T + W_f n_f^T) per face
      using XR = XRows<MODEL, N>;
      constexpr int NE = SplitShape<MODEL, N>::NE;
      const float* nk = a.xg + (size_t(k / NE) * XR::KX + XR::KXM) * NE + k % NE;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const float nx = __ldg(nk + (3 * f) * NE), ny = __ldg(nk + (3 * f + 1) * NE);
        const float nz = __ldg(nk + (3 * f + 2) * NE);
        const float w0 = y(12 + 3 * f), w1 = y(13 + 3 * f), w2 = y(14 + 3 * f);
        const float lnw = lam * (nx * w0 + ny * w1 + nz * w2);
        r[3] += lnw + 2.f * mu * nx * w0;
        r[4] += lnw + 2.f * mu * ny * w1;
        r[5] += lnw + 2.f * mu * nz * w2;
        r[6] += mu * (nx * w1 + ny * w0);
        r[7] += mu * (nx * w2 + nz * w0);
        r[8] += mu * (ny * w2 + nz * w1);
      }
    }
    if (k == a.src_elem && a.srcvec) {
#pragma unroll
      for (int f = 0; f < Nf; ++f) r[f] = fmaf(a.src_amp, __ldg(a.srcvec + f * Np + i), r[f]);
    }
    const size_t base = size_t(k) * Nf * Np + i;
#pragma unroll
    for (int f = 0; f < Nf; ++f) {
      const size_t idx = base + size_t(f) * Np;
      if (a.mode == 0) {
        const float acc = a.a1 * r[f] + a.a2 * __ldg(a.r1 + idx) + a.a3 * a.r2[idx];
        a.qn[idx] = fmaf(a.dt, acc, __ldg(a.q + idx));
        a.r2[idx] = r[f];
      } else {
        a.rout[idx] = r[f];
      }
    }
  }
}

static int g_sms = 0;
static int sm_count() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

template <int MODEL, int N>
static cudaError_t epi_launch(const StepArgs& a, const float* Y, size_t yprod, cudaStream_t s) {
  const size_t total = size_t(a.K) * Sz<N>::Np;
  const size_t want = (total + 255) / 256;
  const unsigned grid = unsigned(want < size_t(8 * sm_count()) ? want : size_t(8 * sm_count()));
  if (grid == 0) return cudaSuccess;
  library_epilogue_kernel<MODEL, N><<<grid, 256, 0, s>>>(a, Y, yprod);
  return cudaGetLastError();
}

cudaError_t launch_library_epilogue(int model, int N, const StepArgs& a, const float* Y, size_t yprod,
                                    cudaStream_t s) {
#define DG_EPI(M, NN) \
  if (model == M && N == NN) return epi_launch<M, NN>(a, Y, yprod, s);
  DG_EPI(0, 1) DG_EPI(0, 2) DG_EPI(0, 3) DG_EPI(0, 4) DG_EPI(0, 5) DG_EPI(0, 6) DG_EPI(0, 7) DG_EPI(0, 8)
  DG_EPI(1, 1) DG_EPI(1, 2) DG_EPI(1, 3) DG_EPI(1, 4) DG_EPI(1, 5) DG_EPI(1, 6) DG_EPI(1, 7) DG_EPI(1, 8)
#undef DG_EPI
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- plain multi-kernel route
// EV elements per CTA, one thread per (element, node) or (element, face node).
template <int N>
constexpr int npt_ev() {
  return Sz<N>::Np >= 128 ? 1 : 128 / Sz<N>::Np;
}

// Volume kernel: partial RHS from the D_r/D_s/D_t products (no LIFT term):
//   acoustic r_p = sum_d D_d w_d, r_v_c = -(1/rho) sum_d g_cd D_d p
//   elastic  r_v_c = sum_d D_d s_cd, r_sig from dv_i/dx_j = sum_d g_jd D_d v_i
// The volume inputs (p, w_d / v_c, s_cd) of the CTA's elements go to shared
// memory first; each thread then walks its operator rows.
template <int MODEL, int N>
__global__ void npt_volume_kernel(const StepArgs a, float* __restrict__ R0) {
  constexpr int Np = Sz<N>::Np, Nf = MODEL == 0 ? 4 : 9, REC = Rec<MODEL>::size, EV = npt_ev<N>();
  constexpr int NV = MODEL == 0 ? 4 : 12;
  constexpr int Mpad = Sz<N>::Mpad;
  __shared__ float xin[EV][NV][Np];
  const int e = threadIdx.x / Np, i = threadIdx.x - e * Np;
  const int k = blockIdx.x * EV + e;
  const bool on = e < EV && k < a.K;
  if (on) {
    const float* gk = a.rec + size_t(k) * REC;
    const float* qk = a.q + size_t(k) * Nf * Np;
    if constexpr (MODEL == 0) {
      const float kap = __ldg(gk + 9);
      const float v0 = __ldg(qk + Np + i), v1 = __ldg(qk + 2 * Np + i), v2 = __ldg(qk + 3 * Np + i);
      xin[e][0][i] = __ldg(qk + i);
#pragma unroll
      for (int d = 0; d < 3; ++d)
        xin[e][1 + d][i] = -kap * (__ldg(gk + d) * v0 + __ldg(gk + 3 + d) * v1 + __ldg(gk + 6 + d) * v2);
    } else {
      const float rinv = __ldg(gk + 11);
      float sg[3][3];
      sg[0][0] = __ldg(qk + 3 * Np + i); sg[1][1] = __ldg(qk + 4 * Np + i); sg[2][2] = __ldg(qk + 5 * Np + i);
      sg[0][1] = sg[1][0] = __ldg(qk + 6 * Np + i);
      sg[0][2] = sg[2][0] = __ldg(qk + 7 * Np + i);
      sg[1][2] = sg[2][1] = __ldg(qk + 8 * Np + i);
#pragma unroll
      for (int c = 0; c < 3; ++c) xin[e][c][i] = __ldg(qk + c * Np + i);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d)
          xin[e][3 + 3 * c + d][i] =
              rinv * (__ldg(gk + d) * sg[c][0] + __ldg(gk + 3 + d) * sg[c][1] + __ldg(gk + 6 + d) * sg[c][2]);
    }
  }
  __syncthreads();
  if (!on) return;
  const float* gk = a.rec + size_t(k) * REC;
  float g[9];
#pragma unroll
  for (int x = 0; x < 9; ++x) g[x] = __ldg(gk + x);
  float* rk = R0 + size_t(k) * Nf * Np + i;
  if constexpr (MODEL == 0) {
    float G[3] = {0.f, 0.f, 0.f}, R = 0.f;
    for (int j = 0; j < Np; ++j) {
      const float d0 = __ldg(a.ops + size_t(0 * Np + j) * Mpad + i);
      const float d1 = __ldg(a.ops + size_t(1 * Np + j) * Mpad + i);
      const float d2 = __ldg(a.ops + size_t(2 * Np + j) * Mpad + i);
      const float p = xin[e][0][j];
      G[0] = fmaf(d0, p, G[0]);
      G[1] = fmaf(d1, p, G[1]);
      G[2] = fmaf(d2, p, G[2]);
      R = fmaf(d0, xin[e][1][j], R);
      R = fmaf(d1, xin[e][2][j], R);
      R = fmaf(d2, xin[e][3][j], R);
    }
    const float rinv = __ldg(gk + 10);
    rk[0] = R;
#pragma unroll
    for (int c = 0; c < 3; ++c) rk[(1 + c) * Np] = -rinv * (g[3 * c] * G[0] + g[3 * c + 1] * G[1] + g[3 * c + 2] * G[2]);
  } else {
    float U[9], Rv[3];
#pragma unroll
    for (int x = 0; x < 9; ++x) U[x] = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) Rv[c] = 0.f;
    for (int j = 0; j < Np; ++j) {
      float dd[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) dd[d] = __ldg(a.ops + size_t(d * Np + j) * Mpad + i);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v = xin[e][c][j];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          U[3 * c + d] = fmaf(dd[d], v, U[3 * c + d]);
          Rv[c] = fmaf(dd[d], xin[e][3 + 3 * c + d][j], Rv[c]);
        }
      }
    }
    const float lam = __ldg(gk + 9), mu = __ldg(gk + 10);
    float gv[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int x = 0; x < 3; ++x) gv[c][x] = g[3 * x] * U[3 * c] + g[3 * x + 1] * U[3 * c + 1] + g[3 * x + 2] * U[3 * c + 2];
    const float div = gv[0][0] + gv[1][1] + gv[2][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) rk[c * Np] = Rv[c];
    rk[3 * Np] = lam * div + 2.f * mu * gv[0][0];
    rk[4 * Np] = lam * div + 2.f * mu * gv[1][1];
    rk[5 * Np] = lam * div + 2.f * mu * gv[2][2];
    rk[6 * Np] = mu * (gv[0][1] + gv[1][0]);
    rk[7 * Np] = mu * (gv[0][2] + gv[2][0]);
    rk[8 * Np] = mu * (gv[1][2] + gv[2][1]);
  }
}

// Surface kernel: the penalty terms at the 4 Nfp face nodes of the CTA's
// elements (own trace through the face mask, neighbour trace through the
// neighbour's mask and face rotation, mirror ghost on the boundary) go to
// shared memory; then r = R0 + LIFT (Fscale penalty) (+ source) per node,
// into `out` (R0 itself for a step, the caller's RHS buffer otherwise).
template <int MODEL, int N>
__global__ void npt_surface_kernel(const StepArgs a, const float* R0, float* out) {
  constexpr int Np = Sz<N>::Np, Nfp = Sz<N>::Nfp, NFN = Sz<N>::NFN, Mpad = Sz<N>::Mpad;
  constexpr int Nf = MODEL == 0 ? 4 : 9, REC = Rec<MODEL>::size, EV = npt_ev<N>();
  constexpr int TPE = Np > NFN ? Np : NFN;  // threads per element
  __shared__ float pen[EV][Nf][NFN];
  const int e = threadIdx.x / TPE, t = threadIdx.x - e * TPE;
  const int k = blockIdx.x * EV + e;
  const bool on = e < EV && k < a.K;
  if (on && t < NFN) {
    const int f = t / Nfp, m = t - f * Nfp;
    const float* gM = a.rec + size_t(k) * REC;
    const int nM = __ldg(a.ftab + f * Nfp + m);
    const int4 nb = __ldg(a.nbr + k);
    const int w = (f == 0) ? nb.x : (f == 1) ? nb.y : (f == 2) ? nb.z : nb.w;
    const bool bnd = w < 0;
    float qM[Nf], qP[Nf];
    const float* qk = a.q + size_t(k) * Nf * Np;
#pragma unroll
    for (int c = 0; c < Nf; ++c) qM[c] = __ldg(qk + c * Np + nM);
    if (!bnd) {
      const int kn = w >> kNbrShift, rot = (w >> 2) & 7, f2 = w & 3;
      const int nP = __ldg(a.ftab + f2 * Nfp + __ldg(a.ftab + 4 * Nfp + rot * Nfp + m));
      const float* qn = a.q + size_t(kn) * Nf * Np;
#pragma unroll
      for (int c = 0; c < Nf; ++c) qP[c] = __ldg(qn + c * Np + nP);
    } else {
#pragma unroll
      for (int c = 0; c < Nf; ++c) qP[c] = 0.f;
    }
    float gl[REC];
#pragma unroll
    for (int x = 0; x < REC; ++x) gl[x] = __ldg(gM + x);
    float pv[Nf];
    face_penalty<MODEL>(gl, f, bnd, qM, qP, face_normal(gl, f), a.flux, a.bc, pv);
#pragma unroll
    for (int c = 0; c < Nf; ++c) pen[e][c][t] = pv[c];
  }
  __syncthreads();
  if (!on || t >= Np) return;
  const int i = t;
  float r[Nf];
  const size_t base = size_t(k) * Nf * Np + i;
#pragma unroll
  for (int c = 0; c < Nf; ++c) r[c] = R0[base + size_t(c) * Np];
  for (int fm = 0; fm < NFN; ++fm) {
    const float l = __ldg(a.ops + size_t(3 * Np + fm) * Mpad + i);
#pragma unroll
    for (int c = 0; c < Nf; ++c) r[c] = fmaf(l, pen[e][c][fm], r[c]);
  }
  if (k == a.src_elem && a.srcvec) {
#pragma unroll
    for (int c = 0; c < Nf; ++c) r[c] = fmaf(a.src_amp, __ldg(a.srcvec + c * Np + i), r[c]);
  }
#pragma unroll
  for (int c = 0; c < Nf; ++c) out[base + size_t(c) * Np] = r[c];
}

// AB3 update: q^{m+1} = q^m + dt (a1 r^m + a2 r^{m-1} + a3 r^{m-2}); r^m into the r^{m-2} slot.
__global__ void npt_update_kernel(const StepArgs a, const float* __restrict__ R, size_t n) {
  for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += size_t(gridDim.x) * blockDim.x) {
    const float rv = R[t];
    const float acc = a.a1 * rv + a.a2 * __ldg(a.r1 + t) + a.a3 * a.r2[t];
    a.qn[t] = fmaf(a.dt, acc, __ldg(a.q + t));
    a.r2[t] = rv;
  }
}

template <int MODEL, int N>
static cudaError_t npt_launch(const StepArgs& a, float* R0, cudaStream_t s) {
  constexpr int Np = Sz<N>::Np, NFN = Sz<N>::NFN, EV = npt_ev<N>(), Nf = MODEL == 0 ? 4 : 9;
  constexpr int TPE = Np > NFN ? Np : NFN;
  const unsigned grid = unsigned((a.K + EV - 1) / EV);
  if (grid == 0) return cudaSuccess;
  npt_volume_kernel<MODEL, N><<<grid, (EV * Np + 31) / 32 * 32, 0, s>>>(a, R0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float* out = a.mode == 0 ? R0 : a.rout;
  npt_surface_kernel<MODEL, N><<<grid, (EV * TPE + 31) / 32 * 32, 0, s>>>(a, R0, out);
  e = cudaGetLastError();
  if (e != cudaSuccess || a.mode != 0) return e;
  const size_t n = size_t(a.K) * Nf * Np;
  const size_t want = (n + 255) / 256;
  npt_update_kernel<<<unsigned(want < size_t(8 * sm_count()) ? want : size_t(8 * sm_count())), 256, 0, s>>>(a, R0, n);
  return cudaGetLastError();
}

cudaError_t launch_plain_step(int model, int N, const StepArgs& a, float* R0, cudaStream_t s) {
#define DG_NPT(M, NN) \
  if (model == M && N == NN) return npt_launch<M, NN>(a, R0, s);
  DG_NPT(0, 1) DG_NPT(0, 2) DG_NPT(0, 3) DG_NPT(0, 4) DG_NPT(0, 5) DG_NPT(0, 6) DG_NPT(0, 7) DG_NPT(0, 8)
  DG_NPT(1, 1) DG_NPT(1, 2) DG_NPT(1, 3) DG_NPT(1, 4) DG_NPT(1, 5) DG_NPT(1, 6) DG_NPT(1, 7) DG_NPT(1, 8)
#undef DG_NPT
  return cudaErrorInvalidValue;
}

}  // namespace dgk
