// Fused step with one element per thread (acoustic N = 1, 2; elastic N = 1).
//
// At low degree an element is a few dozen values and the operator products
// are tiny (Np x Np, Np x 4 Nfp), so the staged block kernel spends its time
// moving those values between phases through shared memory.  Here each
// thread owns one element from its staged fields to its RHS: the operators
// (D_r, D_s, D_t and LIFT, the same FP32 blob as the block kernel's) live
// in constant memory and the face loops are unrolled, so every operator
// product is a chain of FMAs with constant operands on values held in
// registers (Section 3.2: volume term, then the lifted penalty terms of
// Section 2.1, with the two acoustic surface streams: the pressure penalty
// and psi, the magnitude of the velocity penalty psi n_f).
//
// Per block of EB elements (one per thread), persistent CTAs:
//   - q, element records and neighbour words arrive by 1-D TMA bulk copies
//     into one of two stages (mbarrier, bounded waits), the next block's
//     stage issued at the top of this one;
//   - the traces of neighbours outside the block were gathered during the
//     previous block by 4-byte cp.async into two trace slots per element
//     (element-fastest, already in the element's own face-node order); a
//     third or fourth outside face of an element reads its neighbour from
//     global memory directly;
//   - each thread computes its element's RHS in registers and stores it in
//     shared memory; a flat, coalesced float4 pass then applies the AB3
//     update (Eq. updateScheme) with r^{m-1}, r^{m-2} read from global
//     memory (prefetched into L2 at the top of the block).
#include <mutex>
#include <set>

#include "dg_ept.cuh"

namespace dgk {

__constant__ float c_ops1[Sz<1>::KD * Sz<1>::Mpad];
__constant__ float c_ops2[Sz<2>::KD * Sz<2>::Mpad];

template <int N>
__device__ __forceinline__ float opc(int idx) {
  if constexpr (N == 1) return c_ops1[idx];
  else return c_ops2[idx];
}

template <int MODEL, int N, int EB>
struct EptPlan {
  using S = Sz<N>;
  static constexpr int Nf = MODEL == 0 ? 4 : 9, Np = S::Np, Nfp = S::Nfp, NFN = S::NFN, REC = Rec<MODEL>::size;
  static constexpr int QS = Nf * Np;   // floats per element
  // element stride in shared memory: + 4 words when QS is a multiple of 8,
  // so that the float4 rows of 8 consecutive elements fall in 8 different
  // 4-bank groups (per-thread row reads and writes without conflicts)
  static constexpr int QSP = QS % 8 == 0 ? QS + 4 : QS;
  static constexpr int SLOTS = 2;      // gathered neighbour traces per element
  static constexpr int EBP = EB + 1;   // element-fastest row stride of the trace slots
  static constexpr int nStage = round4(EB * QSP + EB * REC) + EB * 4;
  static constexpr int sQ = 0, sRec = EB * QSP, sNbr = round4(EB * QSP + EB * REC);
  static constexpr int oStage0 = 0, oStage1 = nStage;
  static constexpr int oRhs = 2 * nStage;                        // [EB][QSP]
  static constexpr int oT = oRhs + EB * QSP;                     // [SLOTS][Nf][Nfp][EBP]
  static constexpr int oFtab = round4(oT + SLOTS * Nf * Nfp * EBP);  // int [10][Nfp]
  static constexpr int oPtab = oFtab + 10 * Nfp;                 // int [24][Nfp]
  static constexpr int oBar = round4(oPtab + 24 * Nfp);
  static constexpr int nFloats = oBar + 4;                       // 2 mbarriers
  static constexpr size_t bytes = size_t(nFloats) * 4;
  static_assert(EB % 32 == 0, "whole warps, one element per thread");
  static_assert((QS * 4) % 16 == 0, "16-byte bulk copies of the fields");
};

// Body shared by one solve per launch and by a batch of solves (served
// mode): the provider maps a global block to its solve's arguments and local
// block, as for the block kernel.
template <int MODEL, int N, int EB, class Prov>
__device__ __forceinline__ void ept_body(const Prov& prov) {
  using P = EptPlan<MODEL, N, EB>;
  constexpr int Nf = P::Nf, Np = P::Np, Nfp = P::Nfp, QS = P::QS, QSP = P::QSP, REC = P::REC;
  constexpr int Mpad = Sz<N>::Mpad, EBP = P::EBP, SLOTS = P::SLOTS;
  constexpr int NT = EB;
  constexpr auto FN = FaceNodes<N>::tab;

  extern __shared__ __align__(16) float smem[];
  float* sRhs = smem + P::oRhs;
  float* sT = smem + P::oT;
  int* sFtab = reinterpret_cast<int*>(smem + P::oFtab);
  int* sPtab = reinterpret_cast<int*>(smem + P::oPtab);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P::oBar);

  const int tid = threadIdx.x;
  const int nblk = prov.nblocks();
  const int G = gridDim.x;
  const long long lim = prov.limit();
  int* const err = prov.err();
  const int mode = prov.mode();
  constexpr uint32_t kQBytes = uint32_t(EB * QS * 4);
  constexpr uint32_t kStageBytes = kQBytes + uint32_t(EB * REC * 4) + uint32_t(EB * 16);

  // stage copies in flight (bit s, parity in ppar), for the drain after an
  // expired wait; the gathers are cp.async groups, drained per thread
  uint32_t pmask = 0, ppar = 0;
  auto pend_set = [&](int i, uint32_t par) {
    pmask |= 1u << i;
    ppar = (ppar & ~(1u << i)) | (par << i);
  };
  auto pend_clr = [&](int i) { pmask &= ~(1u << i); };
  auto drain = [&]() {
#pragma unroll
    for (int i = 0; i < 2; ++i)
      if (pmask & (1u << i)) mbar_wait_bounded(&bars[i], (ppar >> i) & 1u, nullptr);
    cp_async_wait_all();
  };
  auto stage = [&](int s) { return smem + (s ? P::oStage1 : P::oStage0); };
  // (warp 0) the stage of block b: one bulk copy per element's fields (padded
  // rows), the records and the neighbour words; lane 0 registers the bytes
  // before any lane issues a copy
  auto issue_stage = [&](const StepArgs& a, int lb, int s) {
    float* st = stage(s);
    const int k0 = lb * EB;
    if (tid == 0) mbar_arrive_expect_tx(&bars[s], kStageBytes);
    __syncwarp();
    for (int e = tid; e < EB; e += 32)
      tma_bulk_g2s(st + P::sQ + e * QSP, a.q + size_t(k0 + e) * QS, uint32_t(QS * 4), &bars[s]);
    if (tid == 0) {
      tma_bulk_g2s(st + P::sRec, a.rec + size_t(k0) * REC, uint32_t(EB * REC * 4), &bars[s]);
      tma_bulk_g2s(st + P::sNbr, a.nbr + k0, uint32_t(EB * 16), &bars[s]);
    }
  };
  // traces of the outside neighbours of block b (stage s): thread e fetches
  // its own element's, face by face, into the element's slots
  auto issue_gathers = [&](const StepArgs& a, int lb, int s) {
    const int k0 = lb * EB;
    const int e = tid;
    const int4 nb = reinterpret_cast<const int4*>(stage(s) + P::sNbr)[e];
    int slot = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int w = nbr_word(nb, f);
      if (w < 0) continue;
      const int kn = w >> kNbrShift;
      const int le = kn - k0;
      if (le >= 0 && le < EB) continue;
      if (slot < SLOTS) {
        const int* pt = sPtab + ((w & 3) * 6 + ((w >> 2) & 7)) * Nfp;
        const float* src = a.q + size_t(kn) * QS;
        float* dst = sT + slot * Nf * Nfp * EBP + e;
#pragma unroll
        for (int m = 0; m < Nfp; ++m) {
          const int nP = pt[m];
#pragma unroll
          for (int c = 0; c < Nf; ++c) cp_async4(dst + (c * Nfp + m) * EBP, src + c * Np + nP);
        }
      }
      ++slot;
    }
    cp_async_commit();
  };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  // arguments of the block being processed and of the next one
  StepArgs nxt_a;
  int nxt_lb = 0;
  if ((int)blockIdx.x < nblk) prov.get(blockIdx.x, nxt_a, nxt_lb);
  if (tid < 32 && (int)blockIdx.x < nblk) issue_stage(nxt_a, nxt_lb, 0);
  if ((int)blockIdx.x < nblk) pend_set(0, 0u);
  for (int i = tid; i < 10 * Nfp; i += NT) sFtab[i] = prov.ftab()[i];
  __syncthreads();
  for (int i = tid; i < 24 * Nfp; i += NT) {
    const int m = i % Nfp, fr = i / Nfp;
    sPtab[i] = sFtab[(fr / 6) * Nfp + sFtab[4 * Nfp + (fr % 6) * Nfp + m]];
  }
  if ((int)blockIdx.x < nblk) {
    if (!__syncthreads_and(mbar_wait_bounded(&bars[0], 0u, err, lim))) {
      drain();
      return;
    }
    pend_clr(0);
    issue_gathers(nxt_a, nxt_lb, 0);
  }

  int it = 0;
  for (int b = blockIdx.x; b < nblk; b += G, ++it) {
    const int s = it & 1;
    const StepArgs a = nxt_a;
    const int k0 = nxt_lb * EB;
    if (b + G < nblk) prov.get(b + G, nxt_a, nxt_lb);
    bool ok = mbar_wait_bounded(&bars[s], uint32_t((it >> 1) & 1), err, lim);
    cp_async_wait_all();  // this block's gathered traces
    if (!__syncthreads_and(ok)) {
      drain();
      return;
    }
    pend_clr(s);
    const uint32_t pnext = uint32_t(((it + 1) >> 1) & 1);
    if (tid < 32 && b + G < nblk) issue_stage(nxt_a, nxt_lb, s ^ 1);
    if (tid == 0) {
      if (mode == 0) {
        // this block's AB3 history into L2 for the update pass
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.r1 + size_t(k0) * QS), "r"(kQBytes)
                     : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.r2 + size_t(k0) * QS), "r"(kQBytes)
                     : "memory");
      }
    }
    if (b + G < nblk) pend_set(s ^ 1, pnext);
    const float* sQ = stage(s) + P::sQ;
    const float* sRec = stage(s) + P::sRec;
    const int4* sNbr = reinterpret_cast<const int4*>(stage(s) + P::sNbr);

    // -------- the RHS of element k0 + tid, in registers
    const int e = tid, k = k0 + e;
    if (k < a.K) {
      const float* qe = sQ + e * QSP;
      const float* gk = sRec + e * REC;
      float g[9];
#pragma unroll
      for (int x = 0; x < 9; ++x) g[x] = gk[x];
      float qv[QS];
#pragma unroll
      for (int x = 0; x < QS / 4; ++x) {
        const float4 t = reinterpret_cast<const float4*>(qe)[x];
        qv[4 * x] = t.x;
        qv[4 * x + 1] = t.y;
        qv[4 * x + 2] = t.z;
        qv[4 * x + 3] = t.w;
      }
      const int4 nb = sNbr[e];
      // where the neighbour's traces across face f are read: the outer
      // boundary reads the element's own trace (its ghost state follows from
      // it); a neighbour in this block its staged fields through the
      // face-node permutation; a gathered one its slot (already in this
      // face's node order); a third or fourth outside face global memory
      struct Src {
        bool bnd, glob;
        const float* base;  // field 0 of the traces (shared memory)
        int cs;             // stride between fields
        const int* pt;      // neighbour volume node of each face node (in-block, global)
        const float* gq;    // the neighbour's fields in global memory
        bool inblk;
      };
      auto face_src = [&](int f) {
        const int w = nbr_word(nb, f);
        Src S;
        S.bnd = w < 0;
        const int kn = S.bnd ? 0 : (w >> kNbrShift);
        const int le = kn - k0;
        S.inblk = !S.bnd && le >= 0 && le < EB;
        const int slot = (S.bnd || S.inblk) ? 0 : outside_rank(nb, f, k0, EB);
        S.glob = !S.bnd && !S.inblk && slot >= SLOTS;
        S.pt = sPtab + (S.bnd ? 0 : ((w & 3) * 6 + ((w >> 2) & 7)) * Nfp);
        S.base = S.bnd ? qe : S.inblk ? sQ + le * QSP : sT + slot * Nf * Nfp * EBP + e;
        S.cs = (S.bnd || S.inblk) ? Np : Nfp * EBP;
        S.gq = a.q + size_t(kn) * QS;
        return S;
      };
      // the Nf neighbour values at face node m (own node nM)
      auto nbr_trace = [&](const Src& S, int m, int nM, float* qP) {
        if (!S.glob) {
          const int idx = S.bnd ? nM : S.inblk ? S.pt[m] : m * EBP;
#pragma unroll
          for (int c = 0; c < Nf; ++c) qP[c] = S.base[idx + c * S.cs];
        } else {
          const int nP = S.pt[m];
#pragma unroll
          for (int c = 0; c < Nf; ++c) qP[c] = __ldg(S.gq + c * Np + nP);
        }
      };
      float r[QS];
      if constexpr (MODEL == 0) {
        const float kap = gk[9], rinv = gk[10], ZM = gk[11];
        const float* p = qv;
        const float* v0 = qv + Np;
        const float* v1 = qv + 2 * Np;
        const float* v2 = qv + 3 * Np;
        float R[Np], rv[3][Np];
#pragma unroll
        for (int i = 0; i < Np; ++i) {
          R[i] = 0.f;
          rv[0][i] = rv[1][i] = rv[2][i] = 0.f;
        }
        // volume term: R = sum_d D_d w_d with w_d = -kappa sum_c g_cd v_c; the
        // pressure gradient G_d = D_d p joins r_v,c = -(1/rho) sum_d g_cd G_d
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          float wd[Np];
#pragma unroll
          for (int j = 0; j < Np; ++j) wd[j] = -kap * (g[d] * v0[j] + g[3 + d] * v1[j] + g[6 + d] * v2[j]);
          float Gd[Np];
#pragma unroll
          for (int i = 0; i < Np; ++i) {
            float accR = R[i], accG = 0.f;
#pragma unroll
            for (int j = 0; j < Np; ++j) {
              const float Dij = opc<N>((d * Np + j) * Mpad + i);
              accR = fmaf(Dij, wd[j], accR);
              accG = fmaf(Dij, p[j], accG);
            }
            R[i] = accR;
            Gd[i] = accG;
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float sc = -rinv * g[3 * c + d];
#pragma unroll
            for (int i = 0; i < Np; ++i) rv[c][i] = fmaf(sc, Gd[i], rv[c][i]);
          }
        }
        // surface term, face by face: penalties pen_p = A jp + B jvn and
        // psi = C jp + D jvn (jp = [[p]]/2, jvn = [[v]].n/2, Fscale folded in),
        // R += LIFT_f pen_p, r_v += n_f LIFT_f psi; the rigid wall mirrors the
        // own trace (p+ = p-, v+ = v- - 2 (v-.n) n)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float4 fn = face_normal(g, f);
          const float fs = fn.w, zP = gk[12 + f];
          float A, B, C, D;
          if (a.flux == 0) {
            const float kc = 2.f / (ZM + zP);
            A = fs * kap * kc;
            B = -A * zP;
            C = -fs * (ZM * rinv) * kc;
            D = -C * zP;
          } else {
            A = 0.f;
            B = -fs * kap;
            C = -fs * rinv;
            D = 0.f;
          }
          const Src S = face_src(f);
          const float mir = S.bnd ? 2.f : 0.f;
          float L[Np];
#pragma unroll
          for (int i = 0; i < Np; ++i) L[i] = 0.f;
#pragma unroll
          for (int m = 0; m < Nfp; ++m) {
            const int nM = FN.v[f][m];
            const float pM = p[nM], vM0 = v0[nM], vM1 = v1[nM], vM2 = v2[nM];
            float qP[Nf];
            nbr_trace(S, m, nM, qP);
            const float vn = mir * (qP[1] * fn.x + qP[2] * fn.y + qP[3] * fn.z);
            const float vP0 = qP[1] - vn * fn.x, vP1 = qP[2] - vn * fn.y, vP2 = qP[3] - vn * fn.z;
            const float jp = 0.5f * (qP[0] - pM);
            const float jvn = 0.5f * ((vP0 - vM0) * fn.x + (vP1 - vM1) * fn.y + (vP2 - vM2) * fn.z);
            const float pp = A * jp + B * jvn, ps = C * jp + D * jvn;
#pragma unroll
            for (int i = 0; i < Np; ++i) {
              const float l = opc<N>((3 * Np + f * Nfp + m) * Mpad + i);
              R[i] = fmaf(l, pp, R[i]);
              L[i] = fmaf(l, ps, L[i]);
            }
          }
#pragma unroll
          for (int i = 0; i < Np; ++i) {
            rv[0][i] = fmaf(fn.x, L[i], rv[0][i]);
            rv[1][i] = fmaf(fn.y, L[i], rv[1][i]);
            rv[2][i] = fmaf(fn.z, L[i], rv[2][i]);
          }
        }
#pragma unroll
        for (int i = 0; i < Np; ++i) {
          r[i] = R[i];
          r[Np + i] = rv[0][i];
          r[2 * Np + i] = rv[1][i];
          r[3 * Np + i] = rv[2][i];
        }
      } else {
        // volume term (elastic): U_cd = D_d v_c and Rv_c = sum_d D_d s_cd with
        // s_cd = (1/rho) sum_m g_md sigma_cm; then the stress part lambda
        // (div v) I + mu (grad v + grad v^T) with grad v from U and g
        const float lam = gk[9], mu = gk[10], rinv = gk[11];
        float U[3][3][Np], Rv[3][Np];
#pragma unroll
        for (int i = 0; i < Np; ++i)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            Rv[c][i] = 0.f;
            U[c][0][i] = U[c][1][i] = U[c][2][i] = 0.f;
          }
#pragma unroll
        for (int j = 0; j < Np; ++j) {
          float sg[3][3];
          sg[0][0] = qv[3 * Np + j];
          sg[1][1] = qv[4 * Np + j];
          sg[2][2] = qv[5 * Np + j];
          sg[0][1] = sg[1][0] = qv[6 * Np + j];
          sg[0][2] = sg[2][0] = qv[7 * Np + j];
          sg[1][2] = sg[2][1] = qv[8 * Np + j];
          float sv[3][3];
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) sv[c][d] = rinv * (g[d] * sg[c][0] + g[3 + d] * sg[c][1] + g[6 + d] * sg[c][2]);
#pragma unroll
          for (int i = 0; i < Np; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const float Dij = opc<N>((d * Np + j) * Mpad + i);
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                U[c][d][i] = fmaf(Dij, qv[c * Np + j], U[c][d][i]);
                Rv[c][i] = fmaf(Dij, sv[c][d], Rv[c][i]);
              }
            }
        }
#pragma unroll
        for (int i = 0; i < Np; ++i) {
          float gv[3][3];  // gv[c][x] = d v_c / d x_x = sum_d g[x][d] U[c][d]
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int x = 0; x < 3; ++x) gv[c][x] = g[3 * x] * U[c][0][i] + g[3 * x + 1] * U[c][1][i] + g[3 * x + 2] * U[c][2][i];
          const float div = gv[0][0] + gv[1][1] + gv[2][2];
          r[i] = Rv[0][i];
          r[Np + i] = Rv[1][i];
          r[2 * Np + i] = Rv[2][i];
          r[3 * Np + i] = lam * div + 2.f * mu * gv[0][0];
          r[4 * Np + i] = lam * div + 2.f * mu * gv[1][1];
          r[5 * Np + i] = lam * div + 2.f * mu * gv[2][2];
          r[6 * Np + i] = mu * (gv[0][1] + gv[1][0]);
          r[7 * Np + i] = mu * (gv[0][2] + gv[2][0]);
          r[8 * Np + i] = mu * (gv[1][2] + gv[2][1]);
        }
        // surface term: the nine penalty terms of Section 2.1 at every face
        // node (face_penalty: upwind or centred flux, mirror ghosts on the
        // outer boundary), lifted onto every field
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float4 fn = face_normal(g, f);
          const Src S = face_src(f);
#pragma unroll
          for (int m = 0; m < Nfp; ++m) {
            const int nM = FN.v[f][m];
            float qM[Nf], qP[Nf], pen[Nf];
#pragma unroll
            for (int c = 0; c < Nf; ++c) qM[c] = qv[c * Np + nM];
            nbr_trace(S, m, nM, qP);
            face_penalty<1>(gk, f, S.bnd, qM, qP, fn, a.flux, a.bc, pen);
#pragma unroll
            for (int i = 0; i < Np; ++i) {
              const float l = opc<N>((3 * Np + f * Nfp + m) * Mpad + i);
#pragma unroll
              for (int c = 0; c < Nf; ++c) r[c * Np + i] = fmaf(l, pen[c], r[c * Np + i]);
            }
          }
        }
      }
      if (k == a.src_elem && a.srcvec) {
#pragma unroll
        for (int x = 0; x < QS; ++x) r[x] = fmaf(a.src_amp, __ldg(a.srcvec + x), r[x]);
      }
      if (mode == 0) {
        float4* dst = reinterpret_cast<float4*>(sRhs + e * QSP);
#pragma unroll
        for (int x = 0; x < QS / 4; ++x) dst[x] = make_float4(r[4 * x], r[4 * x + 1], r[4 * x + 2], r[4 * x + 3]);
      } else {  // RHS only: the caller's buffer (4-byte alignment is all it promises)
        float* dst = a.rout + size_t(k) * QS;
#pragma unroll
        for (int x = 0; x < QS; ++x) dst[x] = r[x];
      }
    }
    __syncthreads();  // every RHS of the block is in sRhs

    // -------- AB3 update, a flat float4 pass over the block's elements
    if (mode == 0) {
      const int ne = a.K - k0 < EB ? a.K - k0 : EB;
      const int n4 = ne * QS / 4;
      const size_t g0 = size_t(k0) * QS / 4;
      const float4* gr1 = reinterpret_cast<const float4*>(a.r1) + g0;
      float4* gr2 = reinterpret_cast<float4*>(a.r2) + g0;
      float4* gqn = reinterpret_cast<float4*>(a.qn) + g0;
      const float a1 = a.a1, a2 = a.a2, a3 = a.a3, dt = a.dt;
      constexpr int UB = 4;
      for (int i0 = tid; i0 < n4; i0 += NT * UB) {
        float4 p1[UB], p2[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int i = i0 + u * NT;
          if (i < n4) {
            p1[u] = __ldg(gr1 + i);
            p2[u] = gr2[i];
          }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int i = i0 + u * NT;
          if (i < n4) {
            const int el = i / (QS / 4), o4 = i - el * (QS / 4);  // element, float4 within it
            const float4 q4 = reinterpret_cast<const float4*>(sQ + el * QSP)[o4];
            const float4 r4 = reinterpret_cast<const float4*>(sRhs + el * QSP)[o4];
            gqn[i] = make_float4(fmaf(dt, a1 * r4.x + a2 * p1[u].x + a3 * p2[u].x, q4.x),
                                 fmaf(dt, a1 * r4.y + a2 * p1[u].y + a3 * p2[u].y, q4.y),
                                 fmaf(dt, a1 * r4.z + a2 * p1[u].z + a3 * p2[u].z, q4.z),
                                 fmaf(dt, a1 * r4.w + a2 * p1[u].w + a3 * p2[u].w, q4.w));
            gr2[i] = r4;
          }
        }
      }
    }
    // the next block's stage was issued at the top: once it has landed,
    // gather its outside traces (the trace slots were last read above)
    {
      const bool okn = b + G < nblk ? mbar_wait_bounded(&bars[s ^ 1], pnext, err, lim) : true;
      if (!__syncthreads_and(okn)) {
        drain();
        return;
      }
    }
    if (b + G < nblk) {
      pend_clr(s ^ 1);
      issue_gathers(nxt_a, nxt_lb, s ^ 1);
    }
  }
}

// one solve per launch (dg_step / dg_rhs)
template <int MODEL, int N, int EB>
__global__ void __launch_bounds__(EB) dg_ept_kernel(const StepArgs a) {
  SingleSolve p{a, EB};
  ept_body<MODEL, N, EB>(p);
}

// every solve of a batch (same model and N) in one persistent launch (served mode)
template <int MODEL, int N, int EB>
__global__ void __launch_bounds__(EB) dg_ept_batched_kernel(const BatchArgs b) {
  SolveBatch p{b};
  ept_body<MODEL, N, EB>(p);
}

template <int MODEL, int N, int EB>
KernelCfg make_ept_cfg() {
  using P = EptPlan<MODEL, N, EB>;
  static_assert(P::bytes <= 227 * 1024, "shared memory budget");
  KernelCfg c{};
  c.EB = EB;
  c.TN = 1;
  c.NT = EB;
  c.ops_smem = false;
  c.r_smem = false;
  c.smem = P::bytes;
  c.fn = dg_ept_kernel<MODEL, N, EB>;
  c.fn_batched = dg_ept_batched_kernel<MODEL, N, EB>;
  c.split = 0;
  c.fn_gemm = nullptr;
  c.fn_gemm_batched = nullptr;
  c.smem_gemm = 0;
  c.gemm_threads = c.gemm_ne = c.gemm_mt = c.gemm_mtiles = c.gemm_kx = c.gemm_mp2 = c.gemm_nsplit = 0;
  c.gemm_xtile = 0;
  c.gemm_persistent = false;
  return c;
}

KernelCfg ept_variant(int model, int N, int which) {
  if (model == 1) return which == 0 ? make_ept_cfg<1, 1, 32>() : make_ept_cfg<1, 1, 64>();
  if (N == 1)
    return which == 0 ? make_ept_cfg<0, 1, 64>() : which == 1 ? make_ept_cfg<0, 1, 128>() : make_ept_cfg<0, 1, 32>();
  return which == 0 ? make_ept_cfg<0, 2, 32>() : make_ept_cfg<0, 2, 64>();
}

cudaError_t ept_upload_ops(int N, const float* ops, size_t n) {
  if (N < 1 || N > 2) return cudaSuccess;
  static std::mutex mu;
  static std::set<int> done;  // devices whose operators are in place, per N (device * 8 + N)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(dev * 8 + N)) return cudaSuccess;
  const size_t cap = N == 1 ? sizeof(c_ops1) : sizeof(c_ops2);
  if (n * sizeof(float) != cap) return cudaErrorInvalidValue;
  e = N == 1 ? cudaMemcpyToSymbol(c_ops1, ops, cap) : cudaMemcpyToSymbol(c_ops2, ops, cap);
  if (e == cudaSuccess) done.insert(dev * 8 + N);
  return e;
}

}  // namespace dgk
