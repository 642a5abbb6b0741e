// C ABI of libdg: set-up, state management and the time loop (see include/dg.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <fstream>
#include <sstream>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cublas_v2.h>
#include <cuda_runtime.h>

#include "dg_args.h"
#include "dg_strategies.h"
#include "dg_internal.h"
#include "dg_facemask.h"
#include "dg_handle.h"

namespace dg {

static thread_local std::string g_err;
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  return fail(DG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define DG_CUDA(call)                                  \
  do {                                                 \
    cudaError_t _e = (call);                           \
    if (_e != cudaSuccess) return dg::cuda_fail(_e, #call); \
  } while (0)

// Per-element material numbers (acoustic: kappa, 1/rho, Z; elastic: lambda,
// mu, 1/rho, Zp, Zs, cp, cs) and the impedances seen across each face.
static void materials(const double* coeffs, int model, int64_t k, double* m) {
  if (model == DG_ACOUSTIC) {
    double rho = coeffs[2 * k], c = coeffs[2 * k + 1];
    m[0] = rho * c * c;
    m[1] = 1.0 / rho;
    m[2] = rho * c;
  } else {
    double lam = coeffs[3 * k], mu = coeffs[3 * k + 1], rho = coeffs[3 * k + 2];
    double cp = std::sqrt((lam + 2 * mu) / rho), cs = std::sqrt(mu / rho);
    m[0] = lam;
    m[1] = mu;
    m[2] = 1.0 / rho;
    m[3] = rho * cp;
    m[4] = rho * cs;
    m[5] = cp;
    m[6] = cs;
  }
}

// Pack element records (layout of dgk::Rec) and neighbour words.
void pack_records(const HostMesh& hm, const double* coeffs, int model, int64_t Kpad, std::vector<float>& rec,
                  std::vector<int32_t>& nbr) {
  const int R = model == DG_ACOUSTIC ? dgk::Rec<0>::size : dgk::Rec<1>::size;
  rec.assign(size_t(Kpad) * R, 0.0f);
  nbr.assign(size_t(Kpad) * 4, -1);
  for (int64_t k = 0; k < Kpad; ++k) {
    float* o = &rec[size_t(k) * R];
    if (k >= hm.K) {  // padding element: identity geometry, unit medium
      o[0] = o[4] = o[8] = 1.0f;
      for (int i = 9; i < R; ++i) o[i] = 1.0f;
      continue;
    }
    for (int i = 0; i < 9; ++i) o[i] = float(hm.g[9 * k + i]);
    double m[7];
    materials(coeffs, model, k, m);
    const int nm = model == DG_ACOUSTIC ? 3 : 7;
    for (int i = 0; i < nm; ++i) o[9 + i] = float(m[i]);
    for (int f = 0; f < 4; ++f) {
      const int32_t kn = hm.nbr[4 * k + f];
      double mp[7];
      if (kn >= 0) materials(coeffs, model, kn, mp);
      else materials(coeffs, model, k, mp);
      if (model == DG_ACOUSTIC) {
        o[12 + f] = float(mp[2]);
      } else {
        o[16 + f] = float(mp[3]);
        o[20 + f] = float(mp[4]);
      }
      if (kn >= 0) {
        const uint32_t b = (hm.code[k] >> (8 * f)) & 0xffu;
        nbr[4 * k + f] = int32_t((uint32_t(kn) << dgk::kNbrShift) | (((b >> 2) & 7u) << 2) | (b & 3u));
      }
    }
  }
}

int check_coeffs(const double* coeffs, int64_t K, int model) {
  if (!coeffs) return fail(DG_EINVAL, "coefficients are NULL");
  const int nc = model == DG_ACOUSTIC ? 2 : 3;
  for (int64_t k = 0; k < K; ++k)
    for (int c = 0; c < nc; ++c) {
      double v = coeffs[nc * k + c];
      bool ok = std::isfinite(v) && (model == DG_ELASTIC && c == 0 ? v >= 0 : v > 0);
      if (!ok) return fail(DG_EINVAL, "non-physical coefficient at element " + std::to_string(k));
    }
  return DG_OK;
}

// Build operator blob [KD][Mpad] and face tables in kernel layout.
void pack_ops(const RefElement& R, std::vector<float>& ops, std::vector<int>& ftab) {
  const int Np = R.Np, Nfp = R.Nfp, Mpad = (Np + 3) & ~3, KD = 3 * Np + 4 * Nfp;
  ops.assign(size_t(KD) * Mpad, 0.0f);
  const std::vector<double>* D[3] = {&R.Dr, &R.Ds, &R.Dt};
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < Np; ++j)
      for (int i = 0; i < Np; ++i) ops[size_t(d * Np + j) * Mpad + i] = float((*D[d])[size_t(i) * Np + j]);
  for (int c = 0; c < 4 * Nfp; ++c)
    for (int i = 0; i < Np; ++i) ops[size_t(3 * Np + c) * Mpad + i] = float(R.LIFT[size_t(i) * 4 * Nfp + c]);
  ftab.assign(10 * Nfp, 0);
  for (int i = 0; i < 4 * Nfp; ++i) ftab[i] = R.fmask[i];
  for (int i = 0; i < 6 * Nfp; ++i) ftab[4 * Nfp + i] = R.perm[i];
}

double suggest_dt(const HostMesh& m, const double* coeffs, int N, int model, double cfl) {
  double best = 1e300;
  for (int64_t k = 0; k < m.K; ++k) {
    double cmax;
    if (model == DG_ACOUSTIC) cmax = coeffs[2 * k + 1];
    else cmax = std::sqrt((coeffs[3 * k] + 2 * coeffs[3 * k + 1]) / coeffs[3 * k + 2]);
    for (int f = 0; f < 4; ++f)
      best = std::min(best, 1.0 / (cmax * m.fscale[4 * k + f] * ((N + 1) * (N + 2) / 2.0 + 2.0)));
  }
  return cfl * best;
}

// ---------------------------------------------------------------- variants
// Autotuned choice per (device, model, N), shared by every handle of the process.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, int> g_tuned;

static int device_of_current() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return 0;
  return d;
}

const dgk::KernelCfg* select_variant(int model, int N, int block_elems, int device, int precision) {
  int n = 0;
  const dgk::KernelCfg* v = dgk::kernel_variants(model, N, &n, precision);
  if (!v) return nullptr;
  if (block_elems > 0) {
    for (int i = 0; i < n; ++i)
      if (v[i].EB == block_elems) return &v[i];
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(std::make_tuple(device, model, N, precision));
  return it != g_tuned.end() ? &v[it->second] : &v[0];
}

// ---------------------------------------------------------------- handle
int Handle::init(const dg_mesh* mesh, const double* coeffs_, int N_, int model_, const dg_opts* o) {
  if (model_ != DG_ACOUSTIC && model_ != DG_ELASTIC) return fail(DG_EINVAL, "unknown model");
  if (N_ < 1 || N_ > 8) return fail(DG_EINVAL, "polynomial degree N must be in 1..8");
  model = model_;
  N = N_;
  if (o) opts = *o;
  if (opts.flux != DG_FLUX_UPWIND && opts.flux != DG_FLUX_CENTERED) return fail(DG_EINVAL, "unknown flux");
  if (opts.bc < DG_BC_DEFAULT || opts.bc > DG_BC_FREE) return fail(DG_EINVAL, "unknown boundary condition");
  if (model == DG_ACOUSTIC && opts.bc == DG_BC_FREE)
    return fail(DG_EINVAL, "acoustic model supports rigid walls only");
  if (opts.strategy < DG_STRATEGY_FUSED || opts.strategy > DG_STRATEGY_PLAIN) return fail(DG_EINVAL, "unknown strategy");
  if (opts.strategy == DG_STRATEGY_FUSED && opts.precision != DG_FP32 && opts.precision != DG_BF16X3 &&
      opts.precision != DG_BF16X6)
    return fail(DG_EINVAL, "the fused strategy supports DG_FP32, DG_BF16X3 and DG_BF16X6");
  if (opts.strategy == DG_STRATEGY_LIBRARY && opts.precision != DG_FP32 && opts.precision != DG_TF32)
    return fail(DG_EINVAL, "the library strategy supports DG_FP32 and DG_TF32");
  if (opts.strategy == DG_STRATEGY_PLAIN && opts.precision != DG_FP32)
    return fail(DG_EINVAL, "the plain strategy supports DG_FP32");
  stream = static_cast<cudaStream_t>(opts.stream);
  int rc = ref.build(N);
  if (rc) return rc;
  rc = hm.build(mesh);
  if (rc) return rc;
  rc = check_coeffs(coeffs_, hm.K, model);
  if (rc) return rc;
  Np = ref.Np;
  Nfp = ref.Nfp;
  Nf = num_fields(model);
  K = hm.K;
  cfg = select_variant(model, N, opts.block_elems, device_of_current(),
                       opts.strategy == DG_STRATEGY_FUSED ? opts.precision : DG_FP32);
  if (!cfg) return fail(DG_EINVAL, "no compiled kernel variant with block_elems = " + std::to_string(opts.block_elems));
  // every launch reads whole blocks of EB <= 128 elements with bulk copies:
  // pad the element arrays so that the last block stays inside the allocation
  Kpad = (K + 3) / 4 * 4 + 128;
  coeffs.assign(coeffs_, coeffs_ + K * (model == DG_ACOUSTIC ? 2 : 3));
  verts.assign(mesh->verts, mesh->verts + 3 * mesh->nverts);
  tets.assign(mesh->tets, mesh->tets + 4 * mesh->ntets);
  DG_CUDA(cudaGetDevice(&device));

  if (K >= (int64_t(1) << (31 - dgk::kNbrShift))) return fail(DG_EINVAL, "too many elements for one handle");
  std::vector<float> geo, ops;
  std::vector<int> ftab;
  std::vector<int32_t> nbr;
  pack_records(hm, coeffs.data(), model, Kpad, geo, nbr);
  pack_ops(ref, ops, ftab);
  if ((model == DG_ACOUSTIC && N <= 2) || (model == DG_ELASTIC && N == 1)) {
    // the element-per-thread kernels unroll their face loops over the
    // compile-time face masks: they must be the tables built here
    for (int f = 0; f < 4; ++f)
      for (int m = 0; m < Nfp; ++m)
        if (dgk::face_node(N, f, m) != ref.fmask[f * Nfp + m])
          return fail(DG_EINVAL, "internal: compile-time face masks disagree with the reference element");
    DG_CUDA(dgk::ept_upload_ops(N, ops.data(), ops.size()));
  }

  const size_t nstate = size_t(Kpad) * Nf * Np;
  state_bytes = nstate * 4;
  auto rnd = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t need = 0;
  for (size_t b : {state_bytes, state_bytes, state_bytes, state_bytes, geo.size() * 4, nbr.size() * 4,
                   ops.size() * 4, ftab.size() * 4, size_t(Nf) * Np * 4, size_t(4)})
    need += rnd(b);
  DG_CUDA(cudaMalloc(&d_base, need));
  device_bytes = need;
  char* p = static_cast<char*>(d_base);
  auto take = [&](size_t bytes) {
    char* r = p;
    p += rnd(bytes);
    return r;
  };
  d_q[0] = reinterpret_cast<float*>(take(state_bytes));
  d_q[1] = reinterpret_cast<float*>(take(state_bytes));
  d_r[0] = reinterpret_cast<float*>(take(state_bytes));
  d_r[1] = reinterpret_cast<float*>(take(state_bytes));
  d_geo = reinterpret_cast<float*>(take(geo.size() * 4));
  d_nbr = reinterpret_cast<int32_t*>(take(nbr.size() * 4));
  d_ops = reinterpret_cast<float*>(take(ops.size() * 4));
  d_ftab = reinterpret_cast<int*>(take(ftab.size() * 4));
  d_src = reinterpret_cast<float*>(take(size_t(Nf) * Np * 4));
  d_err = reinterpret_cast<int*>(take(4));
  DG_CUDA(cudaMemsetAsync(d_base, 0, 4 * state_bytes, stream));
  DG_CUDA(cudaMemcpyAsync(d_geo, geo.data(), geo.size() * 4, cudaMemcpyHostToDevice, stream));
  DG_CUDA(cudaMemcpyAsync(d_nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice, stream));
  DG_CUDA(cudaMemcpyAsync(d_ops, ops.data(), ops.size() * 4, cudaMemcpyHostToDevice, stream));
  DG_CUDA(cudaMemcpyAsync(d_ftab, ftab.data(), ftab.size() * 4, cudaMemcpyHostToDevice, stream));
  DG_CUDA(cudaMemsetAsync(d_err, 0, 4, stream));
  DG_CUDA(cudaStreamSynchronize(stream));  // host vectors go out of scope
  qcur = 0;
  r1slot = 0;
  step = 0;
  have = 0;
  return noalloc_prepare();
}

Handle::~Handle() {
  if (d_base) cudaFree(d_base);
  if (d_split) cudaFree(d_split);
  if (d_tc) cudaFree(d_tc);
  if (d_lib) cudaFree(d_lib);
  if (d_r0) cudaFree(d_r0);
  if (d_recel) cudaFree(d_recel);
  if (d_traces) cudaFree(d_traces);
  if (d_xs) cudaFree(d_xs);
  if (cublas) cublasDestroy(static_cast<cublasHandle_t>(cublas));
}

// Buffers of the comparison strategies, on first use.
int Handle::ensure_strategy() {
  if (opts.strategy == DG_STRATEGY_PLAIN && !d_r0) {
    DG_CUDA(cudaMalloc(reinterpret_cast<void**>(&d_r0), state_bytes));
    split_bytes += state_bytes;
  }
  if (opts.strategy == DG_STRATEGY_LIBRARY && !d_lib) {
    const dgk::KernelCfg* f = dgk::front_cfg(model, N);
    if (!f) return fail(DG_EINVAL, "no library-route front half for this degree");
    const size_t nt = size_t((Kpad + f->gemm_ne - 1) / f->gemm_ne) + 1;
    const size_t xbytes = (nt * f->gemm_xtile + 255) & ~size_t(255);
    const int KD = 3 * Np + 4 * Nfp, MP2 = f->gemm_mp2;
    std::vector<float> ops2(size_t(KD) * MP2, 0.0f);
    const std::vector<double>* D[3] = {&ref.Dr, &ref.Ds, &ref.Dt};
    for (int d = 0; d < 3; ++d)
      for (int j = 0; j < Np; ++j)
        for (int i = 0; i < Np; ++i) ops2[size_t(d * Np + j) * MP2 + i] = float((*D[d])[size_t(i) * Np + j]);
    for (int cc = 0; cc < 4 * Nfp; ++cc)
      for (int i = 0; i < Np; ++i) ops2[size_t(3 * Np + cc) * MP2 + i] = float(ref.LIFT[size_t(i) * 4 * Nfp + cc]);
    const size_t obytes = (ops2.size() * 4 + 255) & ~size_t(255);
    libyprod = nt * size_t(f->gemm_ne) * Np;
    const size_t ybytes = size_t(dgk::library_products(model)) * libyprod * 4;
    DG_CUDA(cudaMalloc(&d_lib, xbytes + obytes + ybytes));
    split_bytes += xbytes + obytes + ybytes;
    d_libx = static_cast<float*>(d_lib);
    d_libops = reinterpret_cast<float*>(static_cast<char*>(d_lib) + xbytes);
    d_liby = reinterpret_cast<float*>(static_cast<char*>(d_lib) + xbytes + obytes);
    DG_CUDA(cudaMemsetAsync(d_libx, 0, xbytes, stream));
    DG_CUDA(cudaMemcpyAsync(d_libops, ops2.data(), ops2.size() * 4, cudaMemcpyHostToDevice, stream));
    DG_CUDA(cudaStreamSynchronize(stream));
    cublasHandle_t hb = nullptr;
    if (cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS) return fail(DG_ECUDA, "cublasCreate failed");
    cublas = hb;
    if (cublasSetMathMode(hb, opts.precision == DG_TF32 ? CUBLAS_TF32_TENSOR_OP_MATH : CUBLAS_DEFAULT_MATH) !=
        CUBLAS_STATUS_SUCCESS)
      return fail(DG_ECUDA, "cublasSetMathMode failed");
  }
  return DG_OK;
}

int Handle::launch(dgk::StepArgs a) {
  const int nx = xs.n > 0 ? 1 : 0;  // the kernel of the sources beyond the first
  if (opts.strategy == DG_STRATEGY_FUSED) {
    DG_CUDA(dgk::launch_step(cfg, a, stream));
    DG_CUDA(dgk::launch_xsrc(xs, step, Nf * Np, a, stream));
    launches += (cfg->split ? 2 : 1) + nx;
    return DG_OK;
  }
  int rc = ensure_strategy();
  if (rc) return rc;
  if (opts.strategy == DG_STRATEGY_PLAIN) {
    DG_CUDA(dgk::launch_plain_step(model, N, a, d_r0, stream));
    DG_CUDA(dgk::launch_xsrc(xs, step, Nf * Np, a, stream));
    launches += 3 + nx;
    return DG_OK;
  }
  // library route: front half, GEMMs, epilogue
  a.xg = d_libx;
  a.ops2 = d_libops;
  DG_CUDA(dgk::launch_step(dgk::front_cfg(model, N), a, stream));
  cublasHandle_t hb = static_cast<cublasHandle_t>(cublas);
  if (cublasSetStream(hb, stream) != CUBLAS_STATUS_SUCCESS) return fail(DG_ECUDA, "cublasSetStream failed");
  const int st = dgk::library_gemms(cublas, model, N, a, d_liby, libyprod);
  if (st != 0) return fail(DG_ECUDA, "cuBLAS SGEMM failed with status " + std::to_string(st));
  DG_CUDA(dgk::launch_library_epilogue(model, N, a, d_liby, libyprod, stream));
  DG_CUDA(dgk::launch_xsrc(xs, step, Nf * Np, a, stream));
  launches += 2 + nx;  // front half and epilogue (the cuBLAS GEMMs are not this library's kernels)
  return DG_OK;
}

// BF16 rounding (nearest, ties to even) of a finite float, as raw bits.
static uint16_t bf16_bits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return uint16_t(u >> 16);
}
static double bf16_value(uint16_t b) {
  const uint32_t u = uint32_t(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return double(f);
}

// Tensor-core split step: the front half's BF16 input pieces (one block per
// column tile of gemm_ne elements, one spare tile) and the operator pieces.
// For every 128-row tile of output nodes, chunk c of 16 input indices holds
// D_r, D_s, D_t (volume chunks) or LIFT (lift chunks), each as nsplit BF16
// pieces x = x_0 + x_1 (+ x_2) of the double-precision entry, every piece in
// the no-swizzle K-major core-matrix layout [16 row groups][2 K halves][8 rows][8].
static int pack_tc_ops(const RefElement& R, int nsplit, int mtiles, std::vector<uint16_t>& blob) {
  const int Np = R.Np, NFN = 4 * R.Nfp;
  const int NKD = (Np + 15) / 16, NKL = (NFN + 15) / 16;
  const size_t piece = 128 * 16, a_d = 3 * size_t(nsplit) * piece, a_l = size_t(nsplit) * piece;
  const size_t per_tile = NKD * a_d + NKL * a_l;
  blob.assign(per_tile * mtiles, 0);
  const std::vector<double>* D[3] = {&R.Dr, &R.Ds, &R.Dt};
  auto put = [&](size_t base, int i_loc, int k_loc, double x) {
    const size_t off = size_t(i_loc / 8) * 128 + size_t(k_loc / 8) * 64 + size_t(i_loc % 8) * 8 + (k_loc % 8);
    double rem = x;
    for (int h = 0; h < nsplit; ++h) {
      const uint16_t b = bf16_bits(float(rem));
      blob[base + h * piece + off] = b;
      rem -= bf16_value(b);
    }
  };
  for (int mt = 0; mt < mtiles; ++mt) {
    const size_t t0 = mt * per_tile;
    for (int il = 0; il < 128; ++il) {
      const int i = mt * 128 + il;
      if (i >= Np) break;
      for (int j = 0; j < Np; ++j)
        for (int d = 0; d < 3; ++d)
          put(t0 + size_t(j / 16) * a_d + size_t(d) * nsplit * piece, il, j % 16, (*D[d])[size_t(i) * Np + j]);
      for (int m = 0; m < NFN; ++m)
        put(t0 + NKD * a_d + size_t(m / 16) * a_l, il, m % 16, R.LIFT[size_t(i) * NFN + m]);
    }
  }
  return DG_OK;
}

// Buffers of the split step: X[tiles][KX][NE] and the operator blob with rows padded.
int Handle::ensure_split(const dgk::KernelCfg* c) {
  if (!c || !c->split || opts.strategy != DG_STRATEGY_FUSED) return DG_OK;
  if (c->split == 2) {
    if (d_tc) return DG_OK;
    const size_t ntiles = size_t((Kpad + c->gemm_ne - 1) / c->gemm_ne) + 1;
    const size_t xbytes = ntiles * c->gemm_xtile;
    std::vector<uint16_t> blob;
    pack_tc_ops(ref, c->gemm_nsplit, c->gemm_mtiles, blob);
    const size_t obytes = (blob.size() * 2 + 255) & ~size_t(255);
    DG_CUDA(cudaMalloc(&d_tc, xbytes + obytes));
    split_bytes += xbytes + obytes;
    d_opstc = d_tc;
    d_xtc = reinterpret_cast<float*>(static_cast<char*>(d_tc) + obytes);
    DG_CUDA(cudaMemsetAsync(d_xtc, 0, xbytes, stream));
    DG_CUDA(cudaMemcpyAsync(d_opstc, blob.data(), blob.size() * 2, cudaMemcpyHostToDevice, stream));
    DG_CUDA(cudaStreamSynchronize(stream));
    return DG_OK;
  }
  if (d_split) return DG_OK;
  const size_t ntiles = size_t((Kpad + c->gemm_ne - 1) / c->gemm_ne);
  const size_t xbytes = ntiles * c->gemm_kx * c->gemm_ne * 4;
  const int KD = 3 * Np + 4 * Nfp, MP2 = c->gemm_mp2;
  std::vector<float> ops2(size_t(KD) * MP2, 0.0f);
  const std::vector<double>* D[3] = {&ref.Dr, &ref.Ds, &ref.Dt};
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < Np; ++j)
      for (int i = 0; i < Np; ++i) ops2[size_t(d * Np + j) * MP2 + i] = float((*D[d])[size_t(i) * Np + j]);
  for (int cc = 0; cc < 4 * Nfp; ++cc)
    for (int i = 0; i < Np; ++i) ops2[size_t(3 * Np + cc) * MP2 + i] = float(ref.LIFT[size_t(i) * 4 * Nfp + cc]);
  const size_t obytes = (ops2.size() * 4 + 255) & ~size_t(255);
  DG_CUDA(cudaMalloc(&d_split, xbytes + obytes));
  split_bytes += xbytes + obytes;
  d_ops2 = static_cast<float*>(d_split);
  d_x = reinterpret_cast<float*>(static_cast<char*>(d_split) + obytes);
  DG_CUDA(cudaMemsetAsync(d_x, 0, xbytes, stream));
  DG_CUDA(cudaMemcpyAsync(d_ops2, ops2.data(), ops2.size() * 4, cudaMemcpyHostToDevice, stream));
  DG_CUDA(cudaStreamSynchronize(stream));
  return DG_OK;
}

dgk::StepArgs Handle::args(int mode) const {
  dgk::StepArgs a{};
  a.q = d_q[qcur];
  a.qn = d_q[1 - qcur];
  a.r1 = d_r[r1slot];
  a.r2 = d_r[1 - r1slot];
  a.rec = d_geo;
  a.nbr = reinterpret_cast<const int4*>(d_nbr);
  a.ops = d_ops;
  a.ftab = d_ftab;
  a.srcvec = src_elem >= 0 ? d_src : nullptr;
  a.src_elem = src_elem;
  a.src_amp = (src_elem >= 0 && step >= 0 && step < int64_t(src_amp.size())) ? float(src_amp[step]) : 0.0f;
  a.K = int(K);
  a.mode = mode;
  a.flux = opts.flux;
  a.bc = (model == DG_ELASTIC && opts.bc == DG_BC_RIGID) ? 1 : 0;
  a.dt = float(opts.dt);
  if (have == 0) { a.a1 = 1.0f; a.a2 = 0.0f; a.a3 = 0.0f; }
  else if (have == 1) { a.a1 = 1.5f; a.a2 = -0.5f; a.a3 = 0.0f; }
  else { a.a1 = float(23.0 / 12.0); a.a2 = float(-16.0 / 12.0); a.a3 = float(5.0 / 12.0); }
  a.err = d_err;
  a.wait_limit = wait_limit;
  split_ptrs(a, cfg);
  return a;
}

void Handle::split_ptrs(dgk::StepArgs& a, const dgk::KernelCfg* c) const {
  const bool tc = c && c->split == 2;
  a.xg = tc ? d_xtc : d_x;
  a.ops2 = d_ops2;
  a.opstc = d_opstc;
}

int Handle::advance(int nsteps) {
  int rc = ensure_split(cfg);
  if (rc) return rc;
  if (nrec > 0 && nsamples + nsteps > trace_cap) {
    // grow the trace buffer (keep what was recorded)
    const int64_t cap = std::max<int64_t>(nsamples + nsteps, 2 * trace_cap);
    float* nb = nullptr;
    const size_t per = size_t(nrec) * Nf * sizeof(float);
    if (cudaMalloc(reinterpret_cast<void**>(&nb), size_t(cap) * per) != cudaSuccess)
      return fail(DG_ENOMEM, "receiver trace buffer");
    if (nsamples > 0) DG_CUDA(cudaMemcpyAsync(nb, d_traces, size_t(nsamples) * per, cudaMemcpyDeviceToDevice, stream));
    if (d_traces) {
      DG_CUDA(cudaStreamSynchronize(stream));
      cudaFree(d_traces);
    }
    d_traces = nb;
    trace_cap = cap;
  }
  for (int s = 0; s < nsteps; ++s) {
    dgk::StepArgs a = args(0);
    int lr = launch(a);
    if (lr) return lr;
    qcur ^= 1;
    r1slot ^= 1;  // r^m was written into the r^{m-2} slot
    ++step;
    have = std::min(have + 1, 2);
    if (nrec > 0) {
      DG_CUDA(dgk::launch_sample(d_q[qcur], d_recel, d_recvec, nrec, Nf, Np,
                                 d_traces + size_t(nsamples) * nrec * Nf, stream));
      ++nsamples;
      ++launches;
    }
    if (finite_every > 0 && step % finite_every == 0) {
      DG_CUDA(dgk::launch_finite_check(d_q[qcur], (long long)K * Nf * Np, d_err, stream));
      ++launches;
    }
  }
  return DG_OK;
}

int64_t Handle::locate(const double x[3], double rst_out[3]) const {
  int64_t best = -1;
  double bestmin = -1e300;
  for (int64_t k = 0; k < K; ++k) {
    const double* x1 = &verts[3 * tets[4 * k]];
    const double* gk = &hm.g[9 * k];
    const double d[3] = {x[0] - x1[0], x[1] - x1[1], x[2] - x1[2]};
    double rst[3];
    for (int j = 0; j < 3; ++j) rst[j] = gk[j] * d[0] + gk[3 + j] * d[1] + gk[6 + j] * d[2] - 1.0;
    const double lam[4] = {-(1 + rst[0] + rst[1] + rst[2]) / 2, (1 + rst[0]) / 2, (1 + rst[1]) / 2,
                           (1 + rst[2]) / 2};
    const double mn = std::min(std::min(lam[0], lam[1]), std::min(lam[2], lam[3]));
    if (mn > bestmin) {
      bestmin = mn;
      best = k;
      std::memcpy(rst_out, rst, sizeof(rst));
    }
  }
  return (best < 0 || bestmin < -1e-9) ? -1 : best;
}

int Handle::source_vector(const double x[3], const double dir[3], int64_t* elem, std::vector<float>& vec) const {
  if (!x) return fail(DG_EINVAL, "source position is NULL");
  double brst[3] = {0, 0, 0};
  const int64_t best = locate(x, brst);
  if (best < 0) return fail(DG_EINVAL, "source position outside the mesh");
  // M_k^{-1} l(x_s) = V psi(x_s) / J_k  (V orthonormal Vandermonde)
  std::vector<double> psi(ref.Np), b(ref.Np, 0.0);
  ref.basis(brst[0], brst[1], brst[2], psi.data());
  for (int i = 0; i < ref.Np; ++i) {
    double acc = 0;
    for (int m = 0; m < ref.Np; ++m) acc += ref.V[size_t(i) * ref.Np + m] * psi[m];
    b[i] = acc / hm.J[best];
  }
  vec.assign(size_t(Nf) * ref.Np, 0.0f);
  if (model == DG_ACOUSTIC) {
    for (int i = 0; i < ref.Np; ++i) vec[i] = float(b[i]);
  } else {
    double dd[3] = {0, 0, 1};
    if (dir) std::memcpy(dd, dir, sizeof(dd));
    const double rho = coeffs[3 * best + 2];
    for (int c = 0; c < 3; ++c)
      for (int i = 0; i < ref.Np; ++i) vec[size_t(c) * ref.Np + i] = float(dd[c] / rho * b[i]);
  }
  *elem = best;
  return DG_OK;
}

// Device copy of the sources beyond the first: elements, vectors and the
// amplitudes zero-padded to the longest history, in one allocation.
int Handle::upload_xsrc() {
  const int n = int(xs_elem.size());
  int namp = 0;
  for (const auto& v : xs_amp) namp = std::max(namp, int(v.size()));
  if (d_xs) {
    DG_CUDA(cudaStreamSynchronize(stream));
    cudaFree(d_xs);
    d_xs = nullptr;
  }
  xs = dgk::XSrc{};
  if (n == 0) return DG_OK;
  const size_t NfNp = size_t(Nf) * Np;
  const size_t o_vec = (size_t(n) * 4 + 15) & ~size_t(15);
  const size_t o_amp = o_vec + size_t(n) * NfNp * 4;
  const size_t bytes = o_amp + size_t(n) * namp * 4;
  if (cudaMalloc(&d_xs, bytes) != cudaSuccess) {
    d_xs = nullptr;
    return fail(DG_ENOMEM, "source tables");
  }
  std::vector<unsigned char> host(bytes, 0);
  std::memcpy(host.data(), xs_elem.data(), size_t(n) * 4);
  std::memcpy(host.data() + o_vec, xs_vec.data(), size_t(n) * NfNp * 4);
  float* ha = reinterpret_cast<float*>(host.data() + o_amp);
  for (int s = 0; s < n; ++s)
    for (size_t m = 0; m < xs_amp[s].size(); ++m) ha[size_t(s) * namp + m] = float(xs_amp[s][m]);
  DG_CUDA(cudaMemcpyAsync(d_xs, host.data(), bytes, cudaMemcpyHostToDevice, stream));
  DG_CUDA(cudaStreamSynchronize(stream));
  auto* base = static_cast<unsigned char*>(d_xs);
  xs.n = n;
  xs.namp = namp;
  xs.elem = reinterpret_cast<const int*>(base);
  xs.vec = reinterpret_cast<const float*>(base + o_vec);
  xs.amp = reinterpret_cast<const float*>(base + o_amp);
  return DG_OK;
}

}  // namespace dg

using dg::fail;

extern "C" {

const char* dg_last_error(void) { return dg::g_err.c_str(); }

int dg_setup(const dg_mesh* mesh, const double* coeffs, int N, int model, const dg_opts* opts,
             dg_handle** out) {
  if (!out) return fail(DG_EINVAL, "out is NULL");
  *out = nullptr;
  auto* h = new (std::nothrow) dg_handle();
  if (!h) return fail(DG_ENOMEM, "host allocation failed");
  int rc = h->init(mesh, coeffs, N, model, opts);
  if (rc) {
    delete h;
    return rc;
  }
  *out = h;
  return DG_OK;
}

void dg_destroy(dg_handle* h) { delete h; }

int dg_info(const dg_handle* h, int64_t* K, int* Np, int* Nfp, int* Nf) {
  if (!h) return fail(DG_EINVAL, "NULL handle");
  if (K) *K = h->K;
  if (Np) *Np = h->Np;
  if (Nfp) *Nfp = h->Nfp;
  if (Nf) *Nf = h->Nf;
  return DG_OK;
}

// Memory kind of a dg_set_state / dg_get_state buffer: 0 host (the call
// waits for its copies), 1 device, 2 page-locked host memory (the copies
// stay in stream order).  Mode 2 refuses memory that is not page-locked.
static int check_transfer(const void* p, int on_device) {
  if (on_device < 0 || on_device > 2) return fail(DG_EINVAL, "on_device must be 0, 1 or 2");
  if (on_device != 2 || !p) return DG_OK;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) return dg::cuda_fail(e, "cudaPointerGetAttributes");
  if (at.type != cudaMemoryTypeHost) return fail(DG_EINVAL, "on_device = 2 needs page-locked host memory");
  return DG_OK;
}

int dg_set_state(dg_handle* h, const float* q, const float* r1, const float* r2, int64_t step,
                 int on_device) {
  if (!h || !q) return fail(DG_EINVAL, "NULL handle or state");
  if ((r1 == nullptr) != (r2 == nullptr)) return fail(DG_EINVAL, "give both r1 and r2 or neither");
  for (const void* p : {static_cast<const void*>(q), static_cast<const void*>(r1), static_cast<const void*>(r2)}) {
    int rc = check_transfer(p, on_device);
    if (rc) return rc;
  }
  const size_t bytes = size_t(h->K) * h->Nf * h->Np * 4;
  const cudaMemcpyKind kind = on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  DG_CUDA(cudaMemcpyAsync(h->d_q[h->qcur], q, bytes, kind, h->stream));
  if (r1) {
    DG_CUDA(cudaMemcpyAsync(h->d_r[h->r1slot], r1, bytes, kind, h->stream));
    DG_CUDA(cudaMemcpyAsync(h->d_r[1 - h->r1slot], r2, bytes, kind, h->stream));
    h->have = 2;
  } else {
    DG_CUDA(cudaMemsetAsync(h->d_r[0], 0, h->state_bytes, h->stream));
    DG_CUDA(cudaMemsetAsync(h->d_r[1], 0, h->state_bytes, h->stream));
    h->have = 0;
  }
  h->step = step;
  if (on_device == 0) DG_CUDA(cudaStreamSynchronize(h->stream));
  return DG_OK;
}

int dg_get_state(dg_handle* h, float* q, float* r1, float* r2, int64_t* step, int* history,
                 int on_device) {
  if (!h) return fail(DG_EINVAL, "NULL handle");
  for (const void* p : {static_cast<const void*>(q), static_cast<const void*>(r1), static_cast<const void*>(r2)}) {
    int rc = check_transfer(p, on_device);
    if (rc) return rc;
  }
  const size_t bytes = size_t(h->K) * h->Nf * h->Np * 4;
  const cudaMemcpyKind kind = on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (q) DG_CUDA(cudaMemcpyAsync(q, h->d_q[h->qcur], bytes, kind, h->stream));
  if (r1) DG_CUDA(cudaMemcpyAsync(r1, h->d_r[h->r1slot], bytes, kind, h->stream));
  if (r2) DG_CUDA(cudaMemcpyAsync(r2, h->d_r[1 - h->r1slot], bytes, kind, h->stream));
  if (step) *step = h->step;
  if (history) *history = h->have;
  if (on_device == 0) DG_CUDA(cudaStreamSynchronize(h->stream));
  return DG_OK;
}

int dg_set_stream(dg_handle* h, void* stream) {
  if (!h) return fail(DG_EINVAL, "NULL handle");
  DG_CUDA(cudaStreamSynchronize(h->stream));  // work already issued finishes on the old stream
  h->stream = static_cast<cudaStream_t>(stream);
  h->opts.stream = stream;
  return DG_OK;
}

int dg_rhs(dg_handle* h, float* r_out, int on_device) {
  if (!h || !r_out) return fail(DG_EINVAL, "NULL handle or output");
  int rc0 = h->ensure_split(h->cfg);
  if (rc0) return rc0;
  dgk::StepArgs a = h->args(1);
  float* tmp = nullptr;
  const size_t bytes = size_t(h->K) * h->Nf * h->Np * 4;
  if (on_device) {
    a.rout = r_out;
  } else {
    DG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&tmp), bytes, h->stream));
    a.rout = tmp;
  }
  const int lr = h->launch(a);
  if (lr) {
    if (tmp) cudaFreeAsync(tmp, h->stream);
    return lr;
  }
  if (!on_device) {
    DG_CUDA(cudaMemcpyAsync(r_out, tmp, bytes, cudaMemcpyDeviceToHost, h->stream));
    DG_CUDA(cudaFreeAsync(tmp, h->stream));
    DG_CUDA(cudaStreamSynchronize(h->stream));
  }
  return DG_OK;
}

int dg_step(dg_handle* h, int nsteps) {
  if (!h || nsteps < 0) return fail(DG_EINVAL, "NULL handle or negative step count");
  if (!(h->opts.dt > 0)) return fail(DG_EINVAL, "dt must be positive (dg_opts.dt or dg_set_dt)");
  return h->advance(nsteps);
}

int dg_set_dt(dg_handle* h, double dt) {
  if (!h || !(dt > 0) || !std::isfinite(dt)) return fail(DG_EINVAL, "dt must be positive");
  h->opts.dt = dt;
  return DG_OK;
}

int dg_sync(dg_handle* h) {
  if (!h) return fail(DG_EINVAL, "NULL handle");
  DG_CUDA(cudaStreamSynchronize(h->stream));
  int err = 0;
  DG_CUDA(cudaMemcpy(&err, h->d_err, 4, cudaMemcpyDeviceToHost));
  if (!err) return DG_OK;
  // report once: the error word starts over for the next steps
  DG_CUDA(cudaMemsetAsync(h->d_err, 0, 4, h->stream));
  DG_CUDA(cudaStreamSynchronize(h->stream));
  if (err & 1) return fail(DG_ETIMEOUT, "a bounded device-side wait expired");
  return fail(DG_ENONFINITE, "the state holds a NaN or an infinity");
}

int dg_set_wait_limit(dg_handle* h, int64_t cycles) {
  if (!h) return fail(DG_EINVAL, "NULL handle");
  h->wait_limit = (long long)cycles;
  return DG_OK;
}

int dg_set_finite_check(dg_handle* h, int every) {
  if (!h || every < 0) return fail(DG_EINVAL, "NULL handle or negative interval");
  h->finite_every = every;
  return DG_OK;
}

int dg_launch_count(const dg_handle* h, int64_t* launches) {
  if (!h || !launches) return fail(DG_EINVAL, "NULL handle or output");
  *launches = h->launches;
  return DG_OK;
}

int dg_node_coords(const dg_handle* h, double* xyz) {
  if (!h || !xyz) return fail(DG_EINVAL, "NULL handle or output");
  const auto& R = h->ref;
  for (int64_t k = 0; k < h->K; ++k) {
    const double* x1 = &h->verts[3 * h->tets[4 * k]];
    const double* A = &h->hm.A[9 * k];
    for (int n = 0; n < R.Np; ++n) {
      double u[3] = {1 + R.r[n], 1 + R.s[n], 1 + R.t[n]};
      for (int i = 0; i < 3; ++i)
        xyz[(size_t(k) * R.Np + n) * 3 + i] = x1[i] + A[3 * i] * u[0] + A[3 * i + 1] * u[1] + A[3 * i + 2] * u[2];
    }
  }
  return DG_OK;
}

int dg_set_source(dg_handle* h, const double xs[3], const double dir[3], const double* amp, int64_t namp) {
  if (!h) return fail(DG_EINVAL, "NULL handle");
  if (!amp || namp <= 0) {
    h->src_elem = -1;
    h->src_amp.clear();
    h->xs_elem.clear();
    h->xs_vec.clear();
    h->xs_amp.clear();
    return h->upload_xsrc();
  }
  int64_t best = -1;
  std::vector<float> vec;
  const int rc = h->source_vector(xs, dir, &best, vec);
  if (rc) return rc;
  DG_CUDA(cudaMemcpyAsync(h->d_src, vec.data(), vec.size() * 4, cudaMemcpyHostToDevice, h->stream));
  DG_CUDA(cudaStreamSynchronize(h->stream));
  h->src_elem = int(best);
  h->src_amp.assign(amp, amp + namp);
  h->xs_elem.clear();
  h->xs_vec.clear();
  h->xs_amp.clear();
  return h->upload_xsrc();
}

int dg_add_source(dg_handle* h, const double xs[3], const double dir[3], const double* amp, int64_t namp) {
  if (!h) return fail(DG_EINVAL, "NULL handle");
  if (!amp || namp <= 0) return fail(DG_EINVAL, "a source needs amplitudes");
  if (h->src_elem < 0) return dg_set_source(h, xs, dir, amp, namp);
  if (int(h->xs_elem.size()) + 1 >= DG_MAX_SOURCES) return fail(DG_EINVAL, "too many sources");
  int64_t best = -1;
  std::vector<float> vec;
  const int rc = h->source_vector(xs, dir, &best, vec);
  if (rc) return rc;
  h->xs_elem.push_back(int(best));
  h->xs_vec.insert(h->xs_vec.end(), vec.begin(), vec.end());
  h->xs_amp.emplace_back(amp, amp + namp);
  return h->upload_xsrc();
}

// Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix.
static bool invert(std::vector<double> a, int n, std::vector<double>& inv) {
  inv.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) inv[size_t(i) * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[size_t(r) * n + c]) > std::fabs(a[size_t(p) * n + c])) p = r;
    if (a[size_t(p) * n + c] == 0.0) return false;
    if (p != c)
      for (int j = 0; j < n; ++j) {
        std::swap(a[size_t(p) * n + j], a[size_t(c) * n + j]);
        std::swap(inv[size_t(p) * n + j], inv[size_t(c) * n + j]);
      }
    const double d = 1.0 / a[size_t(c) * n + c];
    for (int j = 0; j < n; ++j) {
      a[size_t(c) * n + j] *= d;
      inv[size_t(c) * n + j] *= d;
    }
    for (int r = 0; r < n; ++r)
      if (r != c && a[size_t(r) * n + c] != 0.0) {
        const double f = a[size_t(r) * n + c];
        for (int j = 0; j < n; ++j) {
          a[size_t(r) * n + j] -= f * a[size_t(c) * n + j];
          inv[size_t(r) * n + j] -= f * inv[size_t(c) * n + j];
        }
      }
  }
  return true;
}

int dg_set_receivers(dg_handle* h, const double* xyz, int nrec) {
  if (!h || nrec < 0 || (nrec > 0 && !xyz)) return fail(DG_EINVAL, "NULL handle, negative count or NULL points");
  const auto& R = h->ref;
  std::vector<int> el(size_t(std::max(nrec, 0)));
  std::vector<float> vec(size_t(std::max(nrec, 0)) * R.Np);
  if (nrec > 0 && h->Vinv.empty() && !invert(R.V, R.Np, h->Vinv))
    return fail(DG_EINVAL, "singular Vandermonde matrix");
  std::vector<double> psi(R.Np);
  for (int r = 0; r < nrec; ++r) {
    double rst[3];
    const int64_t k = h->locate(xyz + 3 * r, rst);
    if (k < 0) return fail(DG_EINVAL, "receiver " + std::to_string(r) + " outside the mesh");
    el[r] = int(k);
    // l_i(x) = sum_m psi_m(r(x)) (V^{-1})_{m i}
    R.basis(rst[0], rst[1], rst[2], psi.data());
    for (int i = 0; i < R.Np; ++i) {
      double acc = 0.0;
      for (int m = 0; m < R.Np; ++m) acc += psi[m] * h->Vinv[size_t(m) * R.Np + i];
      vec[size_t(r) * R.Np + i] = float(acc);
    }
  }
  DG_CUDA(cudaStreamSynchronize(h->stream));
  if (h->d_recel) cudaFree(h->d_recel);
  if (h->d_traces) cudaFree(h->d_traces);
  h->d_recel = nullptr;
  h->d_recvec = nullptr;
  h->d_traces = nullptr;
  h->trace_cap = h->nsamples = 0;
  h->nrec = 0;
  if (nrec == 0) return DG_OK;
  const size_t eb = (size_t(nrec) * 4 + 255) & ~size_t(255);
  DG_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->d_recel), eb + vec.size() * 4));
  h->d_recvec = reinterpret_cast<float*>(reinterpret_cast<char*>(h->d_recel) + eb);
  DG_CUDA(cudaMemcpyAsync(h->d_recel, el.data(), el.size() * 4, cudaMemcpyHostToDevice, h->stream));
  DG_CUDA(cudaMemcpyAsync(h->d_recvec, vec.data(), vec.size() * 4, cudaMemcpyHostToDevice, h->stream));
  DG_CUDA(cudaStreamSynchronize(h->stream));
  h->nrec = nrec;
  return DG_OK;
}

int dg_get_traces(dg_handle* h, float* out, int64_t* nsamples, int on_device) {
  if (!h) return fail(DG_EINVAL, "NULL handle");
  if (nsamples) *nsamples = h->nsamples;
  if (!out || h->nsamples == 0 || h->nrec == 0) return DG_OK;
  const size_t bytes = size_t(h->nsamples) * h->nrec * h->Nf * 4;
  DG_CUDA(cudaMemcpyAsync(out, h->d_traces, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          h->stream));
  DG_CUDA(cudaStreamSynchronize(h->stream));
  return DG_OK;
}

int dg_autotune(dg_handle* h, int reps, int* block_elems, double* ms_per_step, double* variant_ms) {
  if (!h || reps < 1) return fail(DG_EINVAL, "NULL handle or reps < 1");
  if (h->opts.strategy != DG_STRATEGY_FUSED) return fail(DG_EINVAL, "kernel variants apply to the fused strategy");
  int n = 0;
  const dgk::KernelCfg* v = dgk::kernel_variants(h->model, h->N, &n, h->opts.precision);
  for (int i = 0; i < n; ++i) {
    int rs = h->ensure_split(&v[i]);
    if (rs) return rs;
  }
  // scratch copies of the state so that the handle's state and history stay untouched
  void* scratch = nullptr;
  DG_CUDA(cudaMallocAsync(&scratch, 4 * h->state_bytes, h->stream));
  float* sq[2] = {static_cast<float*>(scratch), static_cast<float*>(scratch) + h->state_bytes / 4};
  float* sr[2] = {sq[1] + h->state_bytes / 4, sq[1] + 2 * (h->state_bytes / 4)};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DG_OK;
  int best = -1;
  float best_ms = 0.0f;
  auto run = [&]() -> int {
    for (int c = 0; c < 2; ++c) {
      DG_CUDA(cudaMemcpyAsync(sq[c], h->d_q[h->qcur], h->state_bytes, cudaMemcpyDeviceToDevice, h->stream));
      DG_CUDA(cudaMemcpyAsync(sr[c], h->d_r[c], h->state_bytes, cudaMemcpyDeviceToDevice, h->stream));
    }
    DG_CUDA(cudaEventCreate(&e0));
    DG_CUDA(cudaEventCreate(&e1));
    for (int i = 0; i < n; ++i) {
      dgk::StepArgs a = h->args(0);
      h->split_ptrs(a, &v[i]);
      a.a1 = 1.0f;
      a.a2 = a.a3 = 0.0f;
      a.src_elem = -1;
      a.srcvec = nullptr;
      int cur = 0;
      auto one = [&]() -> int {
        a.q = sq[cur];
        a.qn = sq[1 - cur];
        a.r1 = sr[cur];
        a.r2 = sr[1 - cur];
        DG_CUDA(dgk::launch_step(&v[i], a, h->stream));
        cur ^= 1;
        return DG_OK;
      };
      int r = one();  // warm-up (and shared-memory opt-in)
      if (r) return r;
      DG_CUDA(cudaEventRecord(e0, h->stream));
      for (int k = 0; k < reps; ++k) {
        r = one();
        if (r) return r;
      }
      DG_CUDA(cudaEventRecord(e1, h->stream));
      DG_CUDA(cudaEventSynchronize(e1));
      float ms = 0.0f;
      DG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      ms /= reps;
      if (variant_ms) variant_ms[i] = ms;
      if (best < 0 || ms < best_ms) {
        best = i;
        best_ms = ms;
      }
    }
    return DG_OK;
  };
  rc = run();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(scratch, h->stream);
  cudaStreamSynchronize(h->stream);
  if (rc) return rc;
  int err = 0;
  DG_CUDA(cudaMemcpy(&err, h->d_err, 4, cudaMemcpyDeviceToHost));
  if (err & 1) {
    DG_CUDA(cudaMemset(h->d_err, 0, 4));
    return fail(DG_ETIMEOUT, "a bounded device-side wait expired during tuning");
  }
  h->cfg = &v[best];
  {
    std::lock_guard<std::mutex> lock(dg::g_tune_mu);
    dg::g_tuned[std::make_tuple(h->device, h->model, h->N, h->opts.precision)] = best;
  }
  if (block_elems) *block_elems = v[best].EB;
  if (ms_per_step) *ms_per_step = best_ms;
  return DG_OK;
}

int dg_set_variant(dg_handle* h, int index) {
  if (!h) return fail(DG_EINVAL, "NULL handle");
  if (h->opts.strategy != DG_STRATEGY_FUSED) return fail(DG_EINVAL, "kernel variants apply to the fused strategy");
  int n = 0;
  const dgk::KernelCfg* v = dgk::kernel_variants(h->model, h->N, &n, h->opts.precision);
  if (index < 0 || index >= n) return fail(DG_EINVAL, "variant index out of range");
  h->cfg = &v[index];
  {
    std::lock_guard<std::mutex> lock(dg::g_tune_mu);
    dg::g_tuned[std::make_tuple(h->device, h->model, h->N, h->opts.precision)] = index;
  }
  return DG_OK;
}

int dg_kernel_info(const dg_handle* h, int* block_elems, int* threads, int64_t* smem_bytes, int* variants,
                   int* tile_elems, int* split, int* variant) {
  if (!h || !h->cfg) return fail(DG_EINVAL, "NULL handle");
  if (variant) {
    int n = 0;
    const dgk::KernelCfg* v = dgk::kernel_variants(h->model, h->N, &n, h->opts.precision);
    *variant = (v && h->cfg >= v && h->cfg < v + n) ? int(h->cfg - v) : -1;
  }
  if (split) *split = h->cfg->split;
  if (tile_elems) *tile_elems = h->cfg->TN;
  if (block_elems) *block_elems = h->cfg->EB;
  if (threads) *threads = h->cfg->NT;
  if (smem_bytes) *smem_bytes = int64_t(h->cfg->smem);
  if (variants) dgk::kernel_variants(h->model, h->N, variants, h->opts.precision);
  return DG_OK;
}

int dg_suggest_dt(const dg_mesh* mesh, const double* coeffs, int N, int model, double cfl, double* dt) {
  if (!dt || !(cfl > 0)) return fail(DG_EINVAL, "bad arguments");
  if (N < 1 || N > 8) return fail(DG_EINVAL, "polynomial degree N must be in 1..8");
  dg::HostMesh m;
  int rc = m.build(mesh);
  if (rc) return rc;
  rc = dg::check_coeffs(coeffs, m.K, model);
  if (rc) return rc;
  *dt = dg::suggest_dt(m, coeffs, N, model, cfl);
  return DG_OK;
}

int dg_reference_element(int N, double* nodes, double* Dr, double* Ds, double* Dt, double* LIFT, int* fmask) {
  dg::RefElement R;
  int rc = R.build(N);
  if (rc) return rc;
  const size_t Np = R.Np;
  if (nodes)
    for (size_t n = 0; n < Np; ++n) {
      nodes[3 * n] = R.r[n];
      nodes[3 * n + 1] = R.s[n];
      nodes[3 * n + 2] = R.t[n];
    }
  if (Dr) std::memcpy(Dr, R.Dr.data(), Np * Np * sizeof(double));
  if (Ds) std::memcpy(Ds, R.Ds.data(), Np * Np * sizeof(double));
  if (Dt) std::memcpy(Dt, R.Dt.data(), Np * Np * sizeof(double));
  if (LIFT) std::memcpy(LIFT, R.LIFT.data(), R.LIFT.size() * sizeof(double));
  if (fmask) std::memcpy(fmask, R.fmask.data(), R.fmask.size() * sizeof(int));
  return DG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- autotune cache
// One line per choice: device name (spaces as '_'), compute capability,
// model, N, precision, variant index and the variant's shape (elements per
// block, threads, split form, GEMM threads), so that a stale line (another
// build's variant table) is recognised and skipped.
namespace {
const char* kTuneHeader = "# libdg autotune cache v1";

int device_tag(int dev, std::string* name, int* major, int* minor) {
  cudaDeviceProp p;
  cudaError_t e = cudaGetDeviceProperties(&p, dev);
  if (e != cudaSuccess) return dg::cuda_fail(e, "cudaGetDeviceProperties");
  std::string n(p.name);
  for (auto& ch : n)
    if (ch == ' ' || ch == '\t') ch = '_';
  *name = n;
  *major = p.major;
  *minor = p.minor;
  return DG_OK;
}
}  // namespace

extern "C" int dg_tune_save(const char* path) {
  if (!path) return fail(DG_EINVAL, "NULL path");
  std::map<std::tuple<int, int, int, int>, int> tuned;
  {
    std::lock_guard<std::mutex> lock(dg::g_tune_mu);
    tuned = dg::g_tuned;
  }
  std::ostringstream out;
  out << kTuneHeader << "\n";
  for (const auto& kv : tuned) {
    const int dev = std::get<0>(kv.first), model = std::get<1>(kv.first), N = std::get<2>(kv.first),
              prec = std::get<3>(kv.first), idx = kv.second;
    int n = 0;
    const dgk::KernelCfg* v = dgk::kernel_variants(model, N, &n, prec);
    if (!v || idx < 0 || idx >= n) continue;
    std::string name;
    int major = 0, minor = 0;
    int rc = device_tag(dev, &name, &major, &minor);
    if (rc) return rc;
    out << name << " " << major << "." << minor << " " << model << " " << N << " " << prec << " " << idx << " "
        << v[idx].EB << " " << v[idx].NT << " " << v[idx].split << " " << v[idx].gemm_threads << "\n";
  }
  std::ofstream f(path);
  if (!f) return fail(DG_EINVAL, std::string("cannot write ") + path);
  f << out.str();
  if (!f) return fail(DG_EINVAL, std::string("cannot write ") + path);
  return DG_OK;
}

extern "C" int dg_tune_load(const char* path, int* applied) {
  if (applied) *applied = 0;
  if (!path) return fail(DG_EINVAL, "NULL path");
  std::ifstream f(path);
  if (!f) return fail(DG_EINVAL, std::string("cannot read ") + path);
  struct Line {
    std::string name;
    int major, minor, model, N, prec, idx, EB, NT, split, gthreads;
  };
  std::vector<Line> lines;
  std::string ln;
  bool header = false;
  int lineno = 0;
  while (std::getline(f, ln)) {
    ++lineno;
    if (ln.empty()) continue;
    if (ln[0] == '#') {
      if (ln == kTuneHeader) header = true;
      continue;
    }
    std::istringstream is(ln);
    Line L;
    std::string cc;
    char dot = 0;
    if (!(is >> L.name >> cc >> L.model >> L.N >> L.prec >> L.idx >> L.EB >> L.NT >> L.split >> L.gthreads))
      return fail(DG_EINVAL, std::string(path) + ": malformed line " + std::to_string(lineno));
    std::istringstream cs(cc);
    if (!(cs >> L.major >> dot >> L.minor) || dot != '.')
      return fail(DG_EINVAL, std::string(path) + ": malformed compute capability on line " + std::to_string(lineno));
    lines.push_back(L);
  }
  if (!header) return fail(DG_EINVAL, std::string(path) + ": not a libdg autotune cache");
  if (lines.empty()) return DG_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dg::cuda_fail(e, "cudaGetDevice");
  std::string name;
  int major = 0, minor = 0;
  int rc = device_tag(dev, &name, &major, &minor);
  if (rc) return rc;
  int taken = 0;
  for (const auto& L : lines) {
    if (L.name != name || L.major != major || L.minor != minor) continue;
    int n = 0;
    const dgk::KernelCfg* v = dgk::kernel_variants(L.model, L.N, &n, L.prec);
    if (!v || L.idx < 0 || L.idx >= n) continue;
    const dgk::KernelCfg& c = v[L.idx];
    if (c.EB != L.EB || c.NT != L.NT || c.split != L.split || c.gemm_threads != L.gthreads) continue;
    std::lock_guard<std::mutex> lock(dg::g_tune_mu);
    dg::g_tuned[std::make_tuple(dev, L.model, L.N, L.prec)] = L.idx;
    ++taken;
  }
  if (applied) *applied = taken;
  return DG_OK;
}

extern "C" int dg_tune_clear(void) {
  std::lock_guard<std::mutex> lock(dg::g_tune_mu);
  dg::g_tuned.clear();
  return DG_OK;
}
