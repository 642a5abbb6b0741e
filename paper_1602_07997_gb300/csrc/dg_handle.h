// The solver handle behind the opaque dg_handle of the C ABI.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "dg_args.h"
#include "dg_internal.h"

namespace dg {

int cuda_fail(cudaError_t e, const char* what);
int check_coeffs(const double* coeffs, int64_t K, int model);
void pack_ops(const RefElement& R, std::vector<float>& ops, std::vector<int>& ftab);
void pack_records(const HostMesh& hm, const double* coeffs, int model, int64_t Kpad, std::vector<float>& rec,
                  std::vector<int32_t>& nbr);
double suggest_dt(const HostMesh& m, const double* coeffs, int N, int model, double cfl);
const dgk::KernelCfg* select_variant(int model, int N, int block_elems, int device, int precision);

struct Handle {
  int model = 0, N = 0, Np = 0, Nfp = 0, Nf = 0, device = 0;
  int64_t K = 0, Kpad = 0;
  dg_opts opts{};
  cudaStream_t stream = nullptr;
  RefElement ref;
  HostMesh hm;
  std::vector<double> coeffs, verts;
  std::vector<int64_t> tets;
  const dgk::KernelCfg* cfg = nullptr;

  // device memory: one allocation carved into the pieces below
  void* d_base = nullptr;
  size_t device_bytes = 0, state_bytes = 0;
  size_t split_bytes = 0;  // split-step buffers allocated on first use
  float* d_q[2] = {nullptr, nullptr};  // ping-pong q^m / q^{m+1}
  float* d_r[2] = {nullptr, nullptr};  // AB3 history slots
  float* d_geo = nullptr;  // element records, dgk::Rec layout
  int32_t* d_nbr = nullptr;
  float* d_ops = nullptr;
  int* d_ftab = nullptr;
  float* d_src = nullptr;
  int* d_err = nullptr;
  // split step (high N): GEMM inputs and the row-padded operator blob, allocated on first use
  void* d_split = nullptr;
  float* d_x = nullptr;
  float* d_ops2 = nullptr;
  // tensor-core split step: FP32 GEMM inputs and the BF16 operator pieces, allocated on first use
  void* d_tc = nullptr;
  float* d_xtc = nullptr;
  void* d_opstc = nullptr;
  // comparison strategies (allocated on first use): library route X, operator
  // blob and GEMM products; plain route partial RHS
  void* cublas = nullptr;
  void* d_lib = nullptr;
  float* d_libx = nullptr;
  float* d_libops = nullptr;
  float* d_liby = nullptr;
  size_t libyprod = 0;
  float* d_r0 = nullptr;

  long long wait_limit = 0;  // bounded device waits (StepArgs::wait_limit)
  int finite_every = 100;    // check the state for NaN/Inf after every this many steps (0 = never)
  int64_t launches = 0;      // kernels of this library launched by the handle
  int qcur = 0;    // which q buffer holds q^m
  int r1slot = 0;  // which r buffer holds r^{m-1}; the other holds r^{m-2}
  int64_t step = 0;
  int have = 0;    // stored RHS levels (0, 1, 2)
  int src_elem = -1;
  std::vector<double> src_amp;
  // point sources beyond the first (added after the step kernels): host
  // copies, one device allocation and its view
  std::vector<int> xs_elem;
  std::vector<float> xs_vec;                // [n][Nf Np]
  std::vector<std::vector<double>> xs_amp;  // amplitudes of each source
  void* d_xs = nullptr;
  dgk::XSrc xs{};
  // receivers: element and interpolation vector per receiver (device), traces
  int nrec = 0;
  int* d_recel = nullptr;
  float* d_recvec = nullptr;  // [nrec][Np]
  float* d_traces = nullptr;  // [trace_cap][nrec][Nf]
  int64_t trace_cap = 0, nsamples = 0;
  std::vector<double> Vinv;   // inverse Vandermonde, on first use
  // dg_rhs_host_noalloc: device address of the library's fixed scratch array
  // and the fused FP32 variant it runs, both resolved (and that kernel
  // loaded) by init; null when the mesh's RHS does not fit the array
  float* noalloc_scratch = nullptr;
  const dgk::KernelCfg* noalloc_cfg = nullptr;

  int init(const dg_mesh* mesh, const double* coeffs, int N, int model, const dg_opts* o);
  // set-up of dg_rhs_host_noalloc (rhs_noalloc.cu), called at the end of init
  int noalloc_prepare();
  // element whose smallest barycentric coordinate of x is largest, and the
  // reference coordinates of x in it; -1 if x is outside the mesh
  int64_t locate(const double x[3], double rst[3]) const;
  // element and RHS vector [Nf][Np] of a point source at x (dg_set_source)
  int source_vector(const double x[3], const double dir[3], int64_t* elem, std::vector<float>& vec) const;
  int upload_xsrc();
  int ensure_split(const dgk::KernelCfg* c);
  int ensure_strategy();
  // one step (a.mode 0) or RHS (mode 1) with the handle's strategy
  int launch(dgk::StepArgs a);
  // the split-step buffers of variant c (own, or those of the handle's variant)
  void split_ptrs(dgk::StepArgs& a, const dgk::KernelCfg* c) const;
  dgk::StepArgs args(int mode) const;
  int advance(int nsteps);
  ~Handle();
};

}  // namespace dg

struct dg_handle : dg::Handle {};
