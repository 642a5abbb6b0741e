// Served solves with continuous batching (dg_server_* / dg_submit / dg_poll).
//
// Two host threads per server, each with its own CUDA stream:
//   1. admission (set-up thread): queued requests are set up (mesh, operators,
//      state) while free device memory minus a reserve, and the optional byte
//      budget, cover them and fewer than max_batch solves are admitted; the
//      GPU keeps stepping the active solves meanwhile;
//   2. batching: active solves are grouped by (model, N); one tick advances
//      every active solve by one AB3 step with one persistent batched launch
//      per group (two for the split step: front half, then the GEMM over all
//      the group's column tiles) plus one tiny launch that advances the
//      per-solve step state on the device; the tick is captured once in a
//      CUDA graph and replayed until the set of active solves changes;
//   3. ticks run in chunks that end when the first active solve finishes (at
//      most kMaxChunk ticks), so that requests that arrived meanwhile join at
//      the next chunk boundary (continuous batching);
//   4. a finished solve's q is copied to host memory owned by the server and
//      its device memory is released before new requests are admitted.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "dg_args.h"
#include "dg_handle.h"

namespace dg {

namespace {

constexpr int kMaxChunk = 32;                  // ticks between admission points
constexpr size_t kReserve = size_t(1) << 30;   // device memory kept free

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

enum Status { kQueued = 0, kRunning = 1, kDone = 2, kCancelled = 3, kFailed = 4 };

struct Request {
  uint64_t id = 0;
  std::vector<double> verts, coeffs, amp;
  std::vector<int64_t> tets;
  std::vector<float> q0;
  int N = 0, model = 0, nsteps = 0;
  dg_opts opts{};
  bool has_src = false;
  double xs[3] = {0, 0, 0}, dir[3] = {0, 0, 1};
  // sources beyond the first: positions [n][3], directions [n][3], amplitudes [n][namp]
  std::vector<double> ex_xyz, ex_dir, ex_amp;
  int64_t ex_namp = 0;
  double t_submit = 0, t_done = 0;
  int status = kQueued;
  bool cancel = false;
  int error = DG_OK;
  std::string message;
  std::vector<float> q_out;
};

struct Active {
  std::shared_ptr<Request> req;
  dg_handle* h = nullptr;
  float* d_amp = nullptr;
  int steps_left = 0;
};

struct Group {
  int model = 0, N = 0;
  const dgk::KernelCfg* cfg = nullptr;
  std::vector<Active*> members;
  dgk::SolveDev* d_solves = nullptr;
  int* d_block_start = nullptr;
  int* d_block_solve = nullptr;
  int* d_tile_start = nullptr;  // split step: GEMM tiles of each solve
  int* d_tile_solve = nullptr;
  int capacity = 0, block_capacity = 0, tile_capacity = 0;
  int total_blocks = 0, total_tiles = 0;
  bool has_xs = false;  // a member has sources beyond the first
};

}  // namespace

struct Server {
  size_t budget = 0;
  int max_batch = 64;
  int device = 0;
  cudaStream_t stream = nullptr;       // steps
  cudaStream_t prep_stream = nullptr;  // set-up of admitted requests
  std::thread thr, prep_thr;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  uint64_t next_id = 1;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::vector<std::unique_ptr<Active>> active;
  std::vector<std::unique_ptr<Active>> ready;  // set up, waiting for the next chunk boundary
  std::map<std::pair<int, int>, Group> groups;
  // kernel variant of each (model, N): the autotuned FP32 choice of the
  // process when it has a batched form, fixed at the first admission
  std::map<std::pair<int, int>, const dgk::KernelCfg*> cfg_of;
  size_t active_bytes = 0;  // admitted (ready + active)
  int admitted = 0;
  std::atomic<int64_t> launches{0};
  cudaGraphExec_t graph = nullptr;
  bool dirty = true;
  int* d_err = nullptr;
  // one side stream per (model, N) group in the tick graph, so that the
  // groups' batched kernels overlap on the device; fork and join events
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;

  ~Server();
  void loop();
  void prep_loop();
  bool admit_one(std::shared_ptr<Request> r);
  void activate_ready();
  int rebuild();
  void retire(Active* a, int status);
  void fail_request(const std::shared_ptr<Request>& r, int code, const std::string& msg);
};

static size_t estimate_bytes(const Request& r, const dgk::KernelCfg* cfg) {
  const int Np = num_nodes(r.N), Nf = num_fields(r.model), Nfp = num_face_nodes(r.N);
  const size_t K = r.tets.size() / 4 + 132;
  const size_t Mpad = size_t((Np + 3) & ~3), KD = size_t(3 * Np + 4 * Nfp);
  size_t b = 4 * K * Nf * Np * 4 + K * (25 * 4 + 16) + KD * Mpad * 4 + r.amp.size() * 4 + (size_t(1) << 20);
  if (cfg && cfg->split)  // GEMM inputs and the row-padded operators
    b += (K / cfg->gemm_ne + 2) * size_t(cfg->gemm_kx) * cfg->gemm_ne * 4 + KD * size_t(cfg->gemm_mp2) * 4;
  return b;
}

void Server::fail_request(const std::shared_ptr<Request>& r, int code, const std::string& msg) {
  std::lock_guard<std::mutex> lock(mu);
  r->status = kFailed;
  r->error = code;
  r->message = msg;
  r->t_done = now_s();
}

bool Server::admit_one(std::shared_ptr<Request> r) {
  const dgk::KernelCfg* cfg = nullptr;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(r->model, r->N);
    auto it = cfg_of.find(key);
    if (it != cfg_of.end()) {
      cfg = it->second;
    } else {
      cfg = dg::select_variant(r->model, r->N, 0, device, DG_FP32);
      if (!cfg || !cfg->fn_batched) cfg = dgk::kernel_cfg(r->model, r->N);
      cfg_of[key] = cfg;
    }
  }
  const size_t need = estimate_bytes(*r, cfg);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return false;
  bool nothing_admitted;
  size_t admitted_bytes;
  {
    std::lock_guard<std::mutex> lock(mu);
    nothing_admitted = admitted == 0;
    admitted_bytes = active_bytes;
  }
  const bool fits_mem = free_b > kReserve && free_b - kReserve >= need;
  const bool fits_budget = budget == 0 || admitted_bytes + need <= budget;
  if (!fits_mem || !fits_budget) {
    if (nothing_admitted) {  // can never fit: refuse instead of waiting forever
      std::lock_guard<std::mutex> lock(mu);
      if (queue.empty() || queue.front() != r) return true;  // cancelled meanwhile
      queue.pop_front();
      r->status = kFailed;
      r->error = DG_ENOMEM;
      r->message = "request does not fit in device memory or the server budget";
      r->t_done = now_s();
      return true;
    }
    return false;
  }
  {
    std::lock_guard<std::mutex> lock(mu);
    if (queue.empty() || queue.front() != r) return true;  // cancelled meanwhile
    queue.pop_front();
    if (r->cancel) {
      r->status = kCancelled;
      r->t_done = now_s();
      return true;
    }
    r->status = kRunning;
  }
  dg_mesh m{int64_t(r->verts.size() / 3), int64_t(r->tets.size() / 4), r->verts.data(), r->tets.data()};
  dg_opts o = r->opts;
  o.stream = prep_stream;
  o.block_elems = 0;
  dg_handle* h = nullptr;
  int rc = dg_setup(&m, r->coeffs.data(), r->N, r->model, &o, &h);
  if (rc == DG_OK) {
    h->cfg = cfg;  // the group's batched variant
    rc = h->ensure_split(cfg);
  }
  if (rc == DG_OK && !r->q0.empty()) rc = dg_set_state(h, r->q0.data(), nullptr, nullptr, 0, 0);
  if (rc == DG_OK && r->has_src) rc = dg_set_source(h, r->xs, r->dir, r->amp.data(), int64_t(r->amp.size()));
  for (size_t s = 0; rc == DG_OK && s < r->ex_xyz.size() / 3; ++s)
    rc = dg_add_source(h, &r->ex_xyz[3 * s], &r->ex_dir[3 * s], &r->ex_amp[s * r->ex_namp], r->ex_namp);
  auto a = std::make_unique<Active>();
  if (rc == DG_OK && h->src_elem >= 0) {
    std::vector<float> af(r->amp.begin(), r->amp.end());
    if (cudaMalloc(&a->d_amp, af.size() * 4) != cudaSuccess ||
        cudaMemcpyAsync(a->d_amp, af.data(), af.size() * 4, cudaMemcpyHostToDevice, prep_stream) != cudaSuccess ||
        cudaStreamSynchronize(prep_stream) != cudaSuccess)
      rc = fail(DG_ECUDA, "source amplitudes");
  }
  if (rc != DG_OK) {
    fail_request(r, rc, dg_last_error());
    if (h) dg_destroy(h);
    if (a->d_amp) cudaFree(a->d_amp);
    return true;
  }
  a->req = r;
  a->h = h;
  a->steps_left = r->nsteps;
  {
    std::lock_guard<std::mutex> lock(mu);
    active_bytes += h->device_bytes + h->split_bytes;
    ++admitted;
    ready.push_back(std::move(a));
  }
  return true;
}

// Tick thread, at a chunk boundary: ready solves join their (model, N) group.
void Server::activate_ready() {
  std::vector<std::unique_ptr<Active>> got;
  {
    std::lock_guard<std::mutex> lock(mu);
    got.swap(ready);
  }
  for (auto& a : got) {
    a->h->stream = stream;
    Group& g = groups[{a->req->model, a->req->N}];
    g.model = a->req->model;
    g.N = a->req->N;
    if (!g.cfg) g.cfg = a->h->cfg;
    g.members.push_back(a.get());
    active.push_back(std::move(a));
    dirty = true;
  }
}

// Set-up thread: admission and host/device set-up of queued requests.
void Server::prep_loop() {
  cudaSetDevice(device);
  while (true) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lock(mu);
      if (stop) break;
      if (queue.empty() || admitted >= max_batch) {
        cv.wait_for(lock, std::chrono::milliseconds(5));
        continue;
      }
      r = queue.front();
    }
    if (!admit_one(r)) {  // does not fit yet: wait for a solve to finish
      std::unique_lock<std::mutex> lock(mu);
      cv.wait_for(lock, std::chrono::milliseconds(5));
    }
    cv.notify_all();
  }
}

// Launch arguments of a group's batched step (tables built by rebuild).
static dgk::BatchArgs batch_args(const Group& g, int* d_err) {
  dgk::BatchArgs b{};
  b.solves = g.d_solves;
  b.block_start = g.d_block_start;
  b.block_solve = g.d_block_solve;
  b.nsolves = int(g.members.size());
  b.total_blocks = g.total_blocks;
  b.ops = g.members[0]->h->d_ops;
  b.ftab = g.members[0]->h->d_ftab;
  b.err = d_err;
  b.ops2 = g.members[0]->h->d_ops2;
  b.tile_start = g.d_tile_start;
  b.tile_solve = g.d_tile_solve;
  b.total_tiles = g.total_tiles;
  return b;
}

// Device-side solve tables and the tick graph for the current active set.
int Server::rebuild() {
  if (graph) {
    cudaGraphExecDestroy(graph);
    graph = nullptr;
  }
  for (auto& kv : groups) {
    Group& g = kv.second;
    const int n = int(g.members.size());
    if (n == 0) continue;
    if (n > g.capacity) {
      if (g.d_solves) cudaFree(g.d_solves);
      if (g.d_block_start) cudaFree(g.d_block_start);
      if (g.d_tile_start) cudaFree(g.d_tile_start);
      g.capacity = std::max(n, 8);
      if (cudaMalloc(&g.d_solves, sizeof(dgk::SolveDev) * g.capacity) != cudaSuccess ||
          cudaMalloc(&g.d_block_start, sizeof(int) * (g.capacity + 1)) != cudaSuccess ||
          cudaMalloc(&g.d_tile_start, sizeof(int) * (g.capacity + 1)) != cudaSuccess)
        return fail(DG_ENOMEM, "server tables");
    }
    std::vector<dgk::SolveDev> sd(n);
    g.has_xs = false;
    std::vector<int> bs(n + 1, 0), ts(n + 1, 0);
    std::vector<int> bsolve, tsolve;
    for (int i = 0; i < n; ++i) {
      const Active* a = g.members[i];
      const dg_handle* h = a->h;
      dgk::SolveDev& d = sd[i];
      std::memset(&d, 0, sizeof(d));
      d.q[0] = h->d_q[0];
      d.q[1] = h->d_q[1];
      d.r[0] = h->d_r[0];
      d.r[1] = h->d_r[1];
      d.rec = h->d_geo;
      d.nbr = reinterpret_cast<const int4*>(h->d_nbr);
      d.srcvec = h->src_elem >= 0 ? h->d_src : nullptr;
      d.amp = a->d_amp;
      d.step = h->step;
      d.namp = int(a->req->amp.size());
      d.src_elem = h->src_elem;
      d.K = int(h->K);
      d.flux = h->opts.flux;
      d.bc = (h->model == DG_ELASTIC && h->opts.bc == DG_BC_RIGID) ? 1 : 0;
      d.dt = float(h->opts.dt);
      d.have = h->have;
      d.qcur = h->qcur;
      d.r1slot = h->r1slot;
      d.steps_left = a->steps_left;
      d.xg = h->d_x;
      d.xs = h->xs;
      g.has_xs = g.has_xs || h->xs.n > 0;
      bs[i + 1] = bs[i] + int((h->K + g.cfg->EB - 1) / g.cfg->EB);
      bsolve.insert(bsolve.end(), size_t(bs[i + 1] - bs[i]), i);
      ts[i + 1] = ts[i] + (g.cfg->split ? g.cfg->gemm_mtiles * int((h->K + g.cfg->gemm_ne - 1) / g.cfg->gemm_ne) : 0);
      tsolve.insert(tsolve.end(), size_t(ts[i + 1] - ts[i]), i);
    }
    g.total_blocks = bs[n];
    g.total_tiles = ts[n];
    if (int(tsolve.size()) > g.tile_capacity) {
      if (g.d_tile_solve) cudaFree(g.d_tile_solve);
      g.tile_capacity = int(tsolve.size()) * 2;
      if (cudaMalloc(&g.d_tile_solve, sizeof(int) * g.tile_capacity) != cudaSuccess)
        return fail(DG_ENOMEM, "server tile table");
    }
    if (!tsolve.empty() && cudaMemcpyAsync(g.d_tile_solve, tsolve.data(), sizeof(int) * tsolve.size(),
                                           cudaMemcpyHostToDevice, stream) != cudaSuccess)
      return fail(DG_ECUDA, "server tile table upload");
    if (cudaMemcpyAsync(g.d_tile_start, ts.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, stream) !=
        cudaSuccess)
      return fail(DG_ECUDA, "server tile table upload");
    if (int(bsolve.size()) > g.block_capacity) {
      if (g.d_block_solve) cudaFree(g.d_block_solve);
      g.block_capacity = int(bsolve.size()) * 2;
      if (cudaMalloc(&g.d_block_solve, sizeof(int) * g.block_capacity) != cudaSuccess)
        return fail(DG_ENOMEM, "server block table");
    }
    if (cudaMemcpyAsync(g.d_block_solve, bsolve.data(), sizeof(int) * bsolve.size(), cudaMemcpyHostToDevice,
                        stream) != cudaSuccess)
      return fail(DG_ECUDA, "server block table upload");
    if (cudaMemcpyAsync(g.d_solves, sd.data(), sizeof(dgk::SolveDev) * n, cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(g.d_block_start, bs.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess)
      return fail(DG_ECUDA, "server tables upload");
  }
  if (cudaStreamSynchronize(stream) != cudaSuccess) return fail(DG_ECUDA, "server sync");
  // warm the kernels outside the capture (shared-memory opt-in, occupancy)
  for (auto& kv : groups) {
    Group& g = kv.second;
    if (g.members.empty()) continue;
    dgk::BatchArgs b = batch_args(g, d_err);
    b.nsolves = 0;
    b.total_blocks = 0;
    b.total_tiles = 0;
    if (dgk::launch_step_batched(g.cfg, b, stream) != cudaSuccess) return fail(DG_ECUDA, "batched warm-up");
  }
  // side streams and events for the groups (created once, kept)
  int ngroups = 0;
  for (auto& kv : groups)
    if (!kv.second.members.empty()) ++ngroups;
  if (!fork && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(DG_ECUDA, "server fork event");
  while (int(side.size()) < ngroups) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
      return fail(DG_ECUDA, "server side stream");
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamDestroy(st);
      return fail(DG_ECUDA, "server join event");
    }
    side.push_back(st);
    join.push_back(ev);
  }
  // the tick: fork, every group's step kernels on its own stream, join, then
  // the advance kernels (they change the state the step kernels read)
  cudaGraph_t gr = nullptr;
  if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(DG_ECUDA, "graph capture");
  cudaError_t e = cudaEventRecord(fork, stream);
  int gi = 0;
  for (auto& kv : groups) {
    Group& g = kv.second;
    const int n = int(g.members.size());
    if (n == 0) continue;
    cudaStream_t st = side[gi];
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, fork, 0);
    dgk::BatchArgs b = batch_args(g, d_err);
    if (e == cudaSuccess) e = dgk::launch_step_batched(g.cfg, b, st);
    if (e == cudaSuccess && g.has_xs)
      e = dgk::launch_xsrc_batched(b, dg::num_fields(g.model) * dg::num_nodes(g.N), st);
    if (e == cudaSuccess) e = cudaEventRecord(join[gi], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, join[gi], 0);
    ++gi;
  }
  for (auto& kv : groups) {
    Group& g = kv.second;
    if (!g.members.empty() && e == cudaSuccess) e = dgk::launch_advance(g.d_solves, int(g.members.size()), stream);
  }
  cudaError_t e2 = cudaStreamEndCapture(stream, &gr);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    return fail(DG_ECUDA, "tick capture failed");
  }
  e = cudaGraphInstantiate(&graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return fail(DG_ECUDA, "graph instantiate");
  dirty = false;
  return DG_OK;
}

void Server::retire(Active* a, int status) {
  dg_handle* h = a->h;
  auto r = a->req;
  std::vector<float> out;
  if (status == kDone) {
    out.resize(size_t(h->K) * h->Nf * h->Np);
    if (cudaMemcpyAsync(out.data(), h->d_q[h->qcur], out.size() * 4, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      status = kFailed;
  }
  {
    std::lock_guard<std::mutex> lock(mu);
    active_bytes -= std::min(active_bytes, h->device_bytes + h->split_bytes);
    --admitted;
  }
  cv.notify_all();
  dg_destroy(h);
  if (a->d_amp) cudaFree(a->d_amp);
  {
    std::lock_guard<std::mutex> lock(mu);
    r->status = status;
    if (status == kFailed) {
      r->error = DG_ECUDA;
      r->message = "result copy failed";
    }
    r->q_out.swap(out);
    r->t_done = now_s();
  }
  for (auto& kv : groups) {
    auto& m = kv.second.members;
    m.erase(std::remove(m.begin(), m.end(), a), m.end());
  }
  active.erase(std::remove_if(active.begin(), active.end(), [a](const std::unique_ptr<Active>& p) { return p.get() == a; }),
               active.end());
  dirty = true;
}

void Server::loop() {
  cudaSetDevice(device);
  while (true) {
    {
      std::unique_lock<std::mutex> lock(mu);
      if (stop) break;
      if (ready.empty() && active.empty()) {
        cv.wait_for(lock, std::chrono::milliseconds(2));
        continue;
      }
    }
    // continuous batching: solves set up meanwhile join at this chunk boundary
    activate_ready();
    // cancellations of running solves
    std::vector<Active*> cancelled;
    {
      std::lock_guard<std::mutex> lock(mu);
      for (auto& a : active)
        if (a->req->cancel) cancelled.push_back(a.get());
    }
    for (Active* a : cancelled) retire(a, kCancelled);
    if (active.empty()) continue;
    if (dirty && rebuild() != DG_OK) {
      std::string msg = dg_last_error();
      std::vector<Active*> all_a;
      for (auto& a : active) all_a.push_back(a.get());
      for (Active* a : all_a) {
        fail_request(a->req, DG_ECUDA, msg);
        dg_destroy(a->h);
        if (a->d_amp) cudaFree(a->d_amp);
      }
      {
        std::lock_guard<std::mutex> lock(mu);
        admitted -= int(all_a.size());
        active_bytes = 0;
      }
      active.clear();
      for (auto& kv : groups) kv.second.members.clear();
      dirty = true;
      continue;
    }
    int chunk = kMaxChunk;
    for (auto& a : active) chunk = std::min(chunk, a->steps_left);
    bool ok = true;
    for (int t = 0; t < chunk && ok; ++t) ok = cudaGraphLaunch(graph, stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(stream) == cudaSuccess;
    int err = 0;
    if (ok) ok = cudaMemcpy(&err, d_err, 4, cudaMemcpyDeviceToHost) == cudaSuccess && err == 0;
    int64_t nlaunch = 0;
    for (auto& kv : groups)
      if (!kv.second.members.empty()) nlaunch += 2;
    launches += nlaunch * chunk;
    // mirror the device-side step state on the host handles
    for (auto& a : active) {
      dg_handle* h = a->h;
      if (chunk & 1) {
        h->qcur ^= 1;
        h->r1slot ^= 1;
      }
      h->step += chunk;
      h->have = std::min(h->have + chunk, 2);
      a->steps_left -= chunk;
    }
    std::vector<Active*> finished;
    for (auto& a : active)
      if (!ok || a->steps_left <= 0) finished.push_back(a.get());
    for (Active* a : finished) retire(a, ok ? kDone : kFailed);
  }
}

Server::~Server() {
  for (auto* lst : {&active, &ready})
    for (auto& a : *lst) {
      dg_destroy(a->h);
      if (a->d_amp) cudaFree(a->d_amp);
    }
  for (auto& kv : groups) {
    if (kv.second.d_solves) cudaFree(kv.second.d_solves);
    if (kv.second.d_block_start) cudaFree(kv.second.d_block_start);
    if (kv.second.d_block_solve) cudaFree(kv.second.d_block_solve);
    if (kv.second.d_tile_start) cudaFree(kv.second.d_tile_start);
    if (kv.second.d_tile_solve) cudaFree(kv.second.d_tile_solve);
  }
  if (graph) cudaGraphExecDestroy(graph);
  if (d_err) cudaFree(d_err);
  for (auto st : side) cudaStreamDestroy(st);
  for (auto ev : join) cudaEventDestroy(ev);
  if (fork) cudaEventDestroy(fork);
  if (stream) cudaStreamDestroy(stream);
  if (prep_stream) cudaStreamDestroy(prep_stream);
}

}  // namespace dg

struct dg_server : dg::Server {};

using dg::fail;

extern "C" {

int dg_server_create(size_t hbm_budget_bytes, int max_batch, dg_server** out) {
  if (!out) return fail(DG_EINVAL, "out is NULL");
  *out = nullptr;
  auto* s = new (std::nothrow) dg_server();
  if (!s) return fail(DG_ENOMEM, "host allocation failed");
  s->budget = hbm_budget_bytes;
  s->max_batch = max_batch > 0 ? max_batch : 64;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->prep_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&s->d_err, 4) != cudaSuccess || cudaMemset(s->d_err, 0, 4) != cudaSuccess) {
    delete s;
    return fail(DG_ECUDA, "server stream / error word");
  }
  s->thr = std::thread([s] { s->loop(); });
  s->prep_thr = std::thread([s] { s->prep_loop(); });
  *out = s;
  return DG_OK;
}

int dg_submit(dg_server* s, const dg_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket || !req->mesh || !req->coeffs) return fail(DG_EINVAL, "NULL argument");
  if (req->N < 1 || req->N > 8) return fail(DG_EINVAL, "polynomial degree N must be in 1..8");
  if (req->model != DG_ACOUSTIC && req->model != DG_ELASTIC) return fail(DG_EINVAL, "unknown model");
  if (req->nsteps < 0) return fail(DG_EINVAL, "negative step count");
  if (req->nsrc < 0 || req->nsrc > DG_MAX_SOURCES) return fail(DG_EINVAL, "source count outside 0..DG_MAX_SOURCES");
  if (!(req->opts.dt > 0)) return fail(DG_EINVAL, "dt must be positive");
  if (req->opts.precision != DG_FP32 || req->opts.strategy != DG_STRATEGY_FUSED)
    return fail(DG_EINVAL, "served solves run the batched FP32 fused kernels: precision must be DG_FP32 and "
                           "strategy DG_STRATEGY_FUSED");
  const dg_mesh* m = req->mesh;
  if (!m->verts || !m->tets || m->ntets <= 0 || m->nverts < 4) return fail(DG_EINVAL, "empty mesh");
  auto r = std::make_shared<dg::Request>();
  r->verts.assign(m->verts, m->verts + 3 * m->nverts);
  r->tets.assign(m->tets, m->tets + 4 * m->ntets);
  const int nc = req->model == DG_ACOUSTIC ? 2 : 3;
  r->coeffs.assign(req->coeffs, req->coeffs + nc * m->ntets);
  r->N = req->N;
  r->model = req->model;
  r->nsteps = req->nsteps;
  r->opts = req->opts;
  if (req->q0) r->q0.assign(req->q0, req->q0 + size_t(m->ntets) * dg::num_fields(req->model) * dg::num_nodes(req->N));
  if (req->src_xyz && req->src_amp && req->src_namp > 0) {
    const int ns = req->nsrc > 0 ? req->nsrc : 1;
    r->has_src = true;
    std::memcpy(r->xs, req->src_xyz, sizeof(r->xs));
    if (req->src_dir) std::memcpy(r->dir, req->src_dir, sizeof(r->dir));
    r->amp.assign(req->src_amp, req->src_amp + req->src_namp);
    if (ns > 1) {
      r->ex_xyz.assign(req->src_xyz + 3, req->src_xyz + 3 * size_t(ns));
      if (req->src_dir) r->ex_dir.assign(req->src_dir + 3, req->src_dir + 3 * size_t(ns));
      else
        for (int j = 1; j < ns; ++j) r->ex_dir.insert(r->ex_dir.end(), {0.0, 0.0, 1.0});
      r->ex_amp.assign(req->src_amp + req->src_namp, req->src_amp + size_t(ns) * req->src_namp);
      r->ex_namp = req->src_namp;
    }
  }
  r->t_submit = dg::now_s();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->queue.push_back(r);
  }
  s->cv.notify_one();
  *ticket = r->id;
  return DG_OK;
}

int dg_poll(dg_server* s, uint64_t ticket, float* q_out, double* latency_s) {
  if (!s) return fail(DG_EINVAL, "NULL server");
  std::shared_ptr<dg::Request> r;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(DG_ENOENT, "unknown ticket");
    r = it->second;
    if (r->status == dg::kQueued || r->status == dg::kRunning) return DG_EAGAIN;
    s->all.erase(it);
  }
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  if (r->status == dg::kCancelled) return fail(DG_ECANCELED, "request cancelled");
  if (r->status == dg::kFailed) return fail(r->error, r->message);
  if (q_out) std::memcpy(q_out, r->q_out.data(), r->q_out.size() * 4);
  return DG_OK;
}

int dg_cancel(dg_server* s, uint64_t ticket) {
  if (!s) return fail(DG_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(DG_ENOENT, "unknown ticket");
  it->second->cancel = true;
  if (it->second->status == dg::kQueued) {
    auto& q = s->queue;
    q.erase(std::remove(q.begin(), q.end(), it->second), q.end());
    it->second->status = dg::kCancelled;
    it->second->t_done = dg::now_s();
  }
  return DG_OK;
}

int dg_server_stats(dg_server* s, int64_t* queued, int64_t* running, int64_t* done, int64_t* launches) {
  if (!s) return fail(DG_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  int64_t q = 0, r = 0, d = 0;
  for (auto& kv : s->all) {
    const int st = kv.second->status;
    if (st == dg::kQueued) ++q;
    else if (st == dg::kRunning) ++r;
    else ++d;
  }
  if (queued) *queued = q;
  if (running) *running = r;
  if (done) *done = d;
  if (launches) *launches = s->launches.load();
  return DG_OK;
}

void dg_server_destroy(dg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->thr.joinable()) s->thr.join();
  if (s->prep_thr.joinable()) s->prep_thr.join();
  delete s;
}

}  // extern "C"
