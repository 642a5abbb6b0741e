/*
 * dg.h -- C ABI of the GB300 nodal discontinuous Galerkin library (libdg).
 *
 * The library evaluates the semi-discrete right-hand side of the nodal DG
 * scheme of Modave, St-Cyr & Warburton (arXiv:1602.07997) on straight-sided
 * tetrahedra, for the acoustic pressure-velocity system (4 fields: p, vx,
 * vy, vz) and the isotropic elastic velocity-stress system (9 fields: vx,
 * vy, vz, sxx, syy, szz, sxy, sxz, syz), and advances it with the
 * third-order Adams-Bashforth scheme:
 *
 *   physics and upwind penalty terms ............ Section 2.1
 *   local RHS  r_k = sum_ij g^vol D_j f + sum_f g^sur L_f p ... Section 2.2, Eq. dgLocalRhs
 *   AB3 update q^{m+1} = q^m + dt sum_s a_s r^{m-s+1} ...... Section 2.2, Eq. updateScheme
 *   acoustic kernel form of the RHS .............. Section 3.2, Eqs. dgRhsAcou1-2
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Polynomial degree N in 1..8; Np = (N+1)(N+2)(N+3)/6 nodes per element,
 *    Nfp = (N+1)(N+2)/2 nodes per face, Nf = 4 (acoustic) or 9 (elastic).
 *  - Nodal arrays use the layout [K][Nf][Np] in float32, node index fastest
 *    (the one-node-per-thread granularity of Table 1).  Node n of an element
 *    is the n-th point of the warp-and-blend set (blend parameter 0) in the
 *    order of the equispaced lattice (i along r fastest, then s, then t),
 *    reference tetrahedron v1=(-1,-1,-1), v2=(1,-1,-1), v3=(-1,1,-1),
 *    v4=(-1,-1,1); dg_node_coords returns the physical positions.
 *  - Meshes: vertex coordinates double [nverts][3]; tetrahedra int64
 *    [ntets][4] (0-based vertex indices), positively oriented
 *    (det[x2-x1, x3-x1, x4-x1] > 0).  The mesh must be conforming (each
 *    face shared by at most two tetrahedra); unshared faces are outer
 *    boundary faces.
 *  - Coefficients, constant per element: acoustic double [K][2] = (rho, c);
 *    elastic double [K][3] = (lambda, mu, rho).
 *  - Ownership: every pointer argument is borrowed for the duration of the
 *    call only; dg_setup copies the mesh, coefficients and operators it
 *    needs.  Device state (fields, AB3 history, geometry) belongs to the
 *    handle and is freed by dg_destroy.  Output buffers are allocated by the
 *    caller.  `on_device` = 1 means the pointer is a CUDA device pointer on
 *    the handle's device (e.g. torch.Tensor.data_ptr()), 0 means host memory.
 *  - Asynchrony: kernels and copies are issued on the CUDA stream given in
 *    dg_opts.stream (NULL = the legacy default stream).  Host outputs are
 *    complete when the call returns; device outputs are complete in stream
 *    order.  dg_sync waits for the stream and reports device-side errors.
 *  - Errors: functions return DG_OK (0) or a negative code below; a
 *    thread-local message is available from dg_last_error().  No function
 *    aborts the process and no kernel traps.
 */
#ifndef DG_H
#define DG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DG_OK = 0,
  DG_EINVAL = -1,      /* bad argument, N outside 1..8, bad mesh (inverted or
                          degenerate tet, non-conforming face, index out of range) */
  DG_ENOMEM = -2,      /* device or host allocation failed, or over the budget  */
  DG_ECUDA = -3,       /* a CUDA runtime call failed (message has the CUDA error) */
  DG_ENONFINITE = -4,  /* a NaN/Inf was found in the state                        */
  DG_ETIMEOUT = -5,    /* a bounded device-side wait expired                      */
  DG_EAGAIN = -6,      /* dg_poll: the request is not finished yet                */
  DG_ECANCELED = -7,   /* dg_poll: the request was cancelled                      */
  DG_ENOENT = -8       /* dg_poll / dg_cancel: unknown ticket                     */
};

enum { DG_ACOUSTIC = 0, DG_ELASTIC = 1 };
enum { DG_FLUX_UPWIND = 0, DG_FLUX_CENTERED = 1 };
/* outer boundary: DEFAULT = rigid wall (acoustic) / traction-free (elastic).
 * Mirror ghost states: acoustic rigid p+ = p-, v+ = v- - 2 (v-.n) n;
 * elastic free v+ = v-, sigma+ = -sigma-; elastic rigid v+ = -v-, sigma+ = sigma-. */
enum { DG_BC_DEFAULT = 0, DG_BC_RIGID = 1, DG_BC_FREE = 2 };
/* Arithmetic of the operator contractions (D_r, D_s, D_t and LIFT products,
 * Section 3.2); flux, geometric combination and AB3 are always float32.
 *   DG_FP32   FP32 FMAs on the CUDA cores.
 *   DG_BF16X3 tensor cores (tcgen05, FP32 accumulation in TMEM); every operand
 *             x is split into two BF16 pieces x0 + x1 and the three products
 *             x0 y0 + x0 y1 + x1 y0 are summed: relative error of each product
 *             about 2^-16 (the RHS of smooth fields at N >= 4 can miss 1e-5).
 *   DG_BF16X6 tensor cores with three BF16 pieces per operand and the six
 *             products of pieces (a, b) with a + b <= 2: float32-level error.
 * The tensor-core modes run the split step (front half on the CUDA cores
 * writing the contraction inputs to a device buffer, then the contraction and
 * the AB3 epilogue on the tensor cores) at every N. */
enum { DG_FP32 = 0, DG_BF16X3 = 1, DG_BF16X6 = 2, DG_TF32 = 3 };

/* Step strategy (the paper's Section 3 compares several ways of organising
 * the same computation):
 *   DG_STRATEGY_FUSED   this library's step: one fused kernel per step (or
 *                       the split step at high N / in the tensor-core modes);
 *                       every precision mode except DG_TF32.
 *   DG_STRATEGY_LIBRARY the library route of Section 3.3: the fused kernel's
 *                       front half writes the operator-product inputs, cuBLAS
 *                       strided-batched SGEMMs compute the D_r/D_s/D_t and LIFT
 *                       products (8 GEMMs per step acoustic, 27 elastic: the
 *                       surface streams are lifted face by face), a
 *                       streaming kernel does the geometric combination and
 *                       AB3.  Precision DG_FP32 (SGEMM) or DG_TF32 (cuBLAS TF32
 *                       tensor-core math; its error is far above 1e-5).
 *   DG_STRATEGY_PLAIN   the one-node-per-thread multi-kernel route of Section
 *                       3.2: volume, surface and AB3 update kernels with the
 *                       partial RHS in device memory between them; DG_FP32.
 * Autotuning and kernel variants apply to DG_STRATEGY_FUSED only. */
enum { DG_STRATEGY_FUSED = 0, DG_STRATEGY_LIBRARY = 1, DG_STRATEGY_PLAIN = 2 };

typedef struct {
  int64_t nverts;
  int64_t ntets;
  const double *verts;  /* [nverts][3] */
  const int64_t *tets;  /* [ntets][4]  */
} dg_mesh;

typedef struct {
  int flux;         /* DG_FLUX_*                                         */
  int bc;           /* DG_BC_*                                           */
  int precision;    /* DG_FP32, DG_BF16X3, DG_BF16X6 (fused strategy) or
                       DG_TF32 (library strategy)                        */
  int block_elems;  /* elements per CTA of a compiled variant; 0 = the autotuned
                       choice for (model, N) if any, else the default variant */
  double dt;        /* time step used by dg_step (may be changed by dg_set_dt) */
  void *stream;     /* cudaStream_t; NULL = legacy default stream        */
  int strategy;     /* DG_STRATEGY_* (0 = fused)                         */
} dg_opts;

typedef struct dg_handle dg_handle;

/* Build a solver for one mesh (Section 2.2): reference operators (warp-and-
 * blend nodes, orthonormal-basis Vandermonde route: D_r = V_r V^{-1},
 * M^{-1} = V V^T, LIFT = M^{-1} [E_1..E_4]), per-element geometric factors
 * g^vol_{ij} = dr_j/dx_i, face normals and g^sur = sJ/J, face connectivity,
 * and the device state.  The state starts at q = 0 with an empty AB3 history.
 * Returns DG_EINVAL for N outside 1..8, a negative or zero Jacobian, a face
 * shared by more than two tetrahedra, or a vertex index out of range.      */
int dg_setup(const dg_mesh *mesh, const double *coeffs, int N, int model,
             const dg_opts *opts, dg_handle **out);
void dg_destroy(dg_handle *h);

/* Sizes: number of elements, nodes per element, nodes per face, fields.     */
int dg_info(const dg_handle *h, int64_t *K, int *Np, int *Nfp, int *Nf);

/* State transfers take `on_device` = 0 (host memory; the call returns when
 * its copies are complete), 1 (device memory on the handle's device) or
 * DG_HOST_ASYNC = 2 (page-locked host memory, e.g. cudaHostAlloc'd or a
 * pinned torch tensor: the copies are ordered on the handle's stream and
 * complete at the next dg_sync or any later synchronising call; the caller
 * must not touch the buffer before then; memory that is not page-locked is
 * refused with DG_EINVAL).  Several handles on separate streams then
 * overlap their transfers with one another's kernels.                      */
enum { DG_HOST_ASYNC = 2 };

/* Replace the state.  q [K][Nf][Np].  r1 = r^{m-1} and r2 = r^{m-2} (same
 * layout) are either both NULL -- the next steps then start AB3 with a
 * forward-Euler step and an AB2 step -- or both given (full AB3 history).
 * `step` is the time-step index m of q (it indexes source amplitudes).     */
int dg_set_state(dg_handle *h, const float *q, const float *r1, const float *r2,
                 int64_t step, int on_device);
/* Read the state; r1 / r2 may be NULL.  *step / *history (0, 1 or 2 stored
 * RHS levels) may be NULL.                                                  */
int dg_get_state(dg_handle *h, float *q, float *r1, float *r2, int64_t *step,
                 int *history, int on_device);

/* r_out [K][Nf][Np] = r(q^m, t_m): volume term + lifted penalty terms
 * (Eq. dgLocalRhs) at the current state, plus the source term of step m;
 * the state is not changed.                                                 */
int dg_rhs(dg_handle *h, float *r_out, int on_device);

/* Advance nsteps AB3 steps (Eq. updateScheme) with the handle's dt; each step
 * is one fused launch (RHS + update), or two for the split step (front half,
 * then the operator GEMM with the update), plus one small launch when the
 * handle has more than one point source and one when it has receivers.
 * Asynchronous on the handle's stream.                                      */
int dg_step(dg_handle *h, int nsteps);
int dg_set_dt(dg_handle *h, double dt);
/* Autotuner: time every compiled variant of the step kernel (elements per
 * CTA and threads per CTA) for this handle's (model, N) on its own mesh,
 * `reps` launches each, on scratch copies of the state (the handle's state
 * and history are untouched), keep the fastest for this handle and for
 * handles created later in the process on the same device, model and N.
 * block_elems / ms_per_step (may be NULL) receive the choice and its time;
 * variant_ms (NULL or [variants]) receives every variant's time per step.
 * Allocates and frees scratch device memory of 4 state sizes; synchronous. */
int dg_autotune(dg_handle *h, int reps, int *block_elems, double *ms_per_step, double *variant_ms);
/* Autotuner choices across processes (the paper has no counterpart; its
 * kernels were tuned by hand, Section 4).  dg_tune_save writes every choice
 * of this process (dg_autotune, dg_set_variant) to a text file, one line per
 * (device, model, N, precision): the device's name and compute capability,
 * the variant index and the variant's shape (elements per block, threads,
 * split form, GEMM threads).  dg_tune_load makes the file's choices the
 * process's for the current device -- lines of another device name or
 * compute capability, or naming a variant this build compiles differently,
 * are skipped -- so handles created afterwards start with them (as after
 * dg_autotune); *applied (may be NULL) = lines taken.  dg_tune_clear
 * forgets every choice of the process (handles created afterwards take
 * their default variant).  DG_EINVAL: NULL path, unreadable or unwritable
 * file, or a file that is not such a cache or has a malformed line (nothing
 * is applied then); DG_ECUDA: a device query failed.                       */
int dg_tune_save(const char *path);
int dg_tune_load(const char *path, int *applied);
int dg_tune_clear(void);

/* Launch configuration in use: elements per CTA, threads per CTA, dynamic
 * shared memory per CTA, number of compiled variants (of the handle's
 * precision mode), elements per thread tile, and the step's form in *split:
 * 0 fused, 1 split with the FP32 CUDA-core GEMM, 2 split with the tensor-core
 * GEMM (the operator products run as a separate GEMM over 16-64-element
 * column tiles; needs an extra device buffer, allocated on first use: per
 * element (4 Np + 8 Nfp + 12) floats for the acoustic FP32 split step and
 * (12 Np + 24 Nfp + 12) for the elastic one -- volume inputs, surface
 * streams, face normals -- while the tensor-core form keeps every penalty
 * field: 2 or 3 BF16 pieces of (4 Np + 16 Nfp) or (12 Np + 36 Nfp) values,
 * each part rounded up to 16), and the index of the variant in use (as taken
 * by dg_set_variant).  Pointers may be NULL.                                */
int dg_kernel_info(const dg_handle *h, int *block_elems, int *threads, int64_t *smem_bytes,
                   int *variants, int *tile_elems, int *split, int *variant);
/* Select compiled variant `index` (0 <= index < variants of the handle's
 * precision mode) for this handle and, like dg_autotune, for handles created
 * later in the process on the same device, model, N and precision (servers
 * fix their variant per (model, N) at the first admission).  DG_EINVAL for
 * an index out of range.                                                    */
int dg_set_variant(dg_handle *h, int index);

/* Receivers (seismogram sampling).  The paper samples no point values; the
 * method's nodal polynomial fixes them: the field at a point x in element k
 * is sum_i q_k[f][i] l_i(r(x)) with l_i the Lagrange basis of the element's
 * nodes (Section 2.2) and r(x) the reference coordinates of x.
 * dg_set_receivers places nrec receivers at xyz [nrec][3] (host, borrowed
 * for the call; each in the element whose smallest barycentric coordinate of
 * the point is largest, DG_EINVAL for a point outside the mesh) and clears
 * the recorded traces; nrec = 0 removes them.  After every step of dg_step
 * the fields at the receivers are recorded on the device (one sample =
 * [nrec][Nf] floats, the state q^{m+1} just computed).
 * dg_get_traces copies the samples recorded since dg_set_receivers into out
 * [nsamples][nrec][Nf] (host, or device memory if on_device; NULL to query
 * *nsamples only).  Samples are kept on the device; dg_step grows the buffer
 * as needed (DG_ENOMEM if it cannot).                                     */
int dg_set_receivers(dg_handle *h, const double *xyz, int nrec);
int dg_get_traces(dg_handle *h, float *out, int64_t *nsamples, int on_device);

/* The paper has no counterpart to this entry point.  Same result as
 * dg_rhs(h, r_out, 0) -- the RHS at the current state into the caller's host
 * buffer r_out [K][Nf][Np] -- but without allocating device memory: dg_rhs
 * stages the RHS in a device buffer it allocates per call, this function
 * stages it in a fixed 16 MiB array (4 Mi floats) that the library holds on
 * every device where a handle has been set up, until the process exits.  It
 * is meant for callers that cannot allocate device memory when they need the
 * RHS, e.g. an application whose device memory is already committed to
 * another allocator (a framework's caching allocator or a fixed memory
 * budget), where a fresh allocation could fail or force a device
 * synchronisation.
 *  - Set-up: dg_setup, with the handle's device current, looks up the
 *    array's device address (cudaGetSymbolAddress; the first lookup on a
 *    device loads the array there, 16 MiB) and does the first-use set-up of
 *    the kernels this call launches; it still allocates the handle's state
 *    once.  A call then allocates nothing, so the device's free memory is
 *    the same before and after it.  cudaDeviceReset ends the context that
 *    address belongs to, and with it every handle of that device.
 *  - K*Nf*Np must not exceed 4194304; larger meshes get DG_EINVAL (use
 *    dg_rhs).  The handle's device must be the current device.  The call
 *    synchronises the handle's stream.
 *  - Kernel: the fused FP32 step in RHS mode, whatever the handle's
 *    precision and strategy (the same RHS within FP32 rounding): the
 *    handle's own variant if it is the fused FP32 step, else the process's
 *    FP32 choice for (model, N) at dg_setup (autotuned or the default) if
 *    that is fused, else the first fused variant compiled for N.  A split
 *    variant is never used: it would need its input buffer, which is
 *    allocated on first use.
 *  - Every call shares the one array and leaves its contents behind; calls
 *    whose work overlaps on the GPU (other host threads, other handles on the
 *    same device) race on it and must be serialised by the caller.  Nothing
 *    in it needs clearing: the RHS kernel overwrites every value read back.  */
int dg_rhs_host_noalloc(dg_handle *h, float *r_out);

/* Measurement helper (the paper states its GPU's FP32 peak in Section 4.1;
 * this measures the current device's): FP32 fused multiply-add throughput in
 * TFLOP/s (one FMA = 2 flops).  Every thread of a grid that fills every SM
 * runs 8 independent FMA chains whose operands are kernel arguments; the
 * scalar FP32 FMA and the packed two-lane form (fma.rn.f32x2) are timed
 * separately, `reps` launches of about `target_ms` each after one sizing
 * launch, and the best launch of each form is returned (*scalar_tflops,
 * *packed_tflops; *ms_per_launch = the longer of the two best launches; any
 * pointer may be NULL).  Runs on `stream` (cudaStream_t, NULL = legacy
 * default stream) of the current device and synchronises it; allocates
 * nothing.  DG_EINVAL for reps < 1 or target_ms outside (0, 10000].        */
int dg_fp32_peak(void *stream, int reps, double target_ms, double *scalar_tflops,
                 double *packed_tflops, double *ms_per_launch);

/* Move the handle to another CUDA stream (cudaStream_t; NULL = legacy
 * default stream): the work already issued on its stream finishes first
 * (the call waits for it), later calls issue on the new one.               */
int dg_set_stream(dg_handle *h, void *stream);

/* Wait for the handle's stream and report what the kernels flagged since the
 * last report: DG_ETIMEOUT if a bounded device wait expired (the results of
 * those steps are not valid), else DG_ENONFINITE if a finite-state check
 * found a NaN or an infinity in q.  The flag is cleared when it is reported,
 * so the handle stays usable (e.g. dg_set_state and step again).           */
int dg_sync(dg_handle *h);

/* Failure detection (the paper's method has no counterpart; these guard its
 * time loop).
 * dg_set_finite_check: after every `every`-th step of dg_step (step index m
 * a multiple of `every`) a small kernel reads q^m and flags a NaN or an
 * infinity for dg_sync (DG_ENONFINITE); every = 0 turns it off.  Default
 * 100 (one extra read of q per 100 steps).  DG_EINVAL for every < 0.
 * dg_set_wait_limit: every bounded device wait of the handle's kernels (a
 * wait for a bulk copy or for the tensor cores) gives up after `cycles` SM
 * clock cycles and flags DG_ETIMEOUT for dg_sync; 0 = the default 2^31
 * (about a second).  A negative value makes the first wait of every CTA
 * give up at once without looking: a test hook that exercises the expiry
 * path, after which each CTA waits (with the default limit) for the copies
 * and products it has in flight and leaves.  Neither call launches work.  */
int dg_set_finite_check(dg_handle *h, int every);
int dg_set_wait_limit(dg_handle *h, int64_t cycles);

/* Kernels of this library the handle has launched so far (step kernels,
 * split-step GEMMs, source, receiver and finite-check kernels; the cuBLAS
 * GEMMs of DG_STRATEGY_LIBRARY are not counted).                           */
int dg_launch_count(const dg_handle *h, int64_t *launches);

/* Physical node coordinates, double [K][Np][3].                             */
int dg_node_coords(const dg_handle *h, double *xyz);

/* Point source at xs: at step m the RHS gets amp[m] M_k^{-1} l(xs) on p
 * (acoustic) or amp[m] (dir_i / rho_k) M_k^{-1} l(xs) on v_i (elastic), in
 * the tet whose smallest barycentric coordinate of xs is largest; amp[m] = 0
 * for m >= namp.  dg_set_source replaces every source of the handle by this
 * one (amp == NULL removes them all); dg_add_source adds one more (several
 * sources add their terms; DG_EINVAL past DG_MAX_SOURCES, or with amp ==
 * NULL).  Both copy their inputs (host pointers) and apply to dg_step,
 * dg_rhs and dg_rhs_host_noalloc with every strategy and precision; the
 * first source is added inside the step kernels, the others by one small
 * kernel after them.                                                        */
enum { DG_MAX_SOURCES = 64 };
int dg_set_source(dg_handle *h, const double xs[3], const double dir[3],
                  const double *amp, int64_t namp);
int dg_add_source(dg_handle *h, const double xs[3], const double dir[3],
                  const double *amp, int64_t namp);

/* dt = cfl * min_{k,f} 1 / (c_max,k Fscale_{k,f} ((N+1)(N+2)/2 + 2)), host
 * only; c_max = c (acoustic) or c_p (elastic).  cfl = 0.4 keeps the upwind
 * spectrum inside the AB3 stability region for N = 1..8.                   */
int dg_suggest_dt(const dg_mesh *mesh, const double *coeffs, int N, int model,
                  double cfl, double *dt);

/* Host-only reference element of degree N, double precision, for checking
 * the set-up: nodes [Np][3], Dr/Ds/Dt [Np][Np] (D[i][j] = dl_j/dr(x_i)),
 * LIFT [Np][4 Nfp] with columns in face-major order and, within a face, in
 * the order of fmask [4][Nfp] (the node index of each face node).  Any
 * pointer may be NULL.                                                      */
int dg_reference_element(int N, double *nodes, double *Dr, double *Ds, double *Dt,
                         double *LIFT, int *fmask);

/* Thread-local message of the last failing call on this thread.             */
const char *dg_last_error(void);

/* ----------------------------------------------------------------------------
 * Served solves.  A server owns a host thread and its CUDA streams.  Each
 * request is an independent time-domain solve (mesh, coefficients, N, model,
 * initial state, source, nsteps).  Requests are admitted while free device
 * memory (cudaMemGetInfo) minus a safety margin, and the optional budget,
 * cover their state; admitted solves of the same degree and model are
 * advanced together, one batched step per (model, N) class per time step
 * (one launch, or two for the split step; the classes' launches run
 * concurrently, each class on its own stream of the tick's CUDA graph, then
 * a small launch per class advances every solve's step counter and AB3
 * phase), and new requests join between steps (continuous batching).  A finished
 * solve's q is copied to host memory owned by the server until dg_poll
 * copies it out.
 * ------------------------------------------------------------------------ */
typedef struct dg_server dg_server;

typedef struct {
  const dg_mesh *mesh;
  const double *coeffs;
  int N;
  int model;
  dg_opts opts;          /* flux, bc, dt; precision must be DG_FP32 and
                            strategy DG_STRATEGY_FUSED (served solves run
                            the batched FP32 kernels, else DG_EINVAL);
                            block_elems and stream are ignored */
  const float *q0;       /* host [K][Nf][Np]; NULL = zero state              */
  const double *src_xyz; /* [nsrc][3]; NULL = no source                       */
  const double *src_dir; /* elastic only: [nsrc][3]; NULL = (0,0,1) for all   */
  const double *src_amp; /* [nsrc][src_namp] amplitudes per step              */
  int64_t src_namp;
  int nsteps;
  int nsrc;              /* point sources in the arrays above (as
                            dg_add_source); 0 = one when src_xyz is set,
                            at most DG_MAX_SOURCES                          */
} dg_request;

/* hbm_budget_bytes = 0: no budget beyond the free device memory.           */
int dg_server_create(size_t hbm_budget_bytes, int max_batch, dg_server **out);
int dg_submit(dg_server *s, const dg_request *req, uint64_t *ticket);
/* DG_OK and q_out filled (host, caller-allocated [K][Nf][Np]) when finished;
 * DG_EAGAIN while queued or running.  latency_s (may be NULL) = finish time
 * minus submit time.  A finished ticket can be polled once.                 */
int dg_poll(dg_server *s, uint64_t ticket, float *q_out, double *latency_s);
int dg_cancel(dg_server *s, uint64_t ticket);
/* Counters: queued, running, finished-not-polled, total batched launches.   */
int dg_server_stats(dg_server *s, int64_t *queued, int64_t *running,
                    int64_t *done, int64_t *launches);
void dg_server_destroy(dg_server *s);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
