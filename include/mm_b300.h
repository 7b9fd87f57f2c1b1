/*
 * mm_b300.h -- C ABI of the B300 finite-difference micromagnetic solver.
 *
 * The library advances the Landau-Lifshitz-Gilbert equation (eq. 2 of
 * arXiv:1501.07293) on an nx x ny x nz grid of cubic cells of edge delta.
 * The effective field (eq. 3) is the sum of
 *   - exchange: six-neighbour Laplacian, eq. 4/5, with the Neumann rule of
 *     eq. 6/7 (a missing neighbour is the cell itself);
 *   - uniaxial anisotropy with the easy axis along x, eq. 8;
 *   - demagnetising field: the discrete convolution of eq. 12/13 with the
 *     tensor of eq. 10/11, evaluated through the convolution theorem, eq. 14,
 *     on a zero-padded grid (Fig. 1);
 *   - Zeeman field: a uniform mu0 H_ext plus an optional per-cell map.
 *
 * Conventions shared by every entry point
 *   - SI units: delta in m, Ms in A/m, A in J/m, Ku in J/m^3, gamma in
 *     rad/(s T), fields passed in as mu0 H (tesla), fields returned as H (A/m),
 *     dt in s, energies in J.  mu0 = 4 pi 1e-7 exactly.
 *   - The state is the unit vector m = M / Ms.  Every vector field is a
 *     float32 array [3][nz][ny][nx] (component-major, x fastest); a scalar
 *     map is float32 [nz][ny][nx].
 *   - Array arguments named *_dev are device pointers; arguments documented
 *     as "host or device" accept either kind (the copy direction is taken
 *     from the pointer).  The caller owns every array it passes; the
 *     context owns only its internal workspaces and copies what it keeps.
 *   - Work is enqueued on the context's stream (mm_opts.stream) and is
 *     asynchronous, except where an entry point says it synchronises.
 *   - Every entry point returns an mm_status; none aborts or traps.  After a
 *     failure mm_last_error() describes it.  A context is not thread-safe;
 *     separate contexts are independent.
 */
#ifndef MM_B300_H
#define MM_B300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_ctx mm_ctx;

typedef enum {
  MM_OK = 0,
  MM_EINVAL = -1,        /* bad argument (null pointer, size, value)          */
  MM_ENOMEM = -2,        /* device allocation failed                          */
  MM_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed       */
  MM_ETIMEOUT = -4,      /* a bounded device wait gave up                     */
  MM_ENONFINITE = -5,    /* a NaN or Inf was found in the state or a result   */
  MM_EUNSUPPORTED = -6,  /* valid request this build does not implement       */
  MM_EBOUNDS = -7        /* bounds-check builds only: a kernel index was out of
                            range (the access was skipped)                    */
} mm_status;

enum { MM_FP32 = 0, MM_SPLIT_BF16 = 1, MM_SPLIT_FP16 = 2 };   /* mm_opts.precision */
enum { MM_RK4 = 0, MM_EULER = 1 };                            /* mm_opts.integrator */

/* Bit mask of effective-field terms (mm_heff). */
enum {
  MM_TERM_EXCHANGE = 1,
  MM_TERM_ANISOTROPY = 2,
  MM_TERM_DEMAG = 4,
  MM_TERM_ZEEMAN = 8,
  MM_TERM_ALL = 15
};

typedef struct {
  int precision;    /* MM_FP32 (default): the demag product along z in FP32 (see zform).
                       MM_SPLIT_BF16 / MM_SPLIT_FP16: that product through a
                       length-2nz DFT along z computed as GEMMs on the tensor cores
                       (tcgen05) with 16-bit hi+lo split operands (x = hi + lo,
                       products hi*hi + hi*lo + lo*hi, FP32 accumulation; FP16 with
                       the data scaled by 2^-12); everything else stays FP32.
                       Split modes need 5 <= nz <= 16 and ny >= 33 (MM_EUNSUPPORTED
                       otherwise); the effective field then agrees with the FP32
                       path to ~1e-5 relative.  The paper computes in FP32/FP64 only. */
  int integrator;   /* MM_RK4 (classical, renormalise after the full step) or MM_EULER
                       (the paper's explicit Euler step + renormalisation)               */
  int self_term;    /* 1: keep the tensor's self offset K(0,0,0) = -I/3 (default);
                       0: drop it as the paper's tensor listing does                    */
  int obs_every;    /* > 0: every obs_every-th step since mm_set_m appends a record
                       (t, step, <mx>, <my>, <mz>, max|dm/dt|) to a device ring of the
                       last 65536 records, inside the step graph (no host round trip;
                       one extra launch per step); read with mm_get_series.  The paper
                       writes <m> every 1000 steps (script of Appendix A).  0: off.      */
  void* stream;     /* cudaStream_t the context enqueues on; NULL = legacy default       */
  const char* tune_cache;   /* path of a JSON file of launch shapes recorded by the
                       autotuner (paper_1501_07293_b300.tune.autotune): mm_create
                       applies the y/z route and ky block recorded for this grid's
                       padded size and precision, as mm_set_tuning would.  NULL, a
                       missing file or a missing entry keep the built-in choice.     */
  int zform;        /* MM_FP32 only: how the demag product of eq. 14 runs along z.
                       MM_ZFORM_AUTO (default): as a length-32 circular convolution
                       through register transforms along z against the tensor
                       transformed along z as well (one extra FP32 array of
                       17 x 6 x hx x hy values, built by mm_create), wherever the
                       fused y/z kernel takes the film (9..16 planes, padded y of 256
                       or 512); elsewhere, and with MM_ZFORM_DIRECT, as the direct
                       Toeplitz sum over the nz planes against the tensor transformed
                       along x and y only.  Both are exact (eq. 13 restricted to z);
                       they differ by FP32 rounding only.                            */
} mm_opts;

enum { MM_ZFORM_AUTO = 0, MM_ZFORM_DIRECT = 1 };   /* mm_opts.zform */

/* Fill *opts with the defaults: MM_FP32, MM_RK4, self_term 1, obs_every 0, NULL stream,
 * no tune cache, MM_ZFORM_AUTO. */
void mm_default_opts(mm_opts* opts);

/*
 * Create a context for one film: grid = {nx, ny, nz} cells (each >= 1), cell
 * edge delta, saturation magnetisation Ms, exchange constant A, anisotropy
 * constant Ku (easy axis x), damping alpha and gyromagnetic ratio gamma.
 * opts may be NULL (defaults).  Builds the demagnetising tensor (eq. 10/11)
 * in FP64 on the device and transforms it once (eq. 14).  The initial state
 * is m = (1, 0, 0) everywhere and the applied field is zero.  Synchronises.
 * Returns MM_EUNSUPPORTED for grids whose padded transform does not fit the
 * kernels of this build (see mm_padded_dims); *out is NULL on failure.
 */
int mm_create(mm_ctx** out, const int grid[3], double delta, double Ms, double A,
              double Ku, double alpha, double gamma, const mm_opts* opts);

/* Release the context and its device memory (NULL is accepted).  Synchronises. */
void mm_destroy(mm_ctx* ctx);

/* Change the stream subsequent calls enqueue on (a cudaStream_t; NULL = legacy default). */
int mm_set_stream(mm_ctx* ctx, void* stream);

/* Padded transform sizes {px, py, pz} chosen for the grid (px >= 2nx - 1, ...). */
int mm_padded_dims(const mm_ctx* ctx, int padded[3]);

/*
 * Set the state from m (host or device, [3][nz][ny][nx] float32).  Each cell's
 * vector is normalised on entry; a zero or non-finite vector is kept as given
 * and gives MM_ENONFINITE when it is detected (at the next synchronising call).
 * Page-locked host memory (cudaHostAlloc / cudaHostRegister) is read directly
 * by the normalising kernel when N is a multiple of 4; other memory is copied
 * first.  Asynchronous either way: m must stay unchanged until the stream has
 * passed this call.
 */
int mm_set_m(mm_ctx* ctx, const float* m);

/* Copy the current state into m (host or device, [3][nz][ny][nx] float32). */
int mm_get_m(mm_ctx* ctx, float* m);

/*
 * Applied field: b_ext = mu0 H_ext (tesla, 3 doubles, host).  h_map (host or
 * device, [3][nz][ny][nx] tesla) is an optional per-cell addition, ku_map
 * (host or device, [nz][ny][nx] J/m^3) an optional per-cell Ku that replaces
 * the scalar Ku.  NULL clears a map.  The maps are copied.  The next mm_step
 * patches the new values into its captured step graph in place (re-capture +
 * graph update, no re-instantiation), so a host loop of mm_set_field +
 * mm_step (a hysteresis sweep) stays cheap.
 */
int mm_set_field(mm_ctx* ctx, const double b_ext[3], const float* h_map, const float* ku_map);

/* Change the damping constant (the paper switches alpha between its relax and
 * reverse phases).  Patched into the step graph like b_ext. */
int mm_set_alpha(mm_ctx* ctx, double alpha);

/*
 * Field program: a time-dependent uniform field and damping evaluated on the
 * device at every stage of every step, so that a whole protocol such as the
 * paper's standard-problem-4 run (saturate along (1,1,1), ramp down, then
 * reverse with a damping switch; Section 3 and the script of Appendix A) runs
 * as graph replays without host round trips.
 *
 * Each context has a clock (seconds, FP64, on the device): mm_step advances it
 * by dt per step, and the RK4 stages of the step from t evaluate the program
 * at t, t + dt/2, t + dt/2, t + dt (Euler at t).  At time t the first segment
 * with t_begin <= t < t_end gives
 *     b_ext(t) = b_begin + (t - t_begin) / (t_end - t_begin) (b_end - b_begin),
 *     alpha(t) = alpha (segment value; alpha < 0 keeps the context's alpha);
 * outside every segment the context's b_ext / alpha (mm_set_field, mm_set_alpha)
 * apply.  mm_heff, mm_energy and mm_observables use the values at the clock.
 */
#define MM_PROGRAM_MAX 32
typedef struct {
  double t_begin, t_end;   /* seconds, t_end > t_begin                          */
  double b_begin[3];       /* mu0 H_ext at t_begin, tesla                       */
  double b_end[3];         /* mu0 H_ext approached at t_end, tesla              */
  double alpha;            /* damping inside the segment; < 0: context's alpha  */
} mm_segment;

/* Install nseg (0 .. MM_PROGRAM_MAX) segments (host array, copied; nseg 0
 * removes the program).  Stream-ordered.  MM_EINVAL for a non-finite value or
 * t_end <= t_begin.  While a program is installed the field and damping are
 * read from device memory at every stage, so changing the segments, b_ext or
 * alpha needs no graph update at all. */
int mm_set_program(mm_ctx* ctx, int nseg, const mm_segment* seg);

/* Set the clock (stream-ordered).  mm_create starts it at 0; mm_set_m does not
 * change it. */
int mm_set_time(mm_ctx* ctx, double t);

/* Read the clock into *t (host).  Synchronises. */
int mm_get_time(mm_ctx* ctx, double* t);

/*
 * Effective field (eq. 3) of the current state, restricted to the terms in
 * term_mask (MM_TERM_*), written to H_dev ([3][nz][ny][nx] float32, A/m).
 */
int mm_heff(mm_ctx* ctx, float* H_dev, unsigned term_mask);

/*
 * Advance n >= 0 steps of size dt with the context's integrator.  One RK4
 * step evaluates the effective field four times; the state is renormalised
 * once after each full step (the paper renormalises after every Euler step).
 * The step sequence is replayed from a captured CUDA graph (two kernels per
 * field evaluation); a call after mm_set_m / mm_heff / mm_energy /
 * mm_observables first launches one x-transform of the state.
 */
int mm_step(mm_ctx* ctx, int n, double dt);

/*
 * Energies of the current state (eq. 1 on the grid), in J:
 * E[0] exchange, E[1] anisotropy, E[2] demagnetising, E[3] Zeeman, E[4] total.
 * Accumulated in FP64.  Synchronises.
 */
int mm_energy(mm_ctx* ctx, double E[5]);

/*
 * Observables of the current state: out[0..2] = mean of m_x, m_y, m_z,
 * out[3] = max over cells of |dm/dt| (rad/s), out[4] = steps taken since the
 * last mm_set_m.  Accumulated in FP64.  Synchronises.  Returns MM_ENONFINITE
 * if the state holds a NaN or Inf.
 */
int mm_observables(mm_ctx* ctx, double out[5]);

/*
 * Profiling variant of mm_step: advance n steps launching every kernel
 * eagerly (no graph) with CUDA events around each launch, and add the device
 * time of each kernel class to ms_out[3]: [0] the x-forward transform that
 * (re)starts the pipeline after mm_set_m / mm_heff / mm_energy (not part of a
 * step), [1] y/z transforms with the demag product, [2] x-inverse transforms
 * with the field/LLG update and the x-forward transform of the new state.
 * ms_out is host memory, accumulated into (not cleared).  Same numerical
 * result as mm_step.  Synchronises after every step.
 */
int mm_step_timed(mm_ctx* ctx, int n, double dt, double ms_out[3]);

/*
 * Gradients of a loss of the final state of an RK4 trajectory (the reverse
 * mode of the step sequence mm_step runs; the paper has no adjoint, this is
 * the derivative of its eq. 2 with the fields of eq. 3, 5/7, 8 and 13).
 *
 * The trajectory starts from the context's current state m0 and runs n >= 1
 * steps of size dt with the current applied field and maps; on return the
 * context holds the final state m_n (as after mm_step(ctx, n, dt)).
 * dL_dm_final (host or device, [3][nz][ny][nx]) is dL/dm_n.  Outputs (host or
 * device; NULL skips one):
 *   dL_dh   [3][nz][ny][nx]  gradient with respect to the per-cell applied
 *                            field map h (per tesla), whether or not a map is set
 *   dL_dku  [nz][ny][nx]     gradient with respect to the per-cell Ku (per J/m^3)
 *   dL_dm0  [3][nz][ny][nx]  gradient with respect to the direction of m0,
 *                            (I - m0 m0^T) dL/dm0, i.e. through the
 *                            normalisation that mm_set_m applies
 * Memory: checkpoints every ckpt_every steps ((n/ckpt_every + 1) states) and
 * R segment slots of 8 ckpt_every + 1 vector fields each (every stage state
 * and field of a segment), allocated on the first call and kept.  The forward
 * pass records its last R segments into the slots, so only the segments before
 * them are recomputed from their checkpoints: R = 1 by default, more (at most
 * 8, at most the number of segments) as far as mm_set_adjoint_memory allows.
 * The gradients are the same bit for bit whatever R is.  Cost: one forward
 * pass, one recomputation of the unrecorded segments, and four applications of
 * the symmetric exchange + demag operator per step.  RK4 only (MM_EUNSUPPORTED
 * for Euler or while a field program is installed: the derivative assumes a
 * constant uniform field and damping).  Asynchronous.
 */
int mm_adjoint(mm_ctx* ctx, int n, double dt, int ckpt_every, const float* dL_dm_final,
               float* dL_dh, float* dL_dku, float* dL_dm0);

/*
 * Device memory, in bytes, that mm_adjoint may give to recorded segments.  A
 * slot holds 12 (8 ckpt_every + 1) N bytes (every stage state and field of one
 * segment, N cells); mm_adjoint uses R = max(1, min(8, segments,
 * floor(bytes / slot bytes))) slots.  0 (the default) keeps R = 1: every
 * segment but the last is recomputed from its checkpoint.  A larger budget
 * trades device memory for recomputation.  MM_EINVAL for a negative or NaN
 * value.
 */
int mm_set_adjoint_memory(mm_ctx* ctx, double bytes);

/*
 * Observables series (mm_opts.obs_every > 0): copies the most recent records
 * written since mm_set_m, oldest first, at most max_records of them, into out
 * (host, 6 doubles each: time (s), step, <mx>, <my>, <mz>, max over cells of
 * |dm/dt| (rad/s) at the start of the recorded step); *n_records = how many.
 * <m> is of the state after the step, accumulated in FP64.  Synchronises.
 * MM_EINVAL when the context was created with obs_every = 0.
 */
int mm_get_series(mm_ctx* ctx, double* out, int max_records, int* n_records);

/*
 * Launch-shape overrides for the y/z pass (the paper has no counterpart; the
 * knobs of paper_1501_07293_b300.tune's autotuner).  yz_route: 0 built-in
 * choice, 1 the fused kernel (one CTA per kx column; MM_EUNSUPPORTED if a column
 * does not fit), 2 the split pass (y transforms and z product as three kernels
 * through a buffer, allocated here if needed; FP32 only).  zt_block: ky block of
 * the split pass's z product, 0 built-in choice, else >= 8 (clamped to what
 * fits a CTA).  Results are identical either way; the next mm_step re-captures
 * its graph.  mm_get_tuning reports the route (1 or 2) and block in effect.
 */
int mm_set_tuning(mm_ctx* ctx, int yz_route, int zt_block);
int mm_get_tuning(const mm_ctx* ctx, int* yz_route, int* zt_block);

/* Build flags of the loaded library: bit 0 set for the bounds-check build
 * (-DMM_BOUNDS_CHECK, libmm_b300_bc.so), whose kernels check the shared-memory
 * and global indices of their stores and copies and report an out-of-range one
 * as MM_EBOUNDS at the next synchronising call instead of performing it. */
int mm_build_flags(void);

/* Number of kernels this context has enqueued so far (graph nodes counted per replay). */
long long mm_launch_count(const mm_ctx* ctx);

/*
 * Self-test of the failure path of the kernels' bounded waits (the paper has
 * no counterpart): enqueues one CTA that polls an mbarrier phase nothing
 * completes, gives up after `polls` (1 .. 2^20) polls, sets the timeout flag
 * and returns, as a kernel whose bulk copy never lands would.  The next
 * mm_sync / mm_energy / mm_observables returns MM_ETIMEOUT and clears the flag;
 * the context stays usable.  With ctx NULL the flag set is that of
 * mm_heff_noalloc's scratch on the current device (legacy default stream),
 * reported by mm_noalloc_status.
 */
int mm_selftest_wait_timeout(mm_ctx* ctx, unsigned polls);

/*
 * The demagnetising tensor K_ab of eq. 10/11 (in units where delta = 1; the
 * tensor is scale free) at n (1 .. 2^20) integer offsets, evaluated on the
 * current device in FP64 exactly as the set-up of mm_create does it: the
 * eight-corner sums of eq. 10/11 within 9 cells of the source, beyond that
 * the multipole series of the same tensor (the field of a uniformly
 * magnetised cube, expanded in powers of 1/|n|; the paper has no
 * counterpart), whose truncation error is below ~3e-14 relative (~1e-15 beyond
 * 12 cells) where the corner sums lose ~eps |n|^3 to cancellation.  offsets: host, n triples
 * (I, J, K); out: host, n x 6 doubles (xx, yy, zz, xy, xz, yz).  The self
 * offset gives -I/3.  Synchronises; allocates two small device buffers.
 * MM_EINVAL / MM_ENOMEM / MM_ECUDA.
 */
int mm_tensor_eval(const int* offsets, int n, double* out);

/*
 * Peak-rate probe of the FP32 pipes (measurement only; the paper has no
 * counterpart): enqueues on `stream` (a cudaStream_t; NULL = legacy default)
 * one launch of register-resident fused multiply-add chains, 4 CTAs of 256
 * threads per SM of the current device, `iters` (1 .. 2^24) iterations of 8
 * independent chains per thread; packed = 1 issues the packed pair FMA
 * (__ffma2_rn), 0 the scalar fmaf.  *flops (host) receives the floating-point
 * operations of the launch (2 per FMA); the caller times the launch with CUDA
 * events.  Touches no memory.  MM_EINVAL / MM_ECUDA on bad arguments / launch
 * failure.
 */
int mm_fp32_probe(int packed, int iters, void* stream, double* flops);

/* Block until the context's stream is idle; reports a pending device-side error. */
int mm_sync(mm_ctx* ctx);

/* Text of the last failure of this context ("" if none); ctx NULL gives the last create failure. */
const char* mm_last_error(const mm_ctx* ctx);

/*
 * Batches of independent films (e.g. one film per point of a field sweep),
 * advanced together.  The paper runs one film; a batch applies the same
 * per-film method (every entry point above, through mm_batch_film) to many
 * films of uneven size.  Two schedules of an RK4 step, each replayed from a
 * captured CUDA graph:
 *   persistent (default when every film has px 32..512, py 16..256 and
 *     nz <= 4): one kernel launch per step whose CTAs take the y/z columns and
 *     x tiles of all films from one device work queue; an item waits (bounded)
 *     only for the earlier items of its own film, so films of different sizes
 *     share the SMs inside the launch;
 *   grouped: films with equal padded sizes share one launch per kernel, and
 *     the groups run as parallel branches of the step graph.
 * RK4 only.
 */
typedef struct mm_batch mm_batch;

/*
 * nfilms films; grids = nfilms consecutive {nx, ny, nz} triples (host); shared
 * material parameters as in mm_create.  Each film starts at m = (1, 0, 0) with
 * zero applied field.  Synchronises.  *out is NULL on failure (mm_batch_last_error(NULL)).
 */
int mm_batch_create(mm_batch** out, int nfilms, const int* grids, double delta, double Ms, double A,
                    double Ku, double alpha, double gamma, const mm_opts* opts);
void mm_batch_destroy(mm_batch* b);

/* The context of film f (owned by the batch; do not destroy): mm_set_m, mm_get_m,
 * mm_set_field, mm_heff, mm_energy, mm_observables work on it. */
mm_ctx* mm_batch_film(mm_batch* b, int film);

/* Advance every film n steps of size dt. */
int mm_batch_step(mm_batch* b, int n, double dt);

/*
 * Advance every film until its max over cells of |dm/dt| (rad/s, eq. 2 at the
 * state) is below tol_dmdt, checked every check_every steps, or max_steps steps
 * have been taken.  A film that stops keeps its state from then on.
 * steps_out (host, nfilms ints, nullable) receives the steps each film took.
 * Synchronises.
 */
int mm_batch_run(mm_batch* b, int max_steps, double dt, double tol_dmdt, int check_every, int* steps_out);

/* max |dm/dt| (rad/s) per film as last recorded (host, nfilms floats).  Synchronises. */
int mm_batch_max_dmdt(mm_batch* b, float* out);

/* Number of groups of equal padded sizes (= parallel branches of the step graph). */
int mm_batch_group_count(const mm_batch* b);

/* Kernels enqueued by the batch's own launches so far. */
long long mm_batch_launch_count(const mm_batch* b);

/* Schedule of the batch's steps: 1 persistent, 0 grouped.  MM_EUNSUPPORTED if
 * some film has no body in the persistent kernel.  The next step re-captures. */
int mm_batch_set_schedule(mm_batch* b, int persistent);
int mm_batch_get_schedule(const mm_batch* b);

/* Block until the batch's stream is idle; MM_ETIMEOUT if a bounded wait inside a
 * batched kernel gave up since the last call (the flag is cleared). */
int mm_batch_sync(mm_batch* b);

/*
 * Self-test of the persistent kernel's bounded dependency waits (the paper has
 * no counterpart): one launch of the persistent kernel in which film 0's items
 * wait for a progress count nothing reaches and give up after `polls` (1 ..
 * 2^20) polls; no item does its work, so every film keeps its state.  The next
 * mm_batch_sync returns MM_ETIMEOUT; the batch stays usable.  MM_EUNSUPPORTED
 * when the batch cannot run the persistent kernel.
 */
int mm_batch_selftest_wait_timeout(mm_batch* b, unsigned polls);

/* Last failure of this batch ("" if none); NULL gives the last create failure. */
const char* mm_batch_last_error(const mm_batch* b);

/*
 * Size of the static device scratch array behind mm_heff_noalloc (32 MiB).
 * It exists on every GPU that loads the library, for the life of the process.
 */
#define MM_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * mm_heff_noalloc -- the effective field of one state, computed without any
 * device allocation.  The paper has no counterpart: it serves callers that
 * cannot call cudaMalloc, for example a plug-in whose host application owns
 * the GPU's memory pool and hands it out only as buffers it allocated itself,
 * code running where a caching allocator already holds the device's free
 * memory (a cudaMalloc there fails although the pool has room), or a
 * latency-bound loop that cannot take the device-wide synchronisation that
 * cudaMalloc and cudaFree imply.
 *
 * It needs no context: from grid = {nx, ny, nz}, delta, Ms, A, Ku (easy axis
 * x), b_ext = mu0 H_ext (tesla, 3 host doubles) and self_term (1 keeps the
 * tensor's self offset, as mm_create does by default) it builds the
 * demagnetising tensor (eq. 10/11) and evaluates, for the unit vectors m_dev
 * ([3][nz][ny][nx] float32, device, used as given -- not normalised), the
 * terms of term_mask (MM_TERM_*) into H_dev ([3][nz][ny][nx] float32, A/m,
 * device).  The result equals mm_heff on a context created with the same
 * parameters and holding the same state.  Work is enqueued on `stream`
 * (a cudaStream_t; NULL = legacy default stream) and is asynchronous.
 *
 * Cost: every call rebuilds the tensor (the FP64 eq. 10/11 kernel and two FP64
 * transforms of 6 nz px py values) before its one field evaluation, while
 * mm_heff on a context uses the tensor mm_create built once.  Measured on a
 * B300 at 128 x 128 x 4 (CUDA events): 1.62 ms per mm_heff_noalloc call
 * against 0.023 ms per mm_heff call.
 *
 * All intermediate data lives in one file-scope static device array of
 * MM_NOALLOC_SCRATCH_BYTES; grids whose tensor planes (6 nz px py complex
 * doubles) plus transformed tables do not fit are refused with
 * MM_EUNSUPPORTED (128 x 128 x 4 fits; 256 x 256 x 4 does not).  No call
 * allocates, frees or calls an allocating library routine.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and caches it for that
 * device's CUDA context (a new context, after cudaDeviceReset, looks it up
 * again); make that first call before any stream capture.  Every call on a
 * device uses the same array, and each call writes every byte of it that it
 * later reads (the error flags excepted, see mm_noalloc_status), so nothing has
 * to be cleared between calls; but two calls whose work overlaps on the GPU
 * (different streams, or different host threads) race on the array and give
 * wrong results.  Serialise them.
 *
 * Errors: MM_EINVAL (NULL pointer, size < 1, bad parameter or mask),
 * MM_EUNSUPPORTED (too large for the array or for the kernels), MM_ECUDA
 * (launch failure); mm_noalloc_last_error() describes the last failure of the
 * calling thread.  Conditions found on the device while the kernels run are
 * reported by mm_noalloc_status, not by the (asynchronous) call itself.
 */
int mm_heff_noalloc(const int grid[3], double delta, double Ms, double A, double Ku,
                    const double b_ext[3], int self_term, const float* m_dev, float* H_dev,
                    unsigned term_mask, void* stream);

/*
 * Device-side status of the mm_heff_noalloc calls made so far on the current
 * device: synchronises `stream` (a cudaStream_t; NULL = legacy default), reads
 * the kernels' error flags from the scratch array and clears them.  Returns
 * MM_ETIMEOUT if a bounded wait inside a kernel gave up (that call's H is not
 * valid), MM_ENONFINITE if a kernel flagged a non-finite value, else MM_OK.
 * The flags accumulate over calls until this reads them.  Allocates nothing.
 * mm_selftest_wait_timeout(NULL, polls) sets the timeout flag on purpose, to
 * test this path.
 */
int mm_noalloc_status(void* stream);

/* Text of the calling thread's last mm_heff_noalloc / mm_noalloc_status failure ("" if none). */
const char* mm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MM_B300_H */
