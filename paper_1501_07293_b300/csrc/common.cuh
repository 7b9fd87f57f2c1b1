// Internal declarations shared by the CUDA translation units of libmm_b300.
//
// Data layout in HBM (all float32 unless noted):
//   m0, stA, stB, acc, Hs   [3][nz][ny][nx]   unit-vector state, RK4 stage
//                                             buffers, RK4 accumulator, scratch
//   S                       [hx][3][nz][ny]   float2: x-transformed field
//                                             (kx-major, so one kx column of the
//                                             y/z pass is a contiguous slab)
//   Kh                      [hx][hy][6][nz]   demag kernel transformed along x
//                                             and y, real space along z
//                                             (pairs xx yy zz xy xz yz)
//   tw                      [2 Lmax]          float2 twiddles; the table of
//                                             length L sits at offset L
//   hx = px/2 + 1, hy = py/2 + 1 (1 when the padded size is 1).
#pragma once
#include <cuda.h>   // CUtensorMap (a type only; the encoder comes through the runtime)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mm_b300.h"

// Bounds-check builds (-DMM_BOUNDS_CHECK, python -m paper_1501_07293_b300.build
// --bounds-check): the kernels of the single-film path check the shared-memory
// and global indices of their stores and bulk copies; an index out of range
// sets flag[2] (reported as MM_EBOUNDS by the next synchronising call) and the
// access is skipped -- no trap.  In normal builds the checks compile away.
#ifdef MM_BOUNDS_CHECK
static __shared__ int* mm_bc_flag_sh;   // per CTA: the flags an out-of-range index is reported to
extern __shared__ __align__(16) unsigned char mm_bc_dyn_sm[];   // the dynamic shared memory's base
__device__ __forceinline__ unsigned mm_bc_dyn_bytes() {
  unsigned r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}
__device__ __forceinline__ bool mm_bc(bool ok) {
  if (!ok && mm_bc_flag_sh) atomicOr(mm_bc_flag_sh + 2, 1);
  return ok;
}
#define MM_BC_ENTER(flag)                          \
  do {                                             \
    if (threadIdx.x == 0) mm_bc_flag_sh = (flag);  \
    __syncthreads();                               \
  } while (0)
#define MM_BC(cond) mm_bc(cond)
// n bytes at p inside the dynamic shared memory
#define MM_BC_SMEM(p, n)                                                                              \
  mm_bc((const unsigned char*)(p) >= mm_bc_dyn_sm &&                                                  \
        (size_t)((const unsigned char*)(p) - mm_bc_dyn_sm) + (size_t)(n) <= (size_t)mm_bc_dyn_bytes())
#else
#define MM_BC_ENTER(flag) \
  do {                    \
  } while (0)
#define MM_BC(cond) true
#define MM_BC_SMEM(p, n) true
#endif

#define MM_PI 3.14159265358979323846
#define MM_MU0 (4.0e-7 * MM_PI)
#define MM_SERIES_CAP 65536   // records kept by the observables ring (obs_every > 0)

// Grid and launch geometry of one film, passed by value to kernels.
struct Dims {
  int nx, ny, nz;
  int px, py;
  int hx, hy;
  long long N;  // nx*ny*nz
  // split-precision z product (0: FP32 direct sum; MM_SPLIT_BF16 / MM_SPLIT_FP16:
  // tensor-core DFT along z, zsplit.cuh) and its per-context operands
  int prec;
  const float* Kt;             // [hx][PZ/2 + 1][6][hy] tensor transformed along z as well
  const unsigned char* Bdft;   // the two DFT matrices, hi and lo, canonical shared-memory layout
  float2* T;                   // split y/z pass (columns beyond one CTA): [hx][3 nz][py] (else null)
  int route;                   // y/z pass: 0 built-in choice, 1 fused kernel, 2 split pass (mm_set_tuning)
  int ztkb;                    // split pass: ky block of the z product (0: built-in choice)
  int pdl;                     // stage kernels launched with programmatic serialization (large grids)
  int zfft;                    // FP32 fused y/z pass: the z product as a length-32 transform against Kt
                               // (9..16 planes, py = 256 or 512); 0: the direct sum against Kh
  int* flag;                   // the context's device error flags (bounds-check builds report to [2])
};

// Per-cell physics constants, float32, precomputed in double on the host.
struct Phys {
  float c_ex;      // 2A/(Ms delta^2): B_exch = c_ex * sum_nb (m_nb - m)      [T]
  float c_an;      // 2Ku/Ms: B_anis,x = c_an * m_x (scalar Ku)               [T]
  float c_an_map;  // 2/Ms: B_anis,x = c_an_map * Ku(cell) * m_x (Ku map)     [T m^3/J]
  float c_d;       // mu0 Ms/(px py): B_demag = c_d * (inverse transform)     [T]
  float bx, by, bz;  // uniform mu0 H_ext                                      [T]
  float g1, g2;    // -gamma/(1+a^2), -alpha gamma/(1+a^2)
  float inv_mu0;   // 1/mu0 (tesla -> A/m)
};

// Field program (device memory, one per context).  Written only in stream
// order: by single-CTA set-up kernels and, once per step, by the first warp of
// the first y/z CTA (prog_tick), which nothing else in that kernel reads.
struct ProgSeg {
  double t0, t1;        // [t0, t1), seconds
  float b0[3], b1[3];   // mu0 H_ext at t0 and approached at t1 (T), linear in between
  float g1, g2;         // LLG prefactors inside the segment (when own_g)
  int own_g;            // 0: the context's damping applies inside the segment
  int pad;
};
struct ProgState {
  double clock;         // context time (s) of the current state
  long long nstep;      // steps taken since mm_set_m (advanced with the clock)
  float maxdmdt;        // obs_every > 0: max |dm/dt| at the start of the step under way (atomic max of the bits)
  int nseg;
  float base[8];        // bx, by, bz, g1, g2 outside every segment
  float drive[5][8];    // bx, by, bz, g1, g2 at RK4 stages 0..3 of the step under way; [4] at `clock`
  ProgSeg seg[MM_PROGRAM_MAX];
};
// Carried by the first y/z launch of a step: advance the clock by dt and write
// the drive slots of the step (p null: nothing).
struct Tick {
  ProgState* p;
  double dt;
  int euler;
};

// One field evaluation / stage.  mode: 0 = write H_eff, 1 = RK4 stage, 2 = Euler
// step, 3 / 4 = adjoint stage / finish (below).
struct StageArgs {
  const float* m_in;   // state the field is evaluated at (read with neighbours)
  const float* m0;     // RK4 base state
  float* acc;          // RK4 accumulator sum_s w_s k_s
  float* m_out;        // next stage state / new state
  float* H_out;        // mode 0 output (A/m)
  float* B_out;        // modes 1/2: if set, the total field B (tesla) at m_in is stored here
  float* maxdmdt;      // modes 1/2: if set, max over cells of |dm/dt| at m_in is atomically maxed in
  const float* hmap;   // per-cell applied field (T) or null
  const float* kumap;  // per-cell Ku (J/m^3) or null
  const float* drive;  // if set: bx, by, bz, g1, g2 of this evaluation (device), replacing Phys's
  Tick tick;           // launch_stage: passed to its y/z launch
  const CUtensorMap* xmap;   // host: tensor map of S for the x kernel's tile loads (null: per-thread copies)
  int* flag;           // device error flags ([1] <- a bounded wait gave up); set by the launchers
  // modes 3 / 4 (the adjoint sweep, adjoint.cu): m_in is the cotangent lam_B of
  // the field, the kernel forms L lam_B (exchange + demag, tesla) and then
  // closes the stage: ls = loc + L lam_B, lam_m += ls; mode 3 also opens the
  // next stage (lk += c ls, the VJP at (s, B), loc, dL/dh, dL/dKu updated) and
  // writes its lam_B to m_out (and, transformed along x, to S); mode 4
  // writes lam_m + ls to adj_lam
  const float* adj_s;  // the next stage's state and field (mode 3)
  const float* adj_B;
  float* adj_loc;      // local part of the stage's cotangent (read, then rewritten in mode 3)
  float* adj_lam_m;    // running cotangent of the step's start state
  float* adj_lk;       // cotangent of the next stage's k (mode 3)
  float* adj_gh;       // dL/dh, dL/dKu accumulators (mode 3)
  float* adj_gku;
  float* adj_lam;      // mode 4 output
  // mode 5 = mode 4 followed by the start of the previous step's sweep (the
  // renormalisation's cotangent, lk_1..3 and the VJP of its stage 4), whose
  // lam_B goes to m_out and, transformed along x, to S
  const float* adj_sq[4];   // that step's stage states and fields
  const float* adj_Bq[4];
  float* adj_lk0;      // its k cotangents: lk_1, then lk_2, lk_3 at 3N-float strides
  float adj_dt;
  float adj_c;         // dt or dt/2: how the next stage's state depends on its k
  int mode;
  int stage;           // RK4 stage 0..3
  unsigned mask;       // mode 0: MM_TERM_* terms to write
  float dt;
};

// most segments mm_adjoint keeps recorded from its forward pass
static constexpr int kAdjSlots = 8;

struct mm_ctx {
  Dims d;
  double delta, Ms, A, Ku, alpha, gamma;
  double b_ext[3];
  mm_opts opts;
  cudaStream_t stream;       // caller's stream (may be the legacy default stream)
  cudaStream_t cap_stream;   // private stream used only for graph capture
  cudaEvent_t ev;            // orders capture/work between the two streams
  float *m0, *stA, *stB, *acc, *Hs, *hmap, *kumap;
  float2* S;
  float* Kh;
  float2* tw;
  int Lmax;
  double* red;               // reduction partials
  double* red_out;           // final reduction result (device)
  int red_blocks;
  int* dflag;                // device error flags: [0] non-finite state, [1] kernel wait timed out
  ProgState* prog;           // clock, field program and the drive values the stages read
  double* series;            // obs_every > 0: ring of records (t, step, <mx>, <my>, <mz>, max|dm/dt|)
  int series_cap;            // records in the ring
  CUtensorMap* xmap;         // tensor map of S (64-byte aligned host memory) or null
  float* Kt;                 // split precision: tensor transformed along z ([hx][PZ/2+1][6][hy])
  float2* T;                 // split y/z pass buffer (columns beyond one CTA's shared memory)
  unsigned char* Bdft;       // split precision: DFT operands (device)
  int prog_n;                // segments installed
  int cur;                   // Euler: 0 -> state in m0, 1 -> state in stA
  int s_valid;               // S holds the x transform of the current state
  cudaGraphExec_t graph[4];  // RK4: graph[0]; Euler: graph[0] (m0->stA), graph[1] (stA->m0);
                             // graph[2 + g]: kStepsPerGraph steps from the start of graph[g]
  int graph_valid;
  double graph_dt;
  int graph_integrator;
  long long graph_nodes[4];
  long long launches;
  long long steps;
  long long param_gen;        // bumped whenever the field, damping, program or launch shapes change
  // adjoint: captured graphs of a full-length segment, per slot r of the
  // segment buffer: [0] the recomputation into slot 0, [1 + r] the recording in
  // the forward pass (the clock advancing), [1 + kAdjSlots + r] the reverse sweep
  cudaGraphExec_t adj_graph[1 + 2 * kAdjSlots];
  int adj_graph_len;
  double adj_graph_dt;
  long long adj_graph_gen;
  long long adj_graph_nodes[1 + 2 * kAdjSlots];
  double adj_budget;          // bytes of recorded segments the forward pass may keep (mm_set_adjoint_memory)
  // adjoint workspace (allocated by the first mm_adjoint, grown on demand)
  float* adj_ckpt;           // checkpoints [nseg + 1][3N]
  float* adj_seg;            // stage states [k][4][3N] + end state [3N], then fields [k][4][3N]
  float* adj_work;           // cotangents and gradient accumulators
  size_t adj_ckpt_cap, adj_seg_cap, adj_work_cap;   // in floats
  char err[512];
};

// adjoint.cu
void mm_adjoint_free(mm_ctx* c);

// noalloc.cu: device address of mm_heff_noalloc's static scratch on the current
// device (looked up once per device and context); its first ints are the error flags
int mm_noalloc_scratch(unsigned char** base);

// api.cu
Phys mm_make_phys(const mm_ctx* c);

// program.cu: stream-ordered writes of the program state (1 launch each)
int mm_prog_init(mm_ctx* c);        // clock 0, no segments, base and every drive slot from mm_make_phys
int launch_record(mm_ctx* c, const float* m, cudaStream_t s);   // observables record of the new state (1 launch)
int mm_prog_push_base(mm_ctx* c);   // base <- mm_make_phys (b_ext, alpha); drive slots refreshed at the clock

// One film of a batch, as the batched kernels see it (device array).
struct BatchFilm {
  Dims d;
  Phys ph;
  float *m0, *stA, *stB, *acc;
  const float *hmap, *kumap;
  float2* S;
  const float* Kh;
  const float2* tw;
  float* maxdmdt;   // max |dm/dt| recorded at stage 0 (atomic max of the float bits)
  int active;       // 0: the film's CTAs return at once
};

// One persistent launch over every film of a batch (field_inst_persist.cu):
// a work queue of items in the order (stage of the launch, pass, film, tile),
// pass 0 = the y/z columns of every film, pass 1 = the x tiles of every film.
// An item of film f waits (bounded polls) until film f has finished all its
// earlier items, counted in done[f]; items are taken in queue order, so every
// wait is for items already taken by running CTAs.
struct PersistPlan {
  const BatchFilm* F;
  const int* yz_off;     // [nf + 1] prefix sums of the films' y/z items (gyz kx columns each)
  const int* x_off;      // [nf + 1] prefix sums of the films' x items (gx row tiles each)
  int nf, n_yz, n_x;     // films; y/z items and x items of one stage
  int gyz, gx;           // kx columns per y/z item, row tiles per x item
  int nsteps;            // RK4 steps of the launch
  int* next;             // work counter (zeroed before the launch)
  unsigned* done;        // [nf] items finished per film (zeroed before the launch)
  int* flag;             // error flags; [1] <- a dependency or copy wait gave up
  unsigned spin_limit;   // polls before a dependency wait gives up
  int blocked_film;      // self-test: this film's items wait for a count never reached (-1: none)
  int dry;               // self-test: take and order the items, skip their work
  float dt;
};
// 1 if the persistent kernel has bodies for a film of these sizes
int persist_supported(const Dims& d);
// x tiles of a film in the persistent kernel
int persist_x_tiles(const Dims& d);
// kx columns per y/z item and row tiles per x item of the persistent kernel
static constexpr int kPersistGYZ = 16, kPersistGX = 2;
// launch it (grid: every SM's resident CTAs); returns 1 or < 0
int launch_persist(const PersistPlan& p, cudaStream_t s);

// field.cu: one batched launch over the films of a group with equal padded sizes.
// kind: 0 = x forward of m0, 1 = y/z + product, 2 = x inverse + RK4 stage + x forward.
// map[i] = (film, tile) of CTA i; TY = rows per tile of the x kernels (x_batch_tile).
int launch_batch(const BatchFilm* F, int px, int py, int nzm, const int2* map, int nblocks, size_t smem_yz,
                 int kind, int stage, float dt, int* flag, cudaStream_t s);
int x_batch_tile(int px, int kind);
size_t mm_yz_smem(const Dims& d);

// Status helpers (api.cu)
int mm_fail(mm_ctx* c, int code, const char* fmt, ...);
#define MM_CK(ctx, call)                                                              \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return mm_fail((ctx), MM_ECUDA, "%s failed: %s (%s:%d)", #call,                 \
                     cudaGetErrorString(e_), __FILE__, __LINE__);                     \
  } while (0)

// setup.cu: build Kh (FP64 tensor, FP64 2D transform, FP32 store) and the twiddles.
int mm_build_kernel(mm_ctx* c);
// setup.cu: the split-precision operands Kt and Bdft (allocated and built; d.Kt, d.Bdft set)
int mm_build_split(mm_ctx* c);
int mm_build_kz(mm_ctx* c);
// field.cu: padded z size (power of two >= nz) the z product works with
int mm_nzm(int nz);
// field.cu: 1 if one CTA holds a kx column (the fused y/z kernel), 0 if the
// y/z pass runs as three kernels through d.T
int mm_yz_fused(const Dims& d);
// field.cu: kernels one y/z pass launches (1 fused, 3 split)
int mm_yz_launches(const Dims& d);
// field.cu: 1 if a kx column fits one CTA (the fused kernel can run at all)
int mm_yz_fits(const Dims& d);
// field.cu: the largest ky block of the split pass's z product that fits a CTA
int mm_zt_kb_max(const Dims& d);
// field.cu: the ky block the split pass uses
int mm_zt_kb(const Dims& d);

// Same set-up into caller-provided buffers (Kc: 6 nz px py double2 scratch); returns kernels launched or < 0.
int mm_setup_kernel_into(const Dims& d, int self_term, double2* Kc, float* Kh, cudaStream_t s);

// field.cu: launchers (return number of kernels launched, or <0 on launch error)
int mm_supported(const Dims& d, char* why, int nwhy);
// flag: device error flags ([1] <- a bounded wait inside a kernel gave up)
int launch_field_eval(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw,
                      float2* S, const float* Kh, int* flag, cudaStream_t s);
// S holds the x transform of a.m_in: y/z + x inverse/update/forward (2 launches)
int launch_stage(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                 const float* Kh, int* flag, cudaStream_t s);
// S <- x transform of m (1 launch)
int launch_xfwd(const Dims& d, const float* m, const float2* tw, float2* S, cudaStream_t s);
// part: 0 = x-forward, 1 = y/z + product, 2 = x-inverse + update (one launch each)
int launch_field_part(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                      const float* Kh, int* flag, cudaStream_t s, int part);
int launch_normalise(const Dims& d, float* m, int* flag, cudaStream_t s);
// dst <- src normalised (N % 4 == 0, both 16-byte aligned); src may be page-locked host memory
int launch_normalise_from(const Dims& d, const float* src, float* dst, int* flag, cudaStream_t s);

// reduce.cu
// drive: if set, bx, by, bz, g1, g2 (device) replacing Phys's
int launch_reduce(const Dims& d, const Phys& ph, const float* drive, const float* m, const float* Hd,
                  const float* hmap, const float* kumap, double A, double Ku, double delta,
                  double Ms, double* partials, int nblocks, double* out, int* flag,
                  cudaStream_t s);
