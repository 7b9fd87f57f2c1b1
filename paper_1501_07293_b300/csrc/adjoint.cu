// Reverse-mode derivative (adjoint) of the RK4 trajectory that mm_step runs:
// gradients of a loss of the final state with respect to the initial state, the
// per-cell applied field map h and the per-cell anisotropy map Ku.
//
// Forward step (unit vectors m, B = mu0 H_eff of eq. 3 in tesla):
//   k_i = f(s_i), s_1 = m, s_2 = m + dt/2 k_1, s_3 = m + dt/2 k_2, s_4 = m + dt k_3
//   u = m + dt/6 (k_1 + 2 k_2 + 2 k_3 + k_4),  m' = u / |u|
//   f(s) = g1 s x B + g2 s x (s x B)                                     (eq. 2)
//   B(s) = L s + c s_x x^ + b_ext + h,  c = 2 Ku / Ms                     (eq. 5/7, 13, 8)
// L (exchange + demag) is symmetric, so its adjoint is itself: the reverse
// sweep applies the same field kernels to the cotangent lam_B.
// Reverse step, per cell, for a cotangent lam of m':
//   lam_u = (I - m' m'^T) lam / |u|,  lam_m = lam_u,
//   lam_k1 = lam_k4 = dt/6 lam_u,  lam_k2 = lam_k3 = dt/3 lam_u,
//   stage i = 4, 3, 2, 1 (vector-Jacobian product of f at s_i, cotangent lk):
//     lam_B   = g1 (lk x s) + g2 ((lk x s) x s)
//     lam_loc = g1 (B x lk) + g2 ((s x B) x lk) + g2 (B x (lk x s)) + c (lam_B)_x x^
//     lam_s   = lam_loc + L lam_B
//     dL/dh += lam_B,  dL/dKu += (2/Ms) s_x (lam_B)_x,  lam_m += lam_s,
//     and lam_k3 += dt lam_s4, lam_k2 += dt/2 lam_s3, lam_k1 += dt/2 lam_s2.
// The trajectory is kept as checkpoints every `ckpt_every` steps; each segment
// is recomputed once with every stage state s_i and field B_i stored, then
// swept in reverse -- except the last R segments, which the forward pass
// records directly (R = 1, or more within the memory budget of
// mm_set_adjoint_memory).  Per reverse step: per stage the y/z pass and the x kernel
// in its adjoint mode, which applies L to lam_B and does the closing and
// opening updates of the stages in the same pass (StageArgs modes 3 - 5); the
// closing kernel of a step also starts the previous step, so only a segment's
// last step has a separate start (k_adj_start and an x transform).  A
// full-length segment (recomputation and sweep) is a captured graph, replayed
// for every segment.
#include <string.h>

#include "adjoint.cuh"
#include "common.cuh"

struct AdjArgs {
  const float* s[4];   // stage input states of the step
  const float* B[4];   // their fields (tesla)
  float* lam;          // in: cotangent of m' (start); out: cotangent of m (finish)
  float* lam_m;        // running cotangent of m
  float* lk[3];        // cotangents of k_1, k_2, k_3
  float* lamB;         // cotangent of B at the current stage (input of the linear operator)
  float* lamloc;       // local part of the cotangent of the current stage state
  float* gh;           // dL/dh accumulator [3][N]
  float* gku;          // dL/dKu accumulator [N]
  const float* kumap;  // per-cell Ku or null
  float c_an;          // 2 Ku / Ms (scalar Ku)
  float c_an_map;      // 2 / Ms (times Ku(cell) with a map)
  float two_over_Ms;
  float g1, g2, dt;
  long long N;
};

__device__ __forceinline__ float3 ld3v(const float* p, long long N, long long i) {
  return make_float3(p[i], p[i + N], p[i + 2 * N]);
}
__device__ __forceinline__ void st3v(float* p, long long N, long long i, float3 v) {
  p[i] = v.x; p[i + N] = v.y; p[i + 2 * N] = v.z;
}
__device__ __forceinline__ float3 xp3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sc3(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }

__global__ void k_adj_start(AdjArgs A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  float3 s[4], B[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    s[q] = ld3v(A.s[q], A.N, i);
    B[q] = ld3v(A.B[q], A.N, i);
  }
  const float c = A.kumap ? A.c_an_map * A.kumap[i] : A.c_an;
  float3 lu, lamB, loc;
  adj_step_start(A.g1, A.g2, c, A.dt, s, B, ld3v(A.lam, A.N, i), lu, lamB, loc);
  const float h = A.dt * (1.0f / 6.0f);
  st3v(A.lam_m, A.N, i, lu);
  st3v(A.lk[0], A.N, i, sc3(h, lu));
  st3v(A.lk[1], A.N, i, sc3(2.f * h, lu));
  st3v(A.lk[2], A.N, i, sc3(2.f * h, lu));
  st3v(A.lamB, A.N, i, lamB);
  st3v(A.lamloc, A.N, i, loc);
  st3v(A.gh, A.N, i, add3(ld3v(A.gh, A.N, i), lamB));
  A.gku[i] += A.two_over_Ms * s[3].x * lamB.x;
}

// g <- (I - m m^T) g  (the gradient with respect to the direction of the initial state)
__global__ void k_tangent(const float* __restrict__ m, float* __restrict__ g, long long N) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float3 mm = ld3v(m, N, i), gg = ld3v(g, N, i);
  const float d = mm.x * gg.x + mm.y * gg.y + mm.z * gg.z;
  st3v(g, N, i, make_float3(gg.x - d * mm.x, gg.y - d * mm.y, gg.z - d * mm.z));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int grow(mm_ctx* c, float** p, size_t* cap, size_t need_floats) {
  if (*cap >= need_floats) return MM_OK;
  cudaStreamSynchronize(c->stream);
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, need_floats * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return mm_fail(c, MM_ENOMEM, "adjoint workspace: cannot allocate %zu bytes", need_floats * sizeof(float));
  }
  *cap = need_floats;
  return MM_OK;
}

static void drop_adj_graphs(mm_ctx* c) {
  for (int i = 0; i < 1 + 2 * kAdjSlots; ++i)
    if (c->adj_graph[i]) {
      cudaGraphExecDestroy(c->adj_graph[i]);
      c->adj_graph[i] = nullptr;
    }
}

extern "C" int mm_set_adjoint_memory(mm_ctx* c, double bytes) {
  if (!c) return MM_EINVAL;
  if (!(bytes >= 0)) return mm_fail(c, MM_EINVAL, "mm_set_adjoint_memory: bytes = %g", bytes);
  c->adj_budget = bytes;
  return MM_OK;
}

void mm_adjoint_free(mm_ctx* c) {
  for (int i = 0; i < 1 + 2 * kAdjSlots; ++i)
    if (c->adj_graph[i]) {
      cudaGraphExecDestroy(c->adj_graph[i]);
      c->adj_graph[i] = nullptr;
    }
  cudaFree(c->adj_ckpt);
  cudaFree(c->adj_seg);
  cudaFree(c->adj_work);
  c->adj_ckpt = c->adj_seg = c->adj_work = nullptr;
  c->adj_ckpt_cap = c->adj_seg_cap = c->adj_work_cap = 0;
}

extern "C" int mm_adjoint(mm_ctx* c, int n, double dt, int ckpt_every, const float* dL_dm_final, float* dL_dh,
                          float* dL_dku, float* dL_dm0) {
  if (!c) return MM_EINVAL;
  if (n < 1 || ckpt_every < 1) return mm_fail(c, MM_EINVAL, "mm_adjoint: need n >= 1 and ckpt_every >= 1");
  if (!(dt > 0) || dt > 1e-6) return mm_fail(c, MM_EINVAL, "mm_adjoint: dt = %g s out of range", dt);
  if (!dL_dm_final) return mm_fail(c, MM_EINVAL, "mm_adjoint: dL_dm_final is NULL");
  if (c->opts.integrator != MM_RK4) return mm_fail(c, MM_EUNSUPPORTED, "mm_adjoint: only the RK4 integrator");
  if (c->prog_n > 0)
    return mm_fail(c, MM_EUNSUPPORTED, "mm_adjoint: a field program is installed (constant field and damping only)");
  const long long N = c->d.N;
  const size_t v3 = 3 * (size_t)N;
  const int k = ckpt_every < n ? ckpt_every : n;
  const int nseg = (n + k - 1) / k;
  // the forward pass records its last R segments (stage states and fields) in
  // R slots of the segment buffer: the last one always, more while the slots
  // fit the budget of mm_set_adjoint_memory; only the segments before them are
  // recomputed from their checkpoints
  const size_t slot = (size_t)(8 * k + 1) * v3;   // floats of one recorded segment
  int R = (int)(c->adj_budget / ((double)slot * sizeof(float)));
  if (R > nseg) R = nseg;
  if (R > kAdjSlots) R = kAdjSlots;
  if (R < 1) R = 1;
  int rc;
  float* const prev[3] = {c->adj_ckpt, c->adj_seg, c->adj_work};
  if ((rc = grow(c, &c->adj_ckpt, &c->adj_ckpt_cap, (size_t)(nseg + 1) * v3)) != MM_OK) return rc;
  if ((rc = grow(c, &c->adj_seg, &c->adj_seg_cap, (size_t)R * slot)) != MM_OK) return rc;
  if ((rc = grow(c, &c->adj_work, &c->adj_work_cap, 9 * v3 + (size_t)N)) != MM_OK) return rc;
  if (prev[0] != c->adj_ckpt || prev[1] != c->adj_seg || prev[2] != c->adj_work) drop_adj_graphs(c);
  float* W = c->adj_work;
  float *lam = W, *lam_m = W + v3, *lk0 = W + 2 * v3, *lk1 = W + 3 * v3, *lk2 = W + 4 * v3;
  float *lamB = W + 5 * v3, *lamloc = W + 6 * v3, *lamB2 = W + 7 * v3, *gh = W + 8 * v3, *gku = W + 9 * v3;
  // (lamB2: the other lam_B buffer of the fused sweep, ping-pong)
  // slot r: [k][4][3N] stage states, then [1][3N] the segment's end, then
  // [k][4][3N] fields (the workspace addresses are baked into the segment
  // graphs: a workspace that grows is a new allocation, so they are dropped then)
  auto seg_s = [&](int r) { return c->adj_seg + (size_t)r * slot; };
  auto seg_B = [&](int r) { return c->adj_seg + (size_t)r * slot + (size_t)(4 * k + 1) * v3; };
  cudaStream_t s = c->stream;

  const Phys ph = [&] {
    Phys p;
    const double Ms = c->Ms, dl = c->delta;
    p.c_ex = (float)(2.0 * c->A / (Ms * dl * dl));
    p.c_an = (float)(2.0 * c->Ku / Ms);
    p.c_an_map = (float)(2.0 / Ms);
    p.c_d = (float)(MM_MU0 * Ms / ((double)c->d.px * (double)c->d.py));
    p.bx = (float)c->b_ext[0];
    p.by = (float)c->b_ext[1];
    p.bz = (float)c->b_ext[2];
    const double gg = c->gamma / (1.0 + c->alpha * c->alpha);
    p.g1 = (float)(-gg);
    p.g2 = (float)(-c->alpha * gg);
    p.inv_mu0 = (float)(1.0 / MM_MU0);
    return p;
  }();
  Phys lin = ph;          // the linear operator L on a cotangent, output in tesla
  lin.inv_mu0 = 1.0f;
  AdjArgs A;
  memset(&A, 0, sizeof A);
  A.lam = lam; A.lam_m = lam_m; A.lk[0] = lk0; A.lk[1] = lk1; A.lk[2] = lk2;
  A.lamB = lamB; A.lamloc = lamloc; A.gh = gh; A.gku = gku;
  A.kumap = c->kumap; A.c_an = ph.c_an; A.c_an_map = ph.c_an_map; A.two_over_Ms = (float)(2.0 / c->Ms);
  A.g1 = ph.g1; A.g2 = ph.g2; A.dt = (float)dt; A.N = N;
  const unsigned nb = (unsigned)((N + 255) / 256);
  // One segment (its start state already in seg_s): recompute it storing every
  // stage state and field, then sweep it backwards.  Enqueued on stream q;
  // returns the kernels launched or < 0.
  const Dims& dA = c->d;
  // A segment's recording: from its start state in seg_s, len RK4 steps with
  // every stage state and field stored (ticks: the steps advance the context's
  // clock and step count, as mm_step's do).  Enqueued on stream q.
  auto enqueue_record = [&](cudaStream_t q, int r, int len, bool ticks, long long* nk) -> int {
    *nk = 0;
    float* const ss = seg_s(r);
    if (launch_xfwd(dA, ss, c->tw, c->S, q) < 0) return mm_fail(c, MM_ECUDA, "adjoint: x-transform launch failed");
    *nk += 1;
    StageArgs a = {};
    a.hmap = c->hmap; a.kumap = c->kumap; a.mode = 1; a.dt = (float)dt; a.acc = c->acc;
    for (int j = 0; j < len; ++j) {
      float* sj = ss + (size_t)4 * j * v3;
      a.m0 = sj;
      for (int st = 0; st < 4; ++st) {
        a.stage = st;
        a.tick = (ticks && st == 0) ? Tick{c->prog, dt, 0} : Tick{};
        a.m_in = sj + st * v3;
        a.m_out = st < 3 ? sj + (st + 1) * v3 : ss + (size_t)4 * (j + 1) * v3;
        a.B_out = seg_B(r) + ((size_t)4 * j + st) * v3;
        const int kk = launch_stage(dA, ph, a, c->tw, c->S, c->Kh, c->dflag, q);
        if (kk < 0) return mm_fail(c, MM_ECUDA, "adjoint: stage kernels failed to launch");
        *nk += kk;
      }
    }
    return MM_OK;
  };
  auto enqueue_sweep = [&](cudaStream_t q, int r, int len, long long* nk) -> int {
    *nk = 0;
    // the reverse sweep of the segment: one pointwise kernel starts its last step
    // (k_adj_start), then per step and stage one y/z pass and one x kernel that
    // applies L to lam_B, closes the stage and opens the next (mode 3); the
    // closing kernel of a step also starts the sweep of the step before it
    // (mode 5), except for the segment's first step (mode 4)
    auto step_fields = [&](int j, const float** sq, const float** Bq) {
      for (int st = 0; st < 4; ++st) {
        sq[st] = seg_s(r) + ((size_t)4 * j + st) * v3;
        Bq[st] = seg_B(r) + ((size_t)4 * j + st) * v3;
      }
    };
    {
      AdjArgs Aj = A;
      step_fields(len - 1, Aj.s, Aj.B);
      k_adj_start<<<nb, 256, 0, q>>>(Aj);
      if (cudaGetLastError() != cudaSuccess) return mm_fail(c, MM_ECUDA, "adjoint kernel launch failed");
      *nk += 1;
    }
    StageArgs x = {};
    x.kumap = c->kumap;
    x.adj_loc = lamloc; x.adj_lam_m = lam_m; x.adj_gh = gh; x.adj_gku = gku; x.adj_lam = lam;
    x.adj_lk0 = lk0; x.adj_dt = (float)dt;
    x.m_in = lamB;
    if (launch_field_part(dA, lin, x, c->tw, c->S, c->Kh, c->dflag, q, 0) < 0)
      return mm_fail(c, MM_ECUDA, "adjoint: x-transform launch failed");
    *nk += 1;
    float* cur = lamB;
    for (int j = len - 1; j >= 0; --j) {
      const float *sq[4], *Bq[4];
      step_fields(j, sq, Bq);
      float* const lks[3] = {lk0, lk1, lk2};
      for (int st = 2; st >= -1; --st) {
        x.m_in = cur;
        x.m_out = cur == lamB ? lamB2 : lamB;
        if (st >= 0) {
          x.mode = 3;
          x.adj_s = sq[st];
          x.adj_B = Bq[st];
          x.adj_lk = lks[st];
          x.adj_c = st == 2 ? (float)dt : 0.5f * (float)dt;   // s_4 = m + dt k_3, s_3 = m + dt/2 k_2, s_2 = m + dt/2 k_1
        } else if (j > 0) {
          x.mode = 5;   // the step's start cotangent, then the previous step's start
          step_fields(j - 1, x.adj_sq, x.adj_Bq);
        } else {
          x.mode = 4;   // the segment's first step: lam = lam_m + ls
          x.m_out = nullptr;
        }
        for (int part = 1; part <= 2; ++part) {
          const int kk = launch_field_part(dA, lin, x, c->tw, c->S, c->Kh, c->dflag, q, part);
          if (kk < 0) return mm_fail(c, MM_ECUDA, "adjoint: field kernels failed to launch");
          *nk += kk;
        }
        if (x.m_out) cur = x.m_out;
      }
    }
    return MM_OK;
  };
  // full-length segments replay captured graphs (rebuilt when the segment
  // length, dt or the context's field, damping or launch shapes changed);
  // graph 0 recomputes into slot 0, 1 + r records slot r in the forward pass,
  // 1 + kAdjSlots + r sweeps slot r
  if (c->adj_graph_len != k || c->adj_graph_dt != dt || c->adj_graph_gen != c->param_gen) drop_adj_graphs(c);
  auto graph_of = [&](int gi) -> int {
    if (c->adj_graph[gi]) return MM_OK;
    cudaGraph_t graph;
    long long nk = 0;
    MM_CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int r = gi == 0 ? enqueue_record(c->cap_stream, 0, k, false, &nk)
                : gi <= kAdjSlots ? enqueue_record(c->cap_stream, gi - 1, k, true, &nk)
                                  : enqueue_sweep(c->cap_stream, gi - 1 - kAdjSlots, k, &nk);
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (r != MM_OK || e != cudaSuccess) {
      cudaGetLastError();
      return r != MM_OK ? r : mm_fail(c, MM_ECUDA, "adjoint: segment capture failed: %s", cudaGetErrorString(e));
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->adj_graph[gi], graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      c->adj_graph[gi] = nullptr;
      return mm_fail(c, MM_ECUDA, "adjoint: segment graph instantiate failed: %s", cudaGetErrorString(ei));
    }
    c->adj_graph_nodes[gi] = nk;
    MM_CK(c, cudaGraphUpload(c->adj_graph[gi], c->stream));
    return MM_OK;
  };
  if ((rc = graph_of(0)) != MM_OK) return rc;
  for (int r = 0; r < R; ++r) {
    if ((rc = graph_of(1 + r)) != MM_OK) return rc;
    if ((rc = graph_of(1 + kAdjSlots + r)) != MM_OK) return rc;
  }
  c->adj_graph_len = k;
  c->adj_graph_dt = dt;
  c->adj_graph_gen = c->param_gen;
  // kind 0: recompute into slot 0, 1: record slot r in the forward pass, 2: sweep slot r
  auto run = [&](int kind, int r, int len) -> int {   // a full-length segment from its graph, else eagerly
    const int gi = kind == 0 ? 0 : kind == 1 ? 1 + r : 1 + kAdjSlots + r;
    if (len == k) {
      MM_CK(c, cudaGraphLaunch(c->adj_graph[gi], s));
      c->launches += c->adj_graph_nodes[gi];
      return MM_OK;
    }
    long long nk = 0;
    const int rr = kind == 2 ? enqueue_sweep(s, r, len, &nk) : enqueue_record(s, r, len, kind == 1, &nk);
    c->launches += nk;
    return rr;
  };

  // 1. forward n steps from the current state, a checkpoint every k steps up to
  //    the recorded segments; the last R segments are recorded on the way (their
  //    stage states and fields are the first the reverse sweep needs), so they
  //    are not recomputed.  Only the last segment can be shorter than k.
  const int g0 = nseg - R;   // first recorded segment
  MM_CK(c, cudaMemcpyAsync(c->adj_ckpt, c->m0, v3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  for (int g = 0; g < g0; ++g) {
    if ((rc = mm_step(c, k, dt)) != MM_OK) return rc;
    MM_CK(c, cudaMemcpyAsync(c->adj_ckpt + (size_t)(g + 1) * v3, c->m0, v3 * sizeof(float),
                             cudaMemcpyDeviceToDevice, s));
  }
  const int len_last = n - (nseg - 1) * k;
  for (int r = 0; r < R; ++r) {
    const float* start = r == 0 ? c->m0 : seg_s(r - 1) + (size_t)4 * k * v3;
    MM_CK(c, cudaMemcpyAsync(seg_s(r), start, v3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    const int len = r == R - 1 ? len_last : k;
    if ((rc = run(1, r, len)) != MM_OK) return rc;
    c->steps += len;
  }
  const float* m_final = seg_s(R - 1) + (size_t)4 * len_last * v3;
  MM_CK(c, cudaMemcpyAsync(c->m0, m_final, v3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  MM_CK(c, cudaMemcpyAsync(c->adj_ckpt + (size_t)nseg * v3, m_final, v3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  // 2. reverse sweep, segment by segment: the recorded slots first, then each
  //    earlier segment recomputed from its checkpoint into slot 0
  MM_CK(c, cudaMemcpyAsync(lam, dL_dm_final, v3 * sizeof(float), cudaMemcpyDefault, s));
  MM_CK(c, cudaMemsetAsync(gh, 0, (v3 + N) * sizeof(float), s));
  for (int g = nseg - 1; g >= 0; --g) {
    const int len = (g + 1) * k <= n ? k : n - g * k;
    int r = g - g0;
    if (g < g0) {
      r = 0;
      MM_CK(c, cudaMemcpyAsync(seg_s(0), c->adj_ckpt + (size_t)g * v3, v3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
      if ((rc = run(0, 0, len)) != MM_OK) return rc;
    }
    if ((rc = run(2, r, len)) != MM_OK) return rc;
  }
  c->s_valid = 0;   // S was used as scratch
  // 3. outputs
  if (dL_dm0) {
    k_tangent<<<nb, 256, 0, s>>>(c->adj_ckpt, lam, N);
    if (cudaGetLastError() != cudaSuccess) return mm_fail(c, MM_ECUDA, "adjoint kernel launch failed");
    c->launches++;
    MM_CK(c, cudaMemcpyAsync(dL_dm0, lam, v3 * sizeof(float), cudaMemcpyDefault, s));
  }
  if (dL_dh) MM_CK(c, cudaMemcpyAsync(dL_dh, gh, v3 * sizeof(float), cudaMemcpyDefault, s));
  if (dL_dku) MM_CK(c, cudaMemcpyAsync(dL_dku, gku, (size_t)N * sizeof(float), cudaMemcpyDefault, s));
  return MM_OK;
}
