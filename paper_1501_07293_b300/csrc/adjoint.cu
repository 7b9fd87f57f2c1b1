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
// swept in reverse.
#include <string.h>

#include "common.cuh"

struct AdjArgs {
  const float* s[4];   // stage input states of the step
  const float* B[4];   // their fields (tesla)
  float* lam;          // in: cotangent of m' (start); out: cotangent of m (finish)
  float* lam_m;        // running cotangent of m
  float* lk[3];        // cotangents of k_1, k_2, k_3
  float* lamB;         // cotangent of B at the current stage (input of the linear operator)
  float* lamloc;       // local part of the cotangent of the current stage state
  const float* LlamB;  // L applied to lamB (tesla)
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

__device__ __forceinline__ float3 rhs(const AdjArgs& A, float3 s, float3 B) {
  const float3 sxB = xp3(s, B);
  return add3(sc3(A.g1, sxB), sc3(A.g2, xp3(s, sxB)));
}

// vector-Jacobian product of f at (s, B) with cotangent lk; accumulates dL/dh, dL/dKu
__device__ __forceinline__ void vjp_stage(const AdjArgs& A, long long i, float3 s, float3 B, float3 lk) {
  const float3 lxs = xp3(lk, s);
  const float3 lamB = add3(sc3(A.g1, lxs), sc3(A.g2, xp3(lxs, s)));
  float3 loc = add3(add3(sc3(A.g1, xp3(B, lk)), sc3(A.g2, xp3(xp3(s, B), lk))), sc3(A.g2, xp3(B, lxs)));
  const float c = A.kumap ? A.c_an_map * A.kumap[i] : A.c_an;
  loc.x += c * lamB.x;
  st3v(A.lamB, A.N, i, lamB);
  st3v(A.lamloc, A.N, i, loc);
  st3v(A.gh, A.N, i, add3(ld3v(A.gh, A.N, i), lamB));
  A.gku[i] += A.two_over_Ms * s.x * lamB.x;
}

__global__ void k_adj_start(AdjArgs A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  float3 s[4], B[4], k[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    s[q] = ld3v(A.s[q], A.N, i);
    B[q] = ld3v(A.B[q], A.N, i);
    k[q] = rhs(A, s[q], B[q]);
  }
  const float h = A.dt * (1.0f / 6.0f);
  const float3 u = make_float3(s[0].x + h * (k[0].x + 2.f * k[1].x + 2.f * k[2].x + k[3].x),
                               s[0].y + h * (k[0].y + 2.f * k[1].y + 2.f * k[2].y + k[3].y),
                               s[0].z + h * (k[0].z + 2.f * k[1].z + 2.f * k[2].z + k[3].z));
  const float nu = sqrtf(u.x * u.x + u.y * u.y + u.z * u.z);
  const float inv = 1.0f / nu;
  const float3 mn = sc3(inv, u);
  const float3 lam = ld3v(A.lam, A.N, i);
  const float d = mn.x * lam.x + mn.y * lam.y + mn.z * lam.z;
  const float3 lu = sc3(inv, make_float3(lam.x - d * mn.x, lam.y - d * mn.y, lam.z - d * mn.z));
  st3v(A.lam_m, A.N, i, lu);
  st3v(A.lk[0], A.N, i, sc3(h, lu));
  st3v(A.lk[1], A.N, i, sc3(2.f * h, lu));
  st3v(A.lk[2], A.N, i, sc3(2.f * h, lu));
  vjp_stage(A, i, s[3], B[3], sc3(h, lu));
}

// Close stage `st` + 1 (its lamloc + L lamB is the cotangent of its state), then open stage `st`.
__global__ void k_adj_stage(AdjArgs A, int st) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const float3 ls = add3(ld3v(A.lamloc, A.N, i), ld3v(A.LlamB, A.N, i));
  st3v(A.lam_m, A.N, i, add3(ld3v(A.lam_m, A.N, i), ls));
  const float c = (st == 2) ? A.dt : 0.5f * A.dt;   // s_4 = m + dt k_3, s_3 = m + dt/2 k_2, s_2 = m + dt/2 k_1
  float* lkp = A.lk[st];
  const float3 lk = add3(ld3v(lkp, A.N, i), sc3(c, ls));
  st3v(lkp, A.N, i, lk);
  vjp_stage(A, i, ld3v(A.s[st], A.N, i), ld3v(A.B[st], A.N, i), lk);
}

__global__ void k_adj_finish(AdjArgs A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const float3 ls = add3(ld3v(A.lamloc, A.N, i), ld3v(A.LlamB, A.N, i));
  st3v(A.lam, A.N, i, add3(ld3v(A.lam_m, A.N, i), ls));
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

void mm_adjoint_free(mm_ctx* c) {
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
  int rc;
  if ((rc = grow(c, &c->adj_ckpt, &c->adj_ckpt_cap, (size_t)(nseg + 1) * v3)) != MM_OK) return rc;
  if ((rc = grow(c, &c->adj_seg, &c->adj_seg_cap, (size_t)(8 * k + 1) * v3)) != MM_OK) return rc;
  if ((rc = grow(c, &c->adj_work, &c->adj_work_cap, 9 * v3 + (size_t)N)) != MM_OK) return rc;
  float* W = c->adj_work;
  float *lam = W, *lam_m = W + v3, *lk0 = W + 2 * v3, *lk1 = W + 3 * v3, *lk2 = W + 4 * v3;
  float *lamB = W + 5 * v3, *lamloc = W + 6 * v3, *LlamB = W + 7 * v3, *gh = W + 8 * v3, *gku = W + 9 * v3;
  float* seg_s = c->adj_seg;                   // [k][4][3N] stage states, then [1][3N] the segment's end
  float* seg_B = c->adj_seg + (size_t)(4 * k + 1) * v3;   // [k][4][3N] fields
  cudaStream_t s = c->stream;

  // 1. forward n steps from the current state, keeping a checkpoint every k steps
  MM_CK(c, cudaMemcpyAsync(c->adj_ckpt, c->m0, v3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  for (int g = 0; g < nseg; ++g) {
    const int len = (g + 1) * k <= n ? k : n - g * k;
    if ((rc = mm_step(c, len, dt)) != MM_OK) return rc;
    MM_CK(c, cudaMemcpyAsync(c->adj_ckpt + (size_t)(g + 1) * v3, c->m0, v3 * sizeof(float),
                             cudaMemcpyDeviceToDevice, s));
  }
  // 2. reverse sweep
  MM_CK(c, cudaMemcpyAsync(lam, dL_dm_final, v3 * sizeof(float), cudaMemcpyDefault, s));
  MM_CK(c, cudaMemsetAsync(gh, 0, (v3 + N) * sizeof(float), s));
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
  A.lamB = lamB; A.lamloc = lamloc; A.LlamB = LlamB; A.gh = gh; A.gku = gku;
  A.kumap = c->kumap; A.c_an = ph.c_an; A.c_an_map = ph.c_an_map; A.two_over_Ms = (float)(2.0 / c->Ms);
  A.g1 = ph.g1; A.g2 = ph.g2; A.dt = (float)dt; A.N = N;
  const unsigned nb = (unsigned)((N + 255) / 256);
  StageArgs L = {};
  L.m_in = lamB; L.H_out = LlamB; L.mode = 0; L.mask = MM_TERM_EXCHANGE | MM_TERM_DEMAG;
  auto apply_L = [&]() -> int {
    const int kk = launch_field_eval(c->d, lin, L, c->tw, c->S, c->Kh, c->dflag, s);
    if (kk < 0) return mm_fail(c, MM_ECUDA, "adjoint: field kernels failed to launch");
    c->launches += kk;
    return MM_OK;
  };
  for (int g = nseg - 1; g >= 0; --g) {
    const int len = (g + 1) * k <= n ? k : n - g * k;
    // recompute the segment, storing every stage state and field
    float* m_start = seg_s;
    MM_CK(c, cudaMemcpyAsync(m_start, c->adj_ckpt + (size_t)g * v3, v3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (launch_xfwd(c->d, m_start, c->tw, c->S, s) < 0) return mm_fail(c, MM_ECUDA, "adjoint: x-transform launch failed");
    c->launches++;
    StageArgs a = {};
    a.hmap = c->hmap; a.kumap = c->kumap; a.mode = 1; a.dt = (float)dt; a.acc = c->acc;
    for (int j = 0; j < len; ++j) {
      float* sj = seg_s + (size_t)4 * j * v3;
      a.m0 = sj;
      for (int st = 0; st < 4; ++st) {
        a.stage = st;
        a.m_in = sj + st * v3;
        a.m_out = st < 3 ? sj + (st + 1) * v3 : seg_s + (size_t)4 * (j + 1) * v3;
        a.B_out = seg_B + ((size_t)4 * j + st) * v3;
        const int kk = launch_stage(c->d, ph, a, c->tw, c->S, c->Kh, c->dflag, s);
        if (kk < 0) return mm_fail(c, MM_ECUDA, "adjoint: stage kernels failed to launch");
        c->launches += kk;
      }
    }
    // sweep the segment backwards
    for (int j = len - 1; j >= 0; --j) {
      for (int st = 0; st < 4; ++st) {
        A.s[st] = seg_s + ((size_t)4 * j + st) * v3;
        A.B[st] = seg_B + ((size_t)4 * j + st) * v3;
      }
      k_adj_start<<<nb, 256, 0, s>>>(A);
      if (cudaGetLastError() != cudaSuccess) return mm_fail(c, MM_ECUDA, "adjoint kernel launch failed");
      c->launches++;
      for (int st = 2; st >= 0; --st) {
        if ((rc = apply_L()) != MM_OK) return rc;
        k_adj_stage<<<nb, 256, 0, s>>>(A, st);
        if (cudaGetLastError() != cudaSuccess) return mm_fail(c, MM_ECUDA, "adjoint kernel launch failed");
        c->launches++;
      }
      if ((rc = apply_L()) != MM_OK) return rc;
      k_adj_finish<<<nb, 256, 0, s>>>(A);
      if (cudaGetLastError() != cudaSuccess) return mm_fail(c, MM_ECUDA, "adjoint kernel launch failed");
      c->launches++;
    }
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
