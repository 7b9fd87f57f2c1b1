// Vector-Jacobian product of the LLG right-hand side (eq. 2 on unit vectors),
// f(s) = g1 s x B + g2 s x (s x B), shared by the adjoint sweep's pointwise
// kernels (adjoint.cu) and the fused adjoint mode of the x kernel.  For a
// cotangent lk of f at (s, B):
//   lam_B   = g1 (lk x s) + g2 ((lk x s) x s)                (through B)
//   lam_loc = g1 (B x lk) + g2 ((s x B) x lk) + g2 (B x (lk x s)) + c (lam_B)_x x^
// (through s directly and through the anisotropy field c s_x x^, c = 2 Ku / Ms).
#pragma once
#include <cuda_runtime.h>

__device__ __forceinline__ float3 adj_cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ void llg_vjp(float g1, float g2, float c, float3 s, float3 B, float3 lk, float3& lamB,
                                        float3& loc) {
  const float3 lxs = adj_cross(lk, s);
  const float3 lxsxs = adj_cross(lxs, s);
  lamB = make_float3(g1 * lxs.x + g2 * lxsxs.x, g1 * lxs.y + g2 * lxsxs.y, g1 * lxs.z + g2 * lxsxs.z);
  const float3 t1 = adj_cross(B, lk), t2 = adj_cross(adj_cross(s, B), lk), t3 = adj_cross(B, lxs);
  loc = make_float3(g1 * t1.x + g2 * (t2.x + t3.x) + c * lamB.x, g1 * t1.y + g2 * (t2.y + t3.y),
                    g1 * t1.z + g2 * (t2.z + t3.z));
}

// The start of one step's reverse sweep at one cell.  The step ran the stages
// s_q with fields B_q (k_q = f(s_q)) and ended in m' = u / |u|,
// u = s_1 + dt/6 (k_1 + 2 k_2 + 2 k_3 + k_4).  For the cotangent lam of m':
//   lu = (I - m' m'^T) lam / |u|  (the cotangent of u and of the step's start
//   through its identity term), lk_1 = lk_4 = dt/6 lu, lk_2 = lk_3 = dt/3 lu,
// and the VJP of stage 4 at (s_4, B_4, lk_4).
__device__ __forceinline__ void adj_step_start(float g1, float g2, float c, float dt, const float3 (&s)[4],
                                               const float3 (&B)[4], float3 lam, float3& lu, float3& lamB,
                                               float3& loc) {
  float3 k[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float3 sxB = adj_cross(s[q], B[q]);
    const float3 sxsxB = adj_cross(s[q], sxB);
    k[q] = make_float3(g1 * sxB.x + g2 * sxsxB.x, g1 * sxB.y + g2 * sxsxB.y, g1 * sxB.z + g2 * sxsxB.z);
  }
  const float h = dt * (1.0f / 6.0f);
  const float3 u = make_float3(s[0].x + h * (k[0].x + 2.f * k[1].x + 2.f * k[2].x + k[3].x),
                               s[0].y + h * (k[0].y + 2.f * k[1].y + 2.f * k[2].y + k[3].y),
                               s[0].z + h * (k[0].z + 2.f * k[1].z + 2.f * k[2].z + k[3].z));
  const float inv = 1.0f / sqrtf(u.x * u.x + u.y * u.y + u.z * u.z);
  const float3 mn = make_float3(inv * u.x, inv * u.y, inv * u.z);
  const float d = mn.x * lam.x + mn.y * lam.y + mn.z * lam.z;
  lu = make_float3(inv * (lam.x - d * mn.x), inv * (lam.y - d * mn.y), inv * (lam.z - d * mn.z));
  llg_vjp(g1, g2, c, s[3], B[3], make_float3(h * lu.x, h * lu.y, h * lu.z), lamB, loc);
}
