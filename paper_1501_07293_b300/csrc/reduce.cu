// Energies (eq. 1 on the grid) and observables, accumulated in FP64.
//
// Per cell, with B = mu0 H in tesla:
//   exchange   A delta |m_i - m_j|^2 over the +x, +y, +z neighbour pairs
//              (the discrete energy whose gradient is the eq. 5/7 stencil)
//   anisotropy Ku delta^3 (m_y^2 + m_z^2)                 (easy axis x)
//   demag      -1/2 mu0 delta^3 Ms m . H_demag
//   Zeeman     -delta^3 Ms m . (b_ext + h)
//   sum of m (for the mean) and |dm/dt| from eq. 2 with the full field.
// Each block writes its partial sums; k_reduce_final adds them in a fixed
// order, so the result does not depend on scheduling.
#include "common.cuh"

#define NRED 9

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

struct RedParams {
  double A_delta;     // A delta
  double Ku_d3;       // Ku delta^3 (scalar Ku)
  double d3;          // delta^3
  double demag_pref;  // -1/2 mu0 delta^3 Ms
  double zee_pref;    // -delta^3 Ms
};

__global__ void __launch_bounds__(256) k_reduce(const float* __restrict__ m, const float* __restrict__ Hd,
                                                const float* __restrict__ hmap, const float* __restrict__ kumap,
                                                Dims d, Phys ph, const float* __restrict__ drive, RedParams rp,
                                                double* __restrict__ partials) {
  if (drive) { ph.bx = drive[0]; ph.by = drive[1]; ph.bz = drive[2]; ph.g1 = drive[3]; ph.g2 = drive[4]; }
  double acc[NRED];
#pragma unroll
  for (int j = 0; j < NRED; ++j) acc[j] = 0.0;
  const long long N = d.N;
  const float mu0 = (float)MM_MU0;
  for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < N;
       cell += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(cell % d.nx);
    const int y = (int)((cell / d.nx) % d.ny);
    const int z = (int)(cell / ((long long)d.nx * d.ny));
    const float mx = m[cell], my = m[cell + N], mz = m[cell + 2 * N];
    if (!isfinite(mx) || !isfinite(my) || !isfinite(mz)) { acc[8] += 1.0; continue; }
    // exchange pairs with the +x, +y, +z neighbours; sums of m_nb - m for the field
    double pair = 0.0;
    float lx = 0.f, ly = 0.f, lz = 0.f;
    const long long off[6] = {x > 0 ? -1 : 0, x < d.nx - 1 ? 1 : 0,
                              y > 0 ? -(long long)d.nx : 0, y < d.ny - 1 ? (long long)d.nx : 0,
                              z > 0 ? -(long long)d.nx * d.ny : 0, z < d.nz - 1 ? (long long)d.nx * d.ny : 0};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const long long j = cell + off[q];
      const float ax = m[j] - mx, ay = m[j + N] - my, az = m[j + 2 * N] - mz;
      lx += ax; ly += ay; lz += az;
      if ((q & 1) && off[q] != 0) pair += (double)ax * ax + (double)ay * ay + (double)az * az;
    }
    acc[0] += pair;
    const double ku = kumap ? (double)kumap[cell] : -1.0;
    acc[1] += (kumap ? ku : 1.0) * ((double)my * my + (double)mz * mz);
    const float hdx = Hd[cell], hdy = Hd[cell + N], hdz = Hd[cell + 2 * N];
    acc[2] += (double)mx * hdx + (double)my * hdy + (double)mz * hdz;
    float bx = ph.bx, by = ph.by, bz = ph.bz;
    if (hmap) { bx += hmap[cell]; by += hmap[cell + N]; bz += hmap[cell + 2 * N]; }
    acc[3] += (double)mx * bx + (double)my * by + (double)mz * bz;
    acc[4] += mx; acc[5] += my; acc[6] += mz;
    // |dm/dt| with the full effective field
    const float can = kumap ? ph.c_an_map * kumap[cell] : ph.c_an;
    const float Bx = ph.c_ex * lx + can * mx + mu0 * hdx + bx;
    const float By = ph.c_ex * ly + mu0 * hdy + by;
    const float Bz = ph.c_ex * lz + mu0 * hdz + bz;
    const float cx = my * Bz - mz * By, cy = mz * Bx - mx * Bz, cz = mx * By - my * Bx;
    const float dx = my * cz - mz * cy, dy = mz * cx - mx * cz, dz = mx * cy - my * cx;
    const float tx = ph.g1 * cx + ph.g2 * dx, ty = ph.g1 * cy + ph.g2 * dy, tz = ph.g1 * cz + ph.g2 * dz;
    const double t = sqrt((double)tx * tx + (double)ty * ty + (double)tz * tz);
    acc[7] = fmax(acc[7], t);
  }
  // scale into joules / final units before the block reduction
  acc[0] *= rp.A_delta;
  acc[1] *= (kumap ? rp.d3 : rp.Ku_d3);
  acc[2] *= rp.demag_pref;
  acc[3] *= rp.zee_pref;
  __shared__ double sh[8][NRED];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NRED; ++j) {
    const double v = (j == 7) ? warp_max(acc[j]) : warp_sum(acc[j]);
    if (lane == 0) sh[w][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < NRED) {
    const int j = threadIdx.x;
    double v = sh[0][j];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) v = (j == 7) ? fmax(v, sh[q][j]) : v + sh[q][j];
    partials[(long long)blockIdx.x * NRED + j] = v;
  }
}

__global__ void k_reduce_final(const double* __restrict__ partials, int nblocks, double invN,
                               double* __restrict__ out, int* flag) {
  const int j = threadIdx.x;
  if (j >= NRED) return;
  double v = partials[j];
  for (int b = 1; b < nblocks; ++b) {
    const double u = partials[(long long)b * NRED + j];
    v = (j == 7) ? fmax(v, u) : v + u;
  }
  if (j >= 4 && j <= 6) v *= invN;
  out[j] = v;
  if (j == 8 && v > 0.0) atomicOr(flag, 1);
}

int launch_reduce(const Dims& d, const Phys& ph, const float* drive, const float* m, const float* Hd, const float* hmap,
                  const float* kumap, double A, double Ku, double delta, double Ms, double* partials,
                  int nblocks, double* out, int* flag, cudaStream_t s) {
  RedParams rp;
  rp.A_delta = A * delta;
  rp.d3 = delta * delta * delta;
  rp.Ku_d3 = Ku * rp.d3;
  rp.demag_pref = -0.5 * MM_MU0 * rp.d3 * Ms;
  rp.zee_pref = -rp.d3 * Ms;
  k_reduce<<<nblocks, 256, 0, s>>>(m, Hd, hmap, kumap, d, ph, drive, rp, partials);
  if (cudaGetLastError() != cudaSuccess) return -1;
  k_reduce_final<<<1, 32, 0, s>>>(partials, nblocks, 1.0 / (double)d.N, out, flag);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return 2;
}
