// Effective field and LLG stage kernels (FP32).  One field evaluation is three
// launches:
//
//  k_xfwd  (per row tile)   real-to-complex transform of m along x, zero padded
//                           from nx to px (eq. 14 / Fig. 1), through a complex
//                           transform of half length; writes S[kx][c][z][y].
//  k_yz    (per kx column)  forward transform along y (zero padded ny -> py),
//                           the demag product of eq. 14 -- along z a direct
//                           Toeplitz sum over the nz planes with the kernel
//                           transformed along x and y only -- and the inverse
//                           transform along y, keeping the first ny rows.
//  k_xinv  (per row tile)   complex-to-real inverse along x (first nx points),
//                           then per cell: demag + exchange (eq. 5, Neumann rule
//                           eq. 7) + anisotropy (eq. 8) + Zeeman, and either the
//                           field itself or the LLG right-hand side (eq. 2) with
//                           the RK4 / Euler update and renormalisation.
#include <stdio.h>

#include "common.cuh"
#include "fft.cuh"

// ---------------------------------------------------------------------------
// k_xfwd: CTA = (tile of TY rows along y, plane z, component c)
// ---------------------------------------------------------------------------
template <int HALF>
__global__ void __launch_bounds__(512) k_xfwd(const float* __restrict__ m, float2* __restrict__ S,
                                              const float2* __restrict__ twP, Dims d, int TY) {
  const int c = blockIdx.z, z = blockIdx.y, y0 = blockIdx.x * TY;
  if constexpr (HALF == 0) {
    // px = 1 (nx = 1): the transform along x is the identity.
    for (int r = threadIdx.x; r < TY; r += blockDim.x) {
      const int y = y0 + r;
      if (y < d.ny) {
        const float v = m[(long long)c * d.N + (long long)z * d.ny + y];
        S[((long long)c * d.nz + z) * d.ny + y] = make_float2(v, 0.f);
      }
    }
  } else {
    constexpr int T = TeamOf<HALF>::v;
    constexpr int P = 2 * HALF;
    constexpr int RS = HALF + 1;
    extern __shared__ float2 sm[];
    float2* tws = sm;       // exp(-2 pi i m / P), m < P
    float2* rows = sm + P;  // TY rows of HALF complex (+1 pad)
    for (int i = threadIdx.x; i < P; i += blockDim.x) tws[i] = twP[i];
    const int lane = threadIdx.x & 31;
    const int team = threadIdx.x / T, t = threadIdx.x % T, nteams = blockDim.x / T;
    const unsigned mask = team_mask<T>(lane);
    __syncthreads();
    for (int r = team; r < TY; r += nteams) {
      const int y = y0 + r;
      if (y >= d.ny) continue;
      float2* row = rows + r * RS;
      const float* src = m + (long long)c * d.N + ((long long)z * d.ny + y) * d.nx;
      // pack z[n] = x[2n] + i x[2n+1]; x is zero beyond nx (the zero padding)
      for (int n = t; n < HALF; n += T) {
        const float a = (2 * n < d.nx) ? __ldg(src + 2 * n) : 0.f;
        const float b = (2 * n + 1 < d.nx) ? __ldg(src + 2 * n + 1) : 0.f;
        row[n] = make_float2(a, b);
      }
      __syncwarp(mask);
      team_fft<HALF, T, -1, 2>(row, t, mask, tws);
    }
    __syncthreads();
    // X[k] = 1/2 (Z[k] + conj Z[-k]) - i/2 W_P^k (Z[k] - conj Z[-k]),  k = 0..HALF
    const int total = (HALF + 1) * TY;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int r = i % TY, k = i / TY;
      const int y = y0 + r;
      if (y >= d.ny) continue;
      const float2* row = rows + r * RS;
      const float2 zk = row[k & (HALF - 1)];
      const float2 zc = cconj(row[(HALF - k) & (HALF - 1)]);
      const float2 dif = csub(zk, zc);
      const float2 o = cmul(make_float2(dif.y, -dif.x), tws[k]);
      const float2 X = cscale(cadd(cadd(zk, zc), o), 0.5f);
      S[(((long long)k * 3 + c) * d.nz + z) * d.ny + y] = X;
    }
  }
}

// ---------------------------------------------------------------------------
// k_yz: CTA = one kx column, all 3 components and nz planes in shared memory
// ---------------------------------------------------------------------------
__constant__ int c_pair[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};

template <int PY, int NZM>
__global__ void __launch_bounds__(512, 1) k_yz(float2* __restrict__ S, const float* __restrict__ Kh,
                                                const float2* __restrict__ twY, Dims d) {
  constexpr int T = TeamOf<PY>::v;
  extern __shared__ float2 sm[];
  float2* tws = sm;        // exp(-2 pi i m / PY), m < PY
  float2* buf = sm + PY;   // [3 nz][PY]
  const int kx = blockIdx.x;
  const int nz = d.nz, ny = d.ny;
  const int NP = 3 * nz;
  float2* Sk = S + (long long)kx * NP * ny;
  for (int i = threadIdx.x; i < PY; i += blockDim.x) tws[i] = twY[i];
  for (int i = threadIdx.x; i < NP * PY; i += blockDim.x) {
    const int p = i / PY, y = i % PY;
    buf[i] = (y < ny) ? Sk[(long long)p * ny + y] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int team = threadIdx.x / T, t = threadIdx.x % T, nteams = blockDim.x / T;
  const unsigned mask = team_mask<T>(lane);
  if (PY > 1) {
    for (int p = team; p < NP; p += nteams) team_fft<PY, T, -1, 1>(buf + p * PY, t, mask, tws);
    __syncthreads();
  }

  // Product of eq. 14: H_a(kz) = sum_b sum_kz' Kt_ab(kx, ky, kz - kz') M_b(kz').
  // Each round takes a chunk of ky values and all three output components of
  // them, so every input of a ky is read before any output of it is written.
  const float* Kk = Kh + (long long)kx * 6 * nz * d.hy;
  int chunk = (int)(blockDim.x / 3) & ~31;
  if (chunk < 1) chunk = (int)(blockDim.x / 3);
  if (chunk > PY) chunk = PY;
  const int rounds = (PY + chunk - 1) / chunk;
  for (int rd = 0; rd < rounds; ++rd) {
    const int t3 = threadIdx.x;
    const int a = t3 / chunk;
    const int ky = rd * chunk + t3 % chunk;
    const bool act = a < 3 && ky < PY;
    float2 out[NZM];
#pragma unroll
    for (int q = 0; q < NZM; ++q) out[q] = make_float2(0.f, 0.f);
    if (act) {
      int kyf = ky;
      bool mirrored = false;
      if (ky > PY / 2) { kyf = PY - ky; mirrored = true; }
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int p = c_pair[a][b];
        const bool odd_y = (p == 3 || p == 5);
        const bool odd_z = (p == 4 || p == 5);
        const bool imag = (p == 4 || p == 5);
        const float ys = (mirrored && odd_y) ? -1.f : 1.f;
        float kr[NZM];
#pragma unroll
        for (int q = 0; q < NZM; ++q)
          kr[q] = (q < nz) ? ys * __ldg(Kk + ((long long)p * nz + q) * d.hy + kyf) : 0.f;
#pragma unroll
        for (int zi = 0; zi < NZM; ++zi) {
          if (zi < nz) {
            float2 mv = buf[(b * nz + zi) * PY + ky];
            if (imag) mv = cmuli(mv);
            const float2 mn = odd_z ? make_float2(-mv.x, -mv.y) : mv;  // kernel at negative offset
#pragma unroll
            for (int zo = 0; zo < NZM; ++zo) {
              if (zo < nz) {
                const float kv = (zo >= zi) ? kr[zo - zi] : kr[zi - zo];
                const float2 src = (zo >= zi) ? mv : mn;
                out[zo].x = fmaf(kv, src.x, out[zo].x);
                out[zo].y = fmaf(kv, src.y, out[zo].y);
              }
            }
          }
        }
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int zo = 0; zo < NZM; ++zo)
        if (zo < nz) buf[(a * nz + zo) * PY + ky] = out[zo];
    }
    __syncthreads();
  }

  if (PY > 1) {
    for (int p = team; p < NP; p += nteams) team_fft<PY, T, 1, 1>(buf + p * PY, t, mask, tws);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < NP * ny; i += blockDim.x) {
    const int p = i / ny, y = i % ny;
    Sk[i] = buf[p * PY + y];
  }
}

// ---------------------------------------------------------------------------
// per-cell field terms and LLG update
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 ld3(const float* __restrict__ m, long long N, long long i) {
  return make_float3(__ldg(m + i), __ldg(m + i + N), __ldg(m + i + 2 * N));
}

// plain (coherent) loads for buffers the same kernel also writes
__device__ __forceinline__ float3 ld3p(const float* m, long long N, long long i) {
  return make_float3(m[i], m[i + N], m[i + 2 * N]);
}

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Finish one cell given its demag field bd (tesla).
__device__ __forceinline__ void cell_update(const StageArgs& a, const Phys& ph, const Dims& d,
                                            int x, int y, int z, float3 bd) {
  const long long N = d.N;
  const long long cell = ((long long)z * d.ny + y) * d.nx + x;
  const float* mi = a.m_in;
  const float3 m = ld3(mi, N, cell);
  // eq. 5 with eq. 7: a missing neighbour is the cell itself (clamped index)
  const long long xm = cell - (x > 0 ? 1 : 0), xp = cell + (x < d.nx - 1 ? 1 : 0);
  const long long row = d.nx, pl = (long long)d.nx * d.ny;
  const long long ym = cell - (y > 0 ? row : 0), yp = cell + (y < d.ny - 1 ? row : 0);
  const long long zm = cell - (z > 0 ? pl : 0), zp = cell + (z < d.nz - 1 ? pl : 0);
  float3 lap;
  {
    const float3 a1 = ld3(mi, N, xm), a2 = ld3(mi, N, xp), a3 = ld3(mi, N, ym);
    const float3 a4 = ld3(mi, N, yp), a5 = ld3(mi, N, zm), a6 = ld3(mi, N, zp);
    lap.x = ((a1.x - m.x) + (a2.x - m.x)) + ((a3.x - m.x) + (a4.x - m.x)) + ((a5.x - m.x) + (a6.x - m.x));
    lap.y = ((a1.y - m.y) + (a2.y - m.y)) + ((a3.y - m.y) + (a4.y - m.y)) + ((a5.y - m.y) + (a6.y - m.y));
    lap.z = ((a1.z - m.z) + (a2.z - m.z)) + ((a3.z - m.z) + (a4.z - m.z)) + ((a5.z - m.z) + (a6.z - m.z));
  }
  const float3 bex = make_float3(ph.c_ex * lap.x, ph.c_ex * lap.y, ph.c_ex * lap.z);
  const float can = a.kumap ? ph.c_an_map * __ldg(a.kumap + cell) : ph.c_an;
  const float ban = can * m.x;
  float3 bz = make_float3(ph.bx, ph.by, ph.bz);
  if (a.hmap) {
    bz.x += __ldg(a.hmap + cell);
    bz.y += __ldg(a.hmap + cell + N);
    bz.z += __ldg(a.hmap + cell + 2 * N);
  }
  if (a.mode == 0) {
    float3 B = make_float3(0.f, 0.f, 0.f);
    if (a.mask & MM_TERM_EXCHANGE) { B.x += bex.x; B.y += bex.y; B.z += bex.z; }
    if (a.mask & MM_TERM_ANISOTROPY) { B.x += ban; }
    if (a.mask & MM_TERM_DEMAG) { B.x += bd.x; B.y += bd.y; B.z += bd.z; }
    if (a.mask & MM_TERM_ZEEMAN) { B.x += bz.x; B.y += bz.y; B.z += bz.z; }
    a.H_out[cell] = B.x * ph.inv_mu0;
    a.H_out[cell + N] = B.y * ph.inv_mu0;
    a.H_out[cell + 2 * N] = B.z * ph.inv_mu0;
    return;
  }
  const float3 B = make_float3(bex.x + ban + bd.x + bz.x, bex.y + bd.y + bz.y, bex.z + bd.z + bz.z);
  // eq. 2 on the unit vector: dm/dt = g1 m x B + g2 m x (m x B)
  const float3 mxB = cross3(m, B);
  const float3 mxmxB = cross3(m, mxB);
  const float3 k = make_float3(ph.g1 * mxB.x + ph.g2 * mxmxB.x, ph.g1 * mxB.y + ph.g2 * mxmxB.y,
                               ph.g1 * mxB.z + ph.g2 * mxmxB.z);
  float3 nm;
  bool renorm = false;
  if (a.mode == 2) {
    nm = make_float3(m.x + a.dt * k.x, m.y + a.dt * k.y, m.z + a.dt * k.z);
    renorm = true;
  } else {
    const float3 m0 = ld3p(a.m0, N, cell);
    if (a.stage == 0) {
      a.acc[cell] = k.x; a.acc[cell + N] = k.y; a.acc[cell + 2 * N] = k.z;
      const float h = 0.5f * a.dt;
      nm = make_float3(m0.x + h * k.x, m0.y + h * k.y, m0.z + h * k.z);
    } else if (a.stage < 3) {
      float3 s = make_float3(a.acc[cell], a.acc[cell + N], a.acc[cell + 2 * N]);
      s.x = fmaf(2.f, k.x, s.x); s.y = fmaf(2.f, k.y, s.y); s.z = fmaf(2.f, k.z, s.z);
      a.acc[cell] = s.x; a.acc[cell + N] = s.y; a.acc[cell + 2 * N] = s.z;
      const float h = (a.stage == 1) ? 0.5f * a.dt : a.dt;
      nm = make_float3(m0.x + h * k.x, m0.y + h * k.y, m0.z + h * k.z);
    } else {
      const float3 s = make_float3(a.acc[cell] + k.x, a.acc[cell + N] + k.y, a.acc[cell + 2 * N] + k.z);
      const float h = a.dt * (1.0f / 6.0f);
      nm = make_float3(m0.x + h * s.x, m0.y + h * s.y, m0.z + h * s.z);
      renorm = true;
    }
  }
  if (renorm) {
    const float inv = rsqrtf(nm.x * nm.x + nm.y * nm.y + nm.z * nm.z);
    nm.x *= inv; nm.y *= inv; nm.z *= inv;
  }
  a.m_out[cell] = nm.x;
  a.m_out[cell + N] = nm.y;
  a.m_out[cell + 2 * N] = nm.z;
}

// ---------------------------------------------------------------------------
// k_xinv: CTA = (tile of TY rows along y, plane z), all three components
// ---------------------------------------------------------------------------
template <int HALF>
__global__ void __launch_bounds__(512) k_xinv(StageArgs a, Phys ph, const float2* __restrict__ S,
                                              const float2* __restrict__ twP, Dims d, int TY) {
  const int z = blockIdx.y, y0 = blockIdx.x * TY;
  if constexpr (HALF == 0) {
    for (int r = threadIdx.x; r < TY; r += blockDim.x) {
      const int y = y0 + r;
      if (y >= d.ny) continue;
      float3 bd;
      bd.x = ph.c_d * S[((long long)0 * d.nz + z) * d.ny + y].x;
      bd.y = ph.c_d * S[((long long)1 * d.nz + z) * d.ny + y].x;
      bd.z = ph.c_d * S[((long long)2 * d.nz + z) * d.ny + y].x;
      cell_update(a, ph, d, 0, y, z, bd);
    }
  } else {
    constexpr int T = TeamOf<HALF>::v;
    constexpr int P = 2 * HALF;
    constexpr int RS = HALF + 2;
    extern __shared__ float2 sm[];
    float2* tws = sm;
    float2* rows = sm + P;   // [3][TY] rows of HALF+1 spectrum values
    for (int i = threadIdx.x; i < P; i += blockDim.x) tws[i] = twP[i];
    const int total = (HALF + 1) * 3 * TY;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int r = i % TY, rest = i / TY;
      const int c = rest % 3, k = rest / 3;
      const int y = y0 + r;
      float2 v = make_float2(0.f, 0.f);
      if (y < d.ny) v = S[(((long long)k * 3 + c) * d.nz + z) * d.ny + y];
      rows[(c * TY + r) * RS + k] = v;
    }
    __syncthreads();
    // Z[k] = (X[k] + conj X[HALF-k]) + i W_P^{-k} (X[k] - conj X[HALF-k]), k < HALF,
    // so that the half-length inverse gives P (x[2n] + i x[2n+1]).
    const int NR = 3 * TY;
    const int npair = HALF / 2 + 1;
    for (int i = threadIdx.x; i < NR * npair; i += blockDim.x) {
      const int rr = i / npair, k = i % npair;
      float2* row = rows + rr * RS;
      const int k2 = HALF - k;
      const float2 Xa = row[k], Xb = row[k2];
      const float2 w = tws[k];
      const float2 wm = make_float2(w.x, -w.y);   // W_P^{-k}
      const float2 Za = cadd(cadd(Xa, cconj(Xb)), cmuli(cmul(csub(Xa, cconj(Xb)), wm)));
      if (k == 0 || k == k2) {
        row[k] = Za;
      } else {
        const float2 wm2 = make_float2(-w.x, -w.y);  // W_P^{-(HALF-k)} = -W_P^{k}
        const float2 Zb = cadd(cadd(Xb, cconj(Xa)), cmuli(cmul(csub(Xb, cconj(Xa)), wm2)));
        row[k] = Za;
        row[k2] = Zb;
      }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int team = threadIdx.x / T, t = threadIdx.x % T, nteams = blockDim.x / T;
    const unsigned mask = team_mask<T>(lane);
    for (int rr = team; rr < NR; rr += nteams) team_fft<HALF, T, 1, 2>(rows + rr * RS, t, mask, tws);
    __syncthreads();
    for (int i = threadIdx.x; i < TY * d.nx; i += blockDim.x) {
      const int r = i / d.nx, x = i % d.nx;
      const int y = y0 + r;
      if (y >= d.ny) continue;
      float3 bd;
      bd.x = ph.c_d * reinterpret_cast<const float*>(rows + (0 * TY + r) * RS)[x];
      bd.y = ph.c_d * reinterpret_cast<const float*>(rows + (1 * TY + r) * RS)[x];
      bd.z = ph.c_d * reinterpret_cast<const float*>(rows + (2 * TY + r) * RS)[x];
      cell_update(a, ph, d, x, y, z, bd);
    }
  }
}

// ---------------------------------------------------------------------------
// k_normalise: m <- m / |m|; flags zero or non-finite vectors
// ---------------------------------------------------------------------------
__global__ void k_normalise(float* __restrict__ m, long long N, int* flag) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float x = m[i], y = m[i + N], z = m[i + 2 * N];
  const float n2 = x * x + y * y + z * z;
  if (!(n2 > 0.f) || !isfinite(n2)) {
    atomicOr(flag, 1);
    return;
  }
  const float inv = rsqrtf(n2);
  m[i] = x * inv;
  m[i + N] = y * inv;
  m[i + 2 * N] = z * inv;
}

// ---------------------------------------------------------------------------
// launch geometry and dispatch
// ---------------------------------------------------------------------------
static int pow2_ceil(int v) {
  int p = 1;
  while (p < v) p *= 2;
  return p;
}

static int nzm_of(int nz) { return pow2_ceil(nz); }

static int xtile(int half) { return half <= 256 ? 16 : (half <= 512 ? 8 : 4); }
static int xinv_tile(int half) { return half <= 128 ? 8 : (half <= 256 ? 8 : (half <= 512 ? 4 : 2)); }

static size_t yz_smem(const Dims& d) { return sizeof(float2) * ((size_t)d.py + 3ull * d.nz * d.py); }

static const size_t kMaxSmem = 227 * 1024;

int mm_supported(const Dims& d, char* why, int nwhy) {
  if (d.px > 2048 || d.py > 2048) {
    snprintf(why, nwhy, "padded size %dx%d exceeds 2048 (nx, ny <= 1024 supported)", d.px, d.py);
    return 0;
  }
  if (d.nz > 16) {
    snprintf(why, nwhy, "nz = %d > 16 is not supported by the z Toeplitz product of this build", d.nz);
    return 0;
  }
  if (yz_smem(d) > kMaxSmem) {
    snprintf(why, nwhy, "one kx column (3 x nz x py = 3 x %d x %d complex) exceeds shared memory", d.nz, d.py);
    return 0;
  }
  return 1;
}

template <int HALF>
static cudaError_t run_x(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                         cudaStream_t s, bool fwd) {
  const int P = HALF == 0 ? 1 : 2 * HALF;
  const float2* twP = tw + P;
  if (fwd) {
    const int TY = HALF == 0 ? 32 : xtile(HALF);
    const int T = HALF == 0 ? 1 : TeamOf<(HALF > 0 ? HALF : 1)>::v;
    int threads = HALF == 0 ? 32 : TY * T;
    if (threads < 32) threads = 32;
    if (threads > 512) threads = 512;
    const size_t smem = HALF == 0 ? 0 : sizeof(float2) * ((size_t)P + (size_t)TY * (HALF + 1));
    static bool attr = false;  // raise the dynamic shared-memory limit once (not a stream operation)
    if (!attr) { cudaFuncSetAttribute(k_xfwd<HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem); attr = true; }
    dim3 grid((d.ny + TY - 1) / TY, d.nz, 3);
    k_xfwd<HALF><<<grid, threads, smem, s>>>(a.m_in, S, twP, d, TY);
  } else {
    const int TY = HALF == 0 ? 32 : xinv_tile(HALF);
    const int T = HALF == 0 ? 1 : TeamOf<(HALF > 0 ? HALF : 1)>::v;
    int threads = HALF == 0 ? 32 : 3 * TY * T;
    if (threads < 128) threads = 128;
    if (threads > 512) threads = 512;
    const size_t smem = HALF == 0 ? 0 : sizeof(float2) * ((size_t)P + 3ull * TY * (HALF + 2));
    static bool attr = false;
    if (!attr) { cudaFuncSetAttribute(k_xinv<HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem); attr = true; }
    dim3 grid((d.ny + TY - 1) / TY, d.nz, 1);
    k_xinv<HALF><<<grid, threads, smem, s>>>(a, ph, S, twP, d, TY);
  }
  return cudaGetLastError();
}

static cudaError_t dispatch_x(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                              cudaStream_t s, bool fwd) {
  switch (d.px == 1 ? 0 : d.px / 2) {
    case 0: return run_x<0>(d, ph, a, tw, S, s, fwd);
    case 2: return run_x<2>(d, ph, a, tw, S, s, fwd);
    case 4: return run_x<4>(d, ph, a, tw, S, s, fwd);
    case 8: return run_x<8>(d, ph, a, tw, S, s, fwd);
    case 16: return run_x<16>(d, ph, a, tw, S, s, fwd);
    case 32: return run_x<32>(d, ph, a, tw, S, s, fwd);
    case 64: return run_x<64>(d, ph, a, tw, S, s, fwd);
    case 128: return run_x<128>(d, ph, a, tw, S, s, fwd);
    case 256: return run_x<256>(d, ph, a, tw, S, s, fwd);
    case 512: return run_x<512>(d, ph, a, tw, S, s, fwd);
    case 1024: return run_x<1024>(d, ph, a, tw, S, s, fwd);
  }
  return cudaErrorInvalidValue;
}

template <int PY, int NZM>
static cudaError_t run_yz_t(const Dims& d, const float2* tw, float2* S, const float* Kh, cudaStream_t s) {
  const size_t smem = yz_smem(d);
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_yz<PY, NZM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem); attr = true; }
  k_yz<PY, NZM><<<d.hx, 512, smem, s>>>(S, Kh, tw + PY, d);
  return cudaGetLastError();
}

template <int PY>
static cudaError_t run_yz_nz(const Dims& d, const float2* tw, float2* S, const float* Kh, cudaStream_t s) {
  switch (nzm_of(d.nz)) {
    case 1: return run_yz_t<PY, 1>(d, tw, S, Kh, s);
    case 2: return run_yz_t<PY, 2>(d, tw, S, Kh, s);
    case 4: return run_yz_t<PY, 4>(d, tw, S, Kh, s);
    case 8: return run_yz_t<PY, 8>(d, tw, S, Kh, s);
    case 16: return run_yz_t<PY, 16>(d, tw, S, Kh, s);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t dispatch_yz(const Dims& d, const float2* tw, float2* S, const float* Kh, cudaStream_t s) {
  switch (d.py) {
    case 1: return run_yz_nz<1>(d, tw, S, Kh, s);
    case 4: return run_yz_nz<4>(d, tw, S, Kh, s);
    case 8: return run_yz_nz<8>(d, tw, S, Kh, s);
    case 16: return run_yz_nz<16>(d, tw, S, Kh, s);
    case 32: return run_yz_nz<32>(d, tw, S, Kh, s);
    case 64: return run_yz_nz<64>(d, tw, S, Kh, s);
    case 128: return run_yz_nz<128>(d, tw, S, Kh, s);
    case 256: return run_yz_nz<256>(d, tw, S, Kh, s);
    case 512: return run_yz_nz<512>(d, tw, S, Kh, s);
    case 1024: return run_yz_nz<1024>(d, tw, S, Kh, s);
    case 2048: return run_yz_nz<2048>(d, tw, S, Kh, s);
  }
  return cudaErrorInvalidValue;
}

int launch_field_eval(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                      const float* Kh, cudaStream_t s) {
  if (dispatch_x(d, ph, a, tw, S, s, true) != cudaSuccess) return -1;
  if (dispatch_yz(d, tw, S, Kh, s) != cudaSuccess) return -2;
  if (dispatch_x(d, ph, a, tw, S, s, false) != cudaSuccess) return -3;
  return 3;
}

int launch_field_part(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                      const float* Kh, cudaStream_t s, int part) {
  cudaError_t e = cudaErrorInvalidValue;
  if (part == 0) e = dispatch_x(d, ph, a, tw, S, s, true);
  else if (part == 1) e = dispatch_yz(d, tw, S, Kh, s);
  else if (part == 2) e = dispatch_x(d, ph, a, tw, S, s, false);
  return e == cudaSuccess ? 1 : -1;
}

int launch_normalise(const Dims& d, float* m, int* flag, cudaStream_t s) {
  k_normalise<<<(unsigned)((d.N + 255) / 256), 256, 0, s>>>(m, d.N, flag);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}
