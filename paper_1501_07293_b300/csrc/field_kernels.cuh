// Effective field and LLG stage kernels (FP32): device code and the template
// launchers, shared by field.cu (dispatch) and the field_inst_*.cu translation
// units that instantiate them per padded size (compiled in parallel).
//
// One field evaluation is three launches:
//
//  k_xfwd  (per row tile)   real-to-complex transform of m along x, zero padded
//                           from nx to px (eq. 14 / Fig. 1), through a complex
//                           transform of half length; writes S[kx][c][z][y].
//  k_yz    (per kx column)  forward transform along y (zero padded ny -> py),
//                           the demag product of eq. 14 -- along z a direct
//                           Toeplitz sum over the nz planes with the kernel
//                           transformed along x and y only -- and the inverse
//                           transform along y, keeping the first ny rows.
//  k_x     (per row tile)   complex-to-real inverse along x (first nx points),
//                           then per cell: demag + exchange (eq. 5, Neumann rule
//                           eq. 7) + anisotropy (eq. 8) + Zeeman, and either the
//                           field itself or the LLG right-hand side (eq. 2) with
//                           the RK4 / Euler update and renormalisation; when
//                           stepping it also transforms the new state forward
//                           along x into S, so that a stage is k_yz + k_x.
//  k_yt, k_zt               the y/z pass split in three launches, for kx
//                           columns beyond one CTA or thick samples with few
//                           columns (the y transforms and the z product meet
//                           in a global buffer).
// The split-precision z product (tensor cores) lives in zsplit.cuh.
#pragma once
#include <stdio.h>
#include <string.h>

#include <type_traits>
#include <utility>

#include "common.cuh"
#include "fft.cuh"
#include "bulk.cuh"
#include "program.cuh"
#include "zsplit.cuh"
#include "adjoint.cuh"


// Loads of state that another CTA of the same launch may have written (PC: the
// persistent batch kernel, whose items depend on one another through device
// counters) go through L2 (ld.global.cg), never from a stale L1 line or the
// read-only path; otherwise the read-only path (ld_ro) or a plain load (ld_rw).
template <bool PC, typename T>
__device__ __forceinline__ T ld_ro(const T* p) {
  if constexpr (PC) return __ldcg(p);
  else return __ldg(p);
}
template <bool PC, typename T>
__device__ __forceinline__ T ld_rw(const T* p) {
  if constexpr (PC) return __ldcg(p);
  else return *p;
}

// ---------------------------------------------------------------------------
// k_xfwd: CTA = (tile of TY rows along y, plane z, component c)
// ---------------------------------------------------------------------------
template <int HALF>
__device__ __forceinline__ void body_xfwd(const float* __restrict__ m, float2* __restrict__ S,
                                          const float2* __restrict__ twP, const Dims& d, int TY, int c, int z,
                                          int y0) {
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
      if (MM_BC(k < d.hx && z < d.nz && y < d.ny)) S[(((long long)k * 3 + c) * d.nz + z) * d.ny + y] = X;
    }
  }
}

template <int HALF>
__global__ void __launch_bounds__(512) k_xfwd(const float* __restrict__ m, float2* __restrict__ S,
                                              const float2* __restrict__ twP, Dims d, int TY) {
  MM_BC_ENTER(d.flag);
  body_xfwd<HALF>(m, S, twP, d, TY, blockIdx.z, blockIdx.y, blockIdx.x * TY);
}

// ---------------------------------------------------------------------------
// The product of eq. 14 along z for one (kx, ky) and one output component a:
//   out[zo] = sum_b sum_zi Kt_{a b}(kx, ky, zo - zi) M_b(zi)
// Kt at a negative z offset follows from the parity in z, at a mirrored ky
// (ky > py/2) from the parity in y; the pairs xz, yz hold the imaginary part of
// their x/y transform and act as i * Kt.  The (zo, zi) block is unrolled (its
// register indices are static); the loop over b is not, which keeps the code
// small enough for the instruction cache.  Planes zi >= nz enter as zeros and
// outputs zo >= nz are never stored, so the FMA block carries no bounds tests.
// ---------------------------------------------------------------------------
// Tensor loads of the z product: read-only global path, or plain loads when the
// caller staged its tensor slice in shared memory (KS).
template <bool KS>
__device__ __forceinline__ float ldk(const float* p) {
  if constexpr (KS) return *p;
  else return __ldg(p);
}
template <bool KS>
__device__ __forceinline__ float4 ldk4(const float* p) {
  if constexpr (KS) return *reinterpret_cast<const float4*>(p);
  else return __ldg(reinterpret_cast<const float4*>(p));
}
// Row stride of a staged tensor slice: nz + 4 for the 16-byte loads of the
// direct product, nz + 1 for the scalar window loads of the chunked one (rows
// then start in different banks)
template <int NZM>
__host__ __device__ constexpr int kst_pad() { return NZM > 16 ? 1 : 4; }

template <int NZM, bool KS = false>
__device__ __forceinline__ void zprod(int a, const float2* __restrict__ buf, int rs, int pos, int nz,
                                      const float* __restrict__ Kk, int hy, int kyf, bool mirrored,
                                      float2 (&out)[NZM]) {
#pragma unroll
  for (int q = 0; q < NZM; ++q) out[q] = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int b = 0; b < 3; ++b) {
    const int p = (a == b) ? a : 2 + a + b;   // xx yy zz | xy xz yz
    const bool odd_y = (p == 3 || p == 5);
    const bool odd_z = (p >= 4);              // xz, yz: odd in z and imaginary
    const float ys = (mirrored && odd_y) ? -1.f : 1.f;
    const float zs = odd_z ? -ys : ys;
    const float* kp = Kk + ((long long)kyf * 6 + p) * (KS ? nz + kst_pad<NZM>() : nz);   // the nz offsets of this pair
    float kr[NZM], kn[NZM];   // kernel at offsets +q and -q
    float2 mv[NZM];
    if (NZM % 4 == 0 && (nz & 3) == 0) {
#pragma unroll
      for (int q4 = 0; q4 < NZM / 4; ++q4) {
        const float4 v = (4 * q4 < nz) ? ldk4<KS>(kp + 4 * q4) : make_float4(0.f, 0.f, 0.f, 0.f);
        kr[4 * q4 + 0] = ys * v.x; kn[4 * q4 + 0] = zs * v.x;
        kr[4 * q4 + 1] = ys * v.y; kn[4 * q4 + 1] = zs * v.y;
        kr[4 * q4 + 2] = ys * v.z; kn[4 * q4 + 2] = zs * v.z;
        kr[4 * q4 + 3] = ys * v.w; kn[4 * q4 + 3] = zs * v.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < NZM; ++q) {
        const float v = (q < nz) ? ldk<KS>(kp + q) : 0.f;
        kr[q] = ys * v;
        kn[q] = zs * v;
      }
    }
#pragma unroll
    for (int zi = 0; zi < NZM; ++zi) {
      const float2 v = (zi < nz) ? buf[(b * nz + zi) * rs + pos] : make_float2(0.f, 0.f);
      mv[zi] = odd_z ? make_float2(-v.y, v.x) : v;   // i * m for the imaginary pairs
    }
#pragma unroll
    for (int zo = 0; zo < NZM; ++zo) {
#pragma unroll
      for (int zi = 0; zi < NZM; ++zi) {
        const float k = (zo >= zi) ? kr[zo - zi] : kn[zi - zo];
        out[zo] = __ffma2_rn(make_float2(k, k), mv[zi], out[zo]);   // packed FP32 pair
      }
    }
  }
}

// In-place z product over a column of `len` positions of a shared buffer holding
// 3 nz planes of stride rs (position q of a plane at posf(q)).  Each warp takes
// groups of 10 positions with all three output components (lanes 0-29), so every
// input of a position is read before any output of it is written with only a
// warp-level barrier in between.
template <int NZM, int PADS, typename KyOf, bool KS = false>
__device__ __forceinline__ void zprod_column(float2* buf, int rs, int len, int nz, const float* __restrict__ Kk,
                                             int hy, int py, KyOf ky_of) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int a = lane / 10, kl = lane % 10;
  const int ntasks = (len + 9) / 10;
  for (int task = warp; task < ntasks; task += nwarps) {
    const int k = task * 10 + kl;
    const bool act = a < 3 && k < len;
    float2 out[NZM];
    if (act) {
      const int ky = ky_of(k);
      const bool mirrored = ky > py / 2;
      zprod<NZM, KS>(a, buf, rs, pidx<PADS>(k), nz, Kk, hy, mirrored ? py - ky : ky, mirrored, out);
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int zo = 0; zo < NZM; ++zo)
        if (zo < nz && MM_BC_SMEM(&buf[(a * nz + zo) * rs + pidx<PADS>(k)], sizeof(float2)))
          buf[(a * nz + zo) * rs + pidx<PADS>(k)] = out[zo];
    }
    __syncwarp();
  }
}

// Thick films (NZM = 32, 64): the same product with each lane owning one chunk
// of 16 output planes.  The input planes are walked in blocks of 16; between
// input block j and output chunk c the offsets zo - zi span 16 (c - j) - 15 ..
// 16 (c - j) + 15, a window of 31 kernel values loaded once per block.
// Offsets with |zo - zi| >= nz only meet zero inputs or discarded outputs and
// are read as zeros.
template <bool KS = false>
__device__ __forceinline__ void zprod_chunk(int a, int c, const float2* __restrict__ buf, int rs, int pos, int nz,
                                            const float* __restrict__ Kk, int kyf, bool mirrored,
                                            float2 (&out)[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) out[q] = make_float2(0.f, 0.f);
  const int nblk = (nz + 15) >> 4;
#pragma unroll 1
  for (int b = 0; b < 3; ++b) {
    const int p = (a == b) ? a : 2 + a + b;
    const bool odd_y = (p == 3 || p == 5);
    const bool odd_z = (p >= 4);
    const float ys = (mirrored && odd_y) ? -1.f : 1.f;
    const float zs = odd_z ? -ys : ys;
    const float* kp = Kk + ((long long)kyf * 6 + p) * (KS ? nz + kst_pad<32>() : nz);
#pragma unroll 1
    for (int j = 0; j < nblk; ++j) {
      const int base = 16 * (c - j) - 15;
      float w[31];
#pragma unroll
      for (int t = 0; t < 31; ++t) {
        const int off = base + t;
        const int q = off < 0 ? -off : off;
        const float v = q < nz ? ldk<KS>(kp + q) : 0.f;
        w[t] = (off < 0 ? zs : ys) * v;
      }
      float2 mv[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int zi = 16 * j + i;
        const float2 v = zi < nz ? buf[(b * nz + zi) * rs + pos] : make_float2(0.f, 0.f);
        mv[i] = odd_z ? make_float2(-v.y, v.x) : v;
      }
#pragma unroll
      for (int zo = 0; zo < 16; ++zo) {
#pragma unroll
        for (int zi = 0; zi < 16; ++zi) {
          const float k = w[zo - zi + 15];
          out[zo] = __ffma2_rn(make_float2(k, k), mv[zi], out[zo]);
        }
      }
    }
  }
}

// Lanes take (position, output component, chunk): 3 NZM/16 lanes per position,
// all in one warp, so the in-place write-back again needs only __syncwarp.
template <int NZM, int PADS, typename KyOf, bool KS = false>
__device__ __forceinline__ void zprod_column_chunked(float2* buf, int rs, int len, int nz,
                                                     const float* __restrict__ Kk, int py, KyOf ky_of) {
  constexpr int NCH = NZM / 16;
  constexpr int LPK = 3 * NCH;      // lanes per position
  constexpr int KPW = 32 / LPK;     // positions per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int kl = lane / LPK, r = lane % LPK, a = r / NCH, c = r % NCH;
  const int ntasks = (len + KPW - 1) / KPW;
  for (int task = warp; task < ntasks; task += nwarps) {
    const int k = task * KPW + kl;
    const bool act = kl < KPW && k < len && 16 * c < nz;
    float2 out[16];
    if (act) {
      const int ky = ky_of(k);
      const bool mirrored = ky > py / 2;
      zprod_chunk<KS>(a, c, buf, rs, pidx<PADS>(k), nz, Kk, mirrored ? py - ky : ky, mirrored, out);
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int zo = 0; zo < 16; ++zo)
        if (16 * c + zo < nz && MM_BC_SMEM(&buf[(a * nz + 16 * c + zo) * rs + pidx<PADS>(k)], sizeof(float2)))
          buf[(a * nz + 16 * c + zo) * rs + pidx<PADS>(k)] = out[zo];
    }
    __syncwarp();
  }
}

struct KyIdentity {
  __device__ int operator()(int k) const { return k; }
};

// Column buffer of the y/z pass: 3 nz rows of stride RS (padded for the
// Stockham passes, natural order for the two-pass transform).
template <int PY>
struct YzLayout {
  static constexpr int PADS = PY >= 32 ? 4 : 0;
  static constexpr int RS = PY + (PADS ? PY / 16 : 0) + 2;   // even: rows stay 16-byte aligned
};

// ---------------------------------------------------------------------------
// The product of eq. 14 along z as a transform (films of 9..16 planes, py = 256
// or 512, natural ky order in the column buffer).  For nz <= 16 the linear
// convolution along z equals a circular one of length 32:
//   out_a(z) = sum_kz e^{+2 pi i kz z / 32} sum_b Kz_ab(kz) X_b(kz),
//   X_b(kz)  = sum_{z < nz} m_b(z) e^{-2 pi i kz z / 32},
// with Kz the tensor transformed along z (Kt: real for every pair, the 1/32 of
// the inverse folded in; pairs odd in z change sign at kz > 16, pairs odd in y
// at a mirrored ky).  The 32 frequencies split into two halves of 16:
//   X_b(2k)     = DFT16[m_b(z)](k),   X_b(2k + 1) = DFT16[m_b(z) W32^z](k),
//   out_a(z)    = IDFT16[Y_a(2k)](z) + W32^-z IDFT16[Y_a(2k + 1)](z).
// Two lanes share a position ky: lane half h (0: even, 1: odd frequencies)
// holds all three components of its half in registers (16-point register
// transforms, fft.cuh reg_fft), applies the 3 x 3 product per kz, and
// transforms back.  The odd lane keeps its sequence rotated by 8 planes
// (register r holds plane (r + 8) mod 16), which multiplies its spectrum by
// (-1)^k and rotates its inverse output back by 8; then both lanes exchange
// registers 8..15 and keep 0..7, so the even lane ends with out(0..7) and the
// odd lane with out(8..15), with no selects.  A warp takes 16 positions; every
// lane reads its inputs before any lane of the warp writes (__syncwarp).
// ---------------------------------------------------------------------------
template <int PY>
__device__ __forceinline__ void zprod_fft_column(float2* buf, int nz, const float* __restrict__ Kt_col) {
  constexpr int RS = YzLayout<PY>::RS;
  constexpr int HY = PY / 2 + 1;
  static_assert(PY == 256 || PY == 512, "natural-order columns of 256 or 512");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int h = lane >> 4, j = lane & 15;
  const int h8 = h << 3;
  for (int g = warp; g < PY / 16; g += nwarps) {
    const int ky = 16 * g + j;
    const bool mirrored = ky > PY / 2;
    const int kyf = mirrored ? PY - ky : ky;
    const float ys = mirrored ? -1.f : 1.f;
    float2 v[3][16];
    // forward: even lane v[r] = m(r); odd lane v[r] = m(zt) W32^zt, zt = (r + 8) mod 16
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // plane zt = r + h8 (r < 8) or r - h8 (r >= 8): compile-time offsets from two bases
      const float2* lo = buf + (b * nz + h8) * RS + ky;
      const float2* hi = buf + (b * nz - h8) * RS + ky;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int zt = r < 8 ? r + h8 : r - h8;
        v[b][r] = zt < nz ? (r < 8 ? lo : hi)[r * RS] : make_float2(0.f, 0.f);
      }
      if (h) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[b][r] = mul_w32<-1>(v[b][r], (r + 8) & 15);
      }
      reg_fft<16, -1>(v[b]);   // spectrum index k at v[b][brev(k)]
    }
    // 3 x 3 product per frequency kz = 2k + h; Kt holds kz <= 16, kz > 16 reads 32 - kz
    const float* kp = Kt_col + kyf + h * 6 * HY;   // kz = 2k + h   (k <= 7)
    const float* km = Kt_col + kyf - h * 6 * HY;   // kz = 32 - 2k - h (k >= 8)
    const float s8 = h ? -1.f : 1.f;               // z parity at k = 8 (kz 16 or 17)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float* kb = k <= 7 ? kp + (2 * k) * 6 * HY : km + (32 - 2 * k) * 6 * HY;
      const float zs = k <= 7 ? 1.f : (k == 8 ? s8 : -1.f);
      const float kxx = __ldg(kb + 0 * HY), kyy = __ldg(kb + 1 * HY), kzz = __ldg(kb + 2 * HY);
      const float kxy = ys * __ldg(kb + 3 * HY);
      const float kxz = zs * __ldg(kb + 4 * HY);
      const float kyz = (ys * zs) * __ldg(kb + 5 * HY);
      const int q = brev(k, 4);
      const float2 x0 = v[0][q], x1 = v[1][q], x2 = v[2][q];
      v[0][q] = __ffma2_rn(make_float2(kxz, kxz), x2, __ffma2_rn(make_float2(kxy, kxy), x1, __fmul2_rn(make_float2(kxx, kxx), x0)));
      v[1][q] = __ffma2_rn(make_float2(kyz, kyz), x2, __ffma2_rn(make_float2(kyy, kyy), x1, __fmul2_rn(make_float2(kxy, kxy), x0)));
      v[2][q] = __ffma2_rn(make_float2(kzz, kzz), x2, __ffma2_rn(make_float2(kyz, kyz), x1, __fmul2_rn(make_float2(kxz, kxz), x0)));
    }
    // inverse: natural frequency order by renaming, then register r holds the
    // half's contribution at plane r (even) or (r + 8) mod 16 (odd, after W32^-z)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 w[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) w[k] = v[a][brev(k, 4)];
      reg_fft<16, 1>(w);   // plane r at w[brev(r)]
#pragma unroll
      for (int r = 0; r < 16; ++r) v[a][r] = w[brev(r, 4)];
      if (h) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[a][r] = mul_w32<1>(v[a][r], (r + 8) & 15);
      }
    }
    __syncwarp();   // every lane of the warp has read its inputs
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2* col = buf + a * nz * RS + ky;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, v[a][8 + i].x, 16);
        o.y = __shfl_xor_sync(0xffffffffu, v[a][8 + i].y, 16);
        const int z = h8 + i;
        if (z < nz && MM_BC_SMEM(&col[z * RS], sizeof(float2))) col[z * RS] = cadd(v[a][i], o);
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// k_yz: CTA = one kx column, all 3 components and nz planes in shared memory.
//  1. the column's 3 nz rows of ny values arrive by bulk copies (TMA engine)
//     into dense rows of a padded buffer (row stride RS);
//  2. forward y transform of every row: the first pass reads the dense row and
//     takes positions >= ny as zeros (zero padding), the later passes use the
//     padded layout (no shared-memory bank conflicts);
//  3. the product of eq. 14 along z (zprod_column), in place;
//  4. inverse y transform; the last pass writes only the first ny outputs, dense;
//  5. bulk copies back to S.
// On large grids (d.pdl: the first wave of CTAs starts together, right when the
// kernel before completes) the copies of step 1 go in up to YZ_GROUPS groups of
// rows with one mbarrier each, a team waiting only for its row's group, and in
// step 5 each team stores its rows as soon as they are done.  Small films keep
// one barrier and one storing thread (cheaper when launch-bound).
// A failed bounded wait sets flag[1] and abandons the column.
// ---------------------------------------------------------------------------
static constexpr int YZ_GROUPS = 8;   // copy groups (mbarriers) of a y/z column on large grids

// The y transforms of the 3 nz rows of a column by the two-pass transform of
// fft.cuh (py = 256, 512).  Warp w owns rows p = w + nwarps i; pass 1 takes them
// one per warp (R2 = 32) or two per warp (R2 = 16), pass 2 two per warp (one
// per half-warp).  before_row(p) runs (all lanes of the row's group) before
// pass 1 reads row p; after_pair(p, act) runs (all lanes) after pass 2 of the
// half-warp's row p (act: the half-warp had a row).
template <int PY, int DIR, typename Before, typename After>
__device__ __forceinline__ void yz_rows_fft2(float2* buf, int NP, int nin, int nout, const float2* __restrict__ twY,
                                             Before before_row, After after_pair) {
  constexpr int RS = YzLayout<PY>::RS;
  constexpr int R2 = PY / 16;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int half = lane >> 4, k1 = lane & 15;
  const int nmine = warp < NP ? (NP - warp + nwarps - 1) / nwarps : 0;
  {
    float2 tw[16];
    fft2_twiddles<PY, DIR>(tw, lane & (R2 - 1), twY);
    if constexpr (R2 == 32) {   // a whole warp on each row
      for (int i = 0; i < nmine; ++i) {
        const int p = warp + nwarps * i;
        before_row(p);
        float2* const rows[1] = {buf + p * RS};
        const bool act[1] = {true};
        fft2_pass1<32, DIR, (DIR < 0)>(rows, act, lane, nin, tw);
      }
    } else {                    // a row per half-warp
      for (int i = 0; i < nmine; i += 2) {
        const int ii = i + half;
        const bool a1 = ii < nmine;
        const int p = warp + nwarps * (a1 ? ii : i);
        if (a1) before_row(p);
        float2* const rows[1] = {buf + p * RS};
        const bool act[1] = {a1};
        fft2_pass1<R2, DIR, (DIR < 0)>(rows, act, lane & (R2 - 1), nin, tw);
      }
    }
  }
  __syncwarp();
  for (int i = 0; i < nmine; i += 2) {
    const int ii = i + half;
    const bool act = ii < nmine;
    const int p = warp + nwarps * (act ? ii : i);
    fft2_pass2<R2, DIR>(buf + p * RS, act, k1, nout);
    after_pair(p, act);
  }
}

// Split-precision variants (PREC = MM_SPLIT_BF16 / MM_SPLIT_FP16) replace the
// FP32 direct sum of step 3 by zs::zprod_split on the tensor cores; the DFT
// operands follow the rows in shared memory.
template <int PY, int NZM, int PREC = 0, bool PC = false>
__device__ __forceinline__ void body_yz(float2* __restrict__ S, const float* __restrict__ Kh,
                                        const float2* __restrict__ twY, const Dims& d, int* flag, int kx,
                                        const Tick& tk = Tick{}) {
  constexpr int T = TeamOf<PY>::v;
  constexpr int PADS = YzLayout<PY>::PADS;
  constexpr int RS = YzLayout<PY>::RS;
  // py = 256, 512: the two-pass y transform (natural order between the
  // transforms); other sizes: the Stockham passes (padded order in between)
  constexpr bool FFT2 = (PY == 256 || PY == 512);
  constexpr int ZPADS = FFT2 ? 0 : PADS;   // layout the z product reads
  // the z product as a length-32 transform (zprod_fft_column) when the context
  // built Kt for it (d.zfft); the batch kernel (PC) keeps the direct sum
  constexpr bool ZFFT_OK = FFT2 && NZM == 16 && PREC == 0 && !PC;
  extern __shared__ __align__(16) float2 sm[];
  float2* tws = sm;        // exp(-2 pi i m / PY), m < PY
  float2* buf = sm + PY;   // [3 nz][RS]
  // grouped copies only in the instances for tall columns (py >= 128); the
  // short ones keep the single-barrier code alone (smaller and, for the small
  // launch-bound films, measurably faster)
  constexpr bool CAN_GROUP = PY >= 128;
  __shared__ __align__(8) uint64_t bar[CAN_GROUP ? YZ_GROUPS : 1];
  const int nz = d.nz, ny = d.ny;
  const int NP = 3 * nz;
  float2* Sk = S + (long long)kx * NP * ny;
  // rows of ny float2 are then 16-byte multiples; the persistent batch kernel
  // (PC) keeps to plain loads and stores (one memory proxy, ordered by its counters)
  const bool bulk = !PC && (ny % 2) == 0;
  const bool grouped = CAN_GROUP && bulk && d.pdl;
  // rows p of group g: g * rpg <= p < min(NP, (g + 1) * rpg)
  const int rpg = grouped ? (NP + YZ_GROUPS - 1) / YZ_GROUPS : NP;
  const int ngrp = (NP + rpg - 1) / rpg;
  auto issue_copies = [&] {
    for (int g = 0; g < ngrp; ++g) {
      const int p1 = min(NP, (g + 1) * rpg);
      mbar_arrive_expect_tx(&bar[g], (uint32_t)((p1 - g * rpg) * ny * sizeof(float2)));
      for (int p = g * rpg; p < p1; ++p)
        if (MM_BC_SMEM(buf + p * RS, ny * sizeof(float2)) && MM_BC(kx < d.hx && p < NP))
          bulk_g2s(buf + p * RS, Sk + (long long)p * ny, ny * sizeof(float2), &bar[g]);
    }
  };
  if (bulk && threadIdx.x == 0) {
    for (int g = 0; g < ngrp; ++g) mbar_init(&bar[g], 1);
    mbar_fence_init();
  }
  // Without programmatic serialization (small grids) the kernel starts after
  // the one before has completed: the copies go out first and land during the
  // prologue.  With it, the prologue below touches constant data only
  // (twiddles, the tensor's L2 prefetch, the split path's operands) and
  // overlaps the end of the kernel before, which wrote S; the copies follow
  // the dependency wait.
  const bool early = bulk && !d.pdl;
  if (early) {
    __syncthreads();   // the barriers are initialised before anyone polls them
    if (threadIdx.x == 0) issue_copies();
  }
  for (int i = threadIdx.x; i < PY; i += blockDim.x) tws[i] = twY[i];
  // split precision: the DFT operands, the MMA barrier and the tensor memory
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  unsigned char* Bsm = reinterpret_cast<unsigned char*>(buf + 3 * nz * RS);
  if constexpr (PREC != 0) {
    const uint4* src = reinterpret_cast<const uint4*>(d.Bdft);
    uint4* dst = reinterpret_cast<uint4*>(Bsm);
    for (int i = threadIdx.x; i < zs::Dft<NZM>::bytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    if (threadIdx.x == 0) {
      mbar_init(&mbar, 1);
      mbar_fence_init();
    }
    if ((threadIdx.x >> 5) == 0) zs::tmem_alloc(&tbase, 512);
  }
  {
    // the column's slice of the transformed tensor is first read by the z
    // product, after the transforms: start bringing it into L2 now
    const bool kz = PREC || ZFFT_OK && d.zfft;   // the z-transformed tensor Kt
    const char* kc = kz ? reinterpret_cast<const char*>(d.Kt + (long long)kx * d.hy * (NZM + 1) * 6)
                        : reinterpret_cast<const char*>(Kh + (long long)kx * d.hy * 6 * nz);
    const int bytes = kz ? d.hy * (NZM + 1) * 6 * (int)sizeof(float) : d.hy * 6 * nz * (int)sizeof(float);
    const int nlines = (bytes + 127) >> 7;
    for (int i = threadIdx.x; i < nlines; i += blockDim.x) prefetch_l2(kc + ((long long)i << 7));
  }
  grid_dep_wait();     // S and the program state: written by the kernels before
  grid_dep_launch();
  if (!early) {
    __syncthreads();   // the barriers are initialised before anyone polls them
    if (bulk) {
      if (threadIdx.x == 0) issue_copies();
    } else {
      for (int i = threadIdx.x; i < NP * ny; i += blockDim.x)
        if (MM_BC_SMEM(&buf[(i / ny) * RS + i % ny], sizeof(float2)) && MM_BC(kx < d.hx))
          buf[(i / ny) * RS + i % ny] = ld_rw<PC>(Sk + i);
    }
  }
  // first y/z pass of a step: the last warp of CTA 0 advances the field
  // program's clock and writes the drive slots while the copies land (the x
  // kernels that follow read them; nothing in this kernel does)
  if (tk.p && kx == 0 && threadIdx.x >= blockDim.x - 32) prog_tick(tk);
  const int lane = threadIdx.x & 31;
  const int team = threadIdx.x / T, t = threadIdx.x % T, nteams = blockDim.x / T;
  const unsigned mask = team_mask<T>(lane);
  bool arrived = true;
  if (grouped) {   // transforms start on the rows that have landed
    if constexpr (FFT2) {
      yz_rows_fft2<PY, -1>(buf, NP, ny, PY, twY,
                           [&](int p) { arrived = mbar_wait_bounded(&bar[p / rpg], 0) && arrived; },
                           [](int, bool) {});
    } else {
      for (int p = team; p < NP; p += nteams) {
        arrived = mbar_wait_bounded(&bar[p / rpg], 0) && arrived;
        if (PY > 1) team_fft_io<PY, T, -1, 1, 0, PADS, PADS>(buf + p * RS, t, mask, tws, ny, PY);
      }
    }
  } else if (bulk) {
    arrived = mbar_wait_bounded(&bar[0], 0);
  }
  if constexpr (PREC != 0) {
    fence_proxy_async_smem();   // the DFT operands are read by the tensor cores (async proxy)
    zs::fence_before();
  }
  if (!__syncthreads_and(arrived)) {   // uniform: every thread leaves, tensor memory is freed
    if (threadIdx.x == 0) atomicOr(flag + 1, 1);
    if (bulk)   // copies in flight get one more bounded chance
      for (int g = 0; g < ngrp; ++g) mbar_wait_bounded(&bar[g], 0);
    if constexpr (PREC != 0) {
      if ((threadIdx.x >> 5) == 0) zs::tmem_dealloc(tbase, 512);
    }
    return;
  }
  if constexpr (PREC != 0) zs::fence_after();
  if (PY > 1 && !grouped) {
    if constexpr (FFT2) {
      yz_rows_fft2<PY, -1>(buf, NP, ny, PY, twY, [](int) {}, [](int, bool) {});
    } else {
      for (int p = team; p < NP; p += nteams)
        team_fft_io<PY, T, -1, 1, 0, PADS, PADS>(buf + p * RS, t, mask, tws, ny, PY);
    }
    __syncthreads();
  }
  // Product of eq. 14 along z (see zprod).
  if constexpr (PREC != 0) {
    static_assert(NZM == 8 || NZM == 16, "split z product: 8 or 16 planes");
    static_assert(PY >= 128 && PY % 128 == 0, "split z product: chunks of 128 ky");
    const uint32_t tb = tbase;
    uint32_t phase = 0;
    const bool ok = zs::zprod_split<PY, NZM, PREC, ZPADS>(buf, RS, nz, PY, d.hy, d.Kt + (long long)kx * d.hy * (NZM + 1) * 6,
                                                         Bsm, tb, &mbar, phase, flag);
    if (!ok) mbar_wait_bounded(&mbar, phase);   // MMAs still in flight get one more bounded wait
    zs::fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) zs::tmem_dealloc(tb, 512);
    if (!ok) return;
  } else if constexpr (NZM > 16)
    zprod_column_chunked<NZM, (PY > 1 ? ZPADS : 0)>(buf, RS, PY, nz, Kh + (long long)kx * d.hy * 6 * nz, PY,
                                                    KyIdentity());
  else if (ZFFT_OK && d.zfft) {
    if constexpr (ZFFT_OK) zprod_fft_column<PY>(buf, nz, d.Kt + (long long)kx * d.hy * (NZM + 1) * 6);
  } else if (PY > 1)
    zprod_column<NZM, ZPADS>(buf, RS, PY, nz, Kh + (long long)kx * d.hy * 6 * nz, d.hy, PY, KyIdentity());
  else
    zprod_column<NZM, 0>(buf, RS, PY, nz, Kh + (long long)kx * 6 * nz * d.hy, d.hy, PY, KyIdentity());
  __syncthreads();
  if (grouped) {
    // each team stores its own rows: every lane orders its writes of the row
    // before the bulk engine's reads, then the team's first lane issues the copy
    if constexpr (FFT2) {
      bool issued = false;
      yz_rows_fft2<PY, 1>(buf, NP, PY, ny, twY, [](int) {}, [&](int p, bool act) {
        fence_proxy_async_smem();
        __syncwarp();
        if (act && (threadIdx.x & 15) == 0 && MM_BC(kx < d.hx && p < NP)) {
          bulk_s2g(Sk + (long long)p * ny, buf + p * RS, ny * sizeof(float2));
          bulk_commit();
          issued = true;
        }
      });
      if (issued) bulk_wait_read_all();   // the rows stay valid until read
    } else {
      for (int p = team; p < NP; p += nteams) {
        if (PY > 1) team_fft_io<PY, T, 1, 1, PADS, PADS, 0>(buf + p * RS, t, mask, tws, PY, ny);
        fence_proxy_async_smem();
        __syncwarp(mask);
        if (t == 0 && MM_BC(kx < d.hx && p < NP)) {
          bulk_s2g(Sk + (long long)p * ny, buf + p * RS, ny * sizeof(float2));
          bulk_commit();
        }
      }
      if (t == 0) bulk_wait_read_all();   // the rows stay valid until read
    }
    return;
  }
  if (PY > 1) {
    if constexpr (FFT2) {
      yz_rows_fft2<PY, 1>(buf, NP, PY, ny, twY, [](int) {}, [](int, bool) {});
    } else {
      for (int p = team; p < NP; p += nteams)
        team_fft_io<PY, T, 1, 1, PADS, PADS, 0>(buf + p * RS, t, mask, tws, PY, ny);
    }
    __syncthreads();
  }
  if (bulk) {
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      for (int p = 0; p < NP; ++p)
        if (MM_BC(kx < d.hx)) bulk_s2g(Sk + (long long)p * ny, buf + p * RS, ny * sizeof(float2));
      bulk_commit();
      bulk_wait_read_all();
    }
  } else {
    for (int i = threadIdx.x; i < NP * ny; i += blockDim.x)
      if (MM_BC(kx < d.hx)) Sk[i] = buf[(i / ny) * RS + i % ny];
  }
}

template <int PY, int NZM, int PREC>
__global__ void __launch_bounds__(512, 1) k_yz(float2* __restrict__ S, const float* __restrict__ Kh,
                                                const float2* __restrict__ twY, Dims d, int* flag, Tick tk) {
  MM_BC_ENTER(d.flag);
  body_yz<PY, NZM, PREC>(S, Kh, twY, d, flag, blockIdx.x, tk);
}

// ---------------------------------------------------------------------------
// Split y/z pass, for kx columns that do not fit one CTA's shared memory (more
// than 64 planes, or 3 nz py complex values beyond 227 KB): the y transforms
// and the z product meet in a global buffer T[kx][3 nz][py] (L2-resident at
// the sizes it serves).
//   k_yt<PY, DIR>: CTA = (kx, a group of rows, one team each).  DIR -1: rows of
//                  S (ny values) -> forward transform -> T (py values);
//                  DIR +1: T -> inverse transform -> S (first ny values).
//   k_zt<NZM>:     CTA = (kx, KB consecutive ky): the 3 nz values of each ky
//                  from T into shared memory, the z product, back to T.
// ---------------------------------------------------------------------------
template <int PY, int DIR>
__global__ void __launch_bounds__(256) k_yt(float2* __restrict__ S, float2* __restrict__ T,
                                            const float2* __restrict__ twY, Dims d, Tick tk) {
  constexpr int TM = TeamOf<PY>::v;
  constexpr int PADS = YzLayout<PY>::PADS;
  constexpr int RS = YzLayout<PY>::RS;
  extern __shared__ __align__(16) float2 sm[];
  float2* tws = sm;
  float2* rows = sm + PY;
  MM_BC_ENTER(d.flag);
  const int kx = blockIdx.x, ny = d.ny, NP = 3 * d.nz;
  const int nrows = blockDim.x / TM;
  const int r0 = blockIdx.y * nrows;
  float2* Sk = S + (long long)kx * NP * ny;
  float2* Tk = T + (long long)kx * NP * PY;
  for (int i = threadIdx.x; i < PY; i += blockDim.x) tws[i] = twY[i];
  grid_dep_wait();     // S or T: written by the kernel before
  grid_dep_launch();
  const int nin = DIR < 0 ? ny : PY;
  for (int i = threadIdx.x; i < nrows * nin; i += blockDim.x) {
    const int r = i / nin, e = i % nin;
    if (r0 + r >= NP) continue;
    rows[r * RS + e] = DIR < 0 ? Sk[(long long)(r0 + r) * ny + e] : Tk[(long long)(r0 + r) * PY + e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int team = threadIdx.x / TM, t = threadIdx.x % TM;
  if (PY > 1 && r0 + team < NP)
    team_fft_io<PY, TM, DIR, 1, 0, PADS, 0>(rows + team * RS, t, team_mask<TM>(lane), tws, nin, DIR < 0 ? PY : ny);
  __syncthreads();
  const int nout = DIR < 0 ? PY : ny;
  for (int i = threadIdx.x; i < nrows * nout; i += blockDim.x) {
    const int r = i / nout, e = i % nout;
    if (r0 + r >= NP) continue;
    if (DIR < 0) Tk[(long long)(r0 + r) * PY + e] = rows[r * RS + e];
    else Sk[(long long)(r0 + r) * ny + e] = rows[r * RS + e];
  }
  // first y/z launch of a step: the field program's clock and drive slots
  if (DIR < 0 && tk.p && kx == 0 && blockIdx.y == 0 && threadIdx.x < 32) prog_tick(tk);
}

struct KyShift {
  int k0;
  __device__ int operator()(int k) const { return k0 + k; }
};

template <int NZM>
__global__ void __launch_bounds__(512, 1) k_zt(float2* __restrict__ T, const float* __restrict__ Kh, Dims d, int KB) {
  extern __shared__ __align__(16) float2 zb[];   // [3 nz][KB], then the tensor rows of the block
  MM_BC_ENTER(d.flag);
  const int kx = blockIdx.x, ky0 = blockIdx.y * KB;
  const int nz = d.nz, NP = 3 * nz, py = d.py;
  const int len = py - ky0 < KB ? py - ky0 : KB;
  float2* Tk = T + (long long)kx * NP * py;
  // the block's folded ky (py - ky above py/2) form one contiguous range of
  // tensor rows [kmin, kmax]: staged in shared memory (the z product reads each
  // value many times).  The tensor is constant, so its copies start before the
  // dependency wait; T is written by the kernel before.
  auto fold = [&](int ky) { return ky > py / 2 ? py - ky : ky; };
  const int f0 = fold(ky0), f1 = fold(ky0 + len - 1);
  const int kmin = min(f0, f1);   // at most len + 1 rows in every case
  const int kmax = (ky0 <= py / 2 && ky0 + len - 1 >= py / 2) ? py / 2 : max(f0, f1);
  constexpr int PAD = kst_pad<NZM>();
  float* ks = reinterpret_cast<float*>(zb + NP * KB);
  const float* Kg = Kh + ((long long)kx * d.hy + kmin) * 6 * nz;
  for (int i = threadIdx.x; i < (kmax - kmin + 1) * 6 * nz; i += blockDim.x)
    cp_async4(ks + (i / nz) * (nz + PAD) + i % nz, Kg + i);
  grid_dep_wait();
  grid_dep_launch();
  for (int i = threadIdx.x; i < NP * len; i += blockDim.x) {
    const int p = i / len, j = i % len;
    cp_async8(zb + p * KB + j, Tk + (long long)p * py + ky0 + j);
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  const float* Kk = ks - (long long)kmin * 6 * (nz + PAD);   // indexed by the folded ky as the global table
  if constexpr (NZM > 16) zprod_column_chunked<NZM, 0, KyShift, true>(zb, KB, len, nz, Kk, py, KyShift{ky0});
  else zprod_column<NZM, 0, KyShift, true>(zb, KB, len, nz, Kk, d.hy, py, KyShift{ky0});
  __syncthreads();
  for (int i = threadIdx.x; i < NP * len; i += blockDim.x) {
    const int p = i / len, j = i % len;
    Tk[(long long)p * py + ky0 + j] = zb[p * KB + j];
  }
}

// ---------------------------------------------------------------------------
// per-cell field terms and LLG update
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Eq. 2 on the unit vector m in the total field B (tesla), then the integrator:
// mode 2 the explicit Euler step, mode 1 RK4 stage a.stage with base state m0
// and accumulator value accv (read for stages 1..3).  Returns the next stage
// state (renormalised after a full step); *acc_out is the accumulator to store
// (stages 0..2), *kmag |dm/dt| at m.
__device__ __forceinline__ float3 llg_stage(const StageArgs& a, const Phys& ph, float3 m, float3 B, float3 m0,
                                            float3 accv, float3* acc_out, float* kmag) {
  // dm/dt = g1 m x B + g2 m x (m x B)
  const float3 mxB = cross3(m, B);
  const float3 mxmxB = cross3(m, mxB);
  const float3 k = make_float3(ph.g1 * mxB.x + ph.g2 * mxmxB.x, ph.g1 * mxB.y + ph.g2 * mxmxB.y,
                               ph.g1 * mxB.z + ph.g2 * mxmxB.z);
  if (kmag) *kmag = sqrtf(k.x * k.x + k.y * k.y + k.z * k.z);
  float3 nm;
  bool renorm = false;
  if (a.mode == 2) {
    nm = make_float3(m.x + a.dt * k.x, m.y + a.dt * k.y, m.z + a.dt * k.z);
    renorm = true;
  } else if (a.stage == 0) {
    *acc_out = k;
    const float h = 0.5f * a.dt;
    nm = make_float3(m0.x + h * k.x, m0.y + h * k.y, m0.z + h * k.z);
  } else if (a.stage < 3) {
    float3 s = accv;
    s.x = fmaf(2.f, k.x, s.x); s.y = fmaf(2.f, k.y, s.y); s.z = fmaf(2.f, k.z, s.z);
    *acc_out = s;
    const float h = (a.stage == 1) ? 0.5f * a.dt : a.dt;
    nm = make_float3(m0.x + h * k.x, m0.y + h * k.y, m0.z + h * k.z);
  } else {
    const float3 s = make_float3(accv.x + k.x, accv.y + k.y, accv.z + k.z);
    const float h = a.dt * (1.0f / 6.0f);
    nm = make_float3(m0.x + h * s.x, m0.y + h * s.y, m0.z + h * s.z);
    renorm = true;
  }
  if (renorm) {
    const float inv = rsqrtf(nm.x * nm.x + nm.y * nm.y + nm.z * nm.z);
    nm.x *= inv; nm.y *= inv; nm.z *= inv;
  }
  return nm;
}

// One cell given its demag field bd (tesla).  Mode 0 writes H; modes 1/2 write
// and return the next stage / new state.
template <bool PC = false>
__device__ __forceinline__ float3 cell_update(const StageArgs& a, const Phys& ph, const Dims& d,
                                              int x, int y, int z, float3 bd, float* kmag = nullptr) {
  const long long N = d.N;
  const long long cell = ((long long)z * d.ny + y) * d.nx + x;
  if (!MM_BC(x < d.nx && y < d.ny && z < d.nz)) return make_float3(0.f, 0.f, 0.f);
  const float* __restrict__ mi = a.m_in;
  // eq. 5 with eq. 7: a missing neighbour is the cell itself (clamped index)
  const long long row = d.nx, pl = (long long)d.nx * d.ny;
  const long long nb[6] = {cell - (x > 0 ? 1 : 0), cell + (x < d.nx - 1 ? 1 : 0),
                           cell - (y > 0 ? row : 0), cell + (y < d.ny - 1 ? row : 0),
                           cell - (z > 0 ? pl : 0), cell + (z < d.nz - 1 ? pl : 0)};
  float3 m, lap = make_float3(0.f, 0.f, 0.f);
  {
    float v[3][7];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[c][6] = ld_ro<PC>(mi + cell + c * N);
#pragma unroll
      for (int q = 0; q < 6; ++q) v[c][q] = ld_ro<PC>(mi + nb[q] + c * N);
    }
    m = make_float3(v[0][6], v[1][6], v[2][6]);
    lap.x = ((v[0][0] - m.x) + (v[0][1] - m.x)) + ((v[0][2] - m.x) + (v[0][3] - m.x)) + ((v[0][4] - m.x) + (v[0][5] - m.x));
    lap.y = ((v[1][0] - m.y) + (v[1][1] - m.y)) + ((v[1][2] - m.y) + (v[1][3] - m.y)) + ((v[1][4] - m.y) + (v[1][5] - m.y));
    lap.z = ((v[2][0] - m.z) + (v[2][1] - m.z)) + ((v[2][2] - m.z) + (v[2][3] - m.z)) + ((v[2][4] - m.z) + (v[2][5] - m.z));
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
    return m;
  }
  if (a.mode >= 3) {
    // the adjoint sweep (StageArgs): m holds lam_B, and L lam_B (exchange + demag,
    // tesla) closes the stage whose cotangent this kernel completes
    const float3 L = make_float3(bex.x + bd.x, bex.y + bd.y, bex.z + bd.z);
    const float3 ls = make_float3(a.adj_loc[cell] + L.x, a.adj_loc[cell + N] + L.y, a.adj_loc[cell + 2 * N] + L.z);
    const float3 lm = make_float3(a.adj_lam_m[cell] + ls.x, a.adj_lam_m[cell + N] + ls.y,
                                  a.adj_lam_m[cell + 2 * N] + ls.z);
    if (a.mode == 4) {
      a.adj_lam[cell] = lm.x; a.adj_lam[cell + N] = lm.y; a.adj_lam[cell + 2 * N] = lm.z;
      return m;
    }
    if (a.mode == 5) {   // lm is the cotangent of the previous step's end state: start its sweep
      float3 sq[4], Bq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sq[q] = make_float3(a.adj_sq[q][cell], a.adj_sq[q][cell + N], a.adj_sq[q][cell + 2 * N]);
        Bq[q] = make_float3(a.adj_Bq[q][cell], a.adj_Bq[q][cell + N], a.adj_Bq[q][cell + 2 * N]);
      }
      float3 lu, lamB, loc;
      adj_step_start(ph.g1, ph.g2, can, a.adj_dt, sq, Bq, lm, lu, lamB, loc);
      const float h = a.adj_dt * (1.0f / 6.0f);
      a.adj_lam_m[cell] = lu.x; a.adj_lam_m[cell + N] = lu.y; a.adj_lam_m[cell + 2 * N] = lu.z;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        float* lkq = a.adj_lk0 + 3 * N * q;
        const float f = q == 0 ? h : 2.f * h;   // lk_1 = dt/6 lu, lk_2 = lk_3 = dt/3 lu
        lkq[cell] = f * lu.x; lkq[cell + N] = f * lu.y; lkq[cell + 2 * N] = f * lu.z;
      }
      a.adj_loc[cell] = loc.x; a.adj_loc[cell + N] = loc.y; a.adj_loc[cell + 2 * N] = loc.z;
      a.adj_gh[cell] += lamB.x; a.adj_gh[cell + N] += lamB.y; a.adj_gh[cell + 2 * N] += lamB.z;
      a.adj_gku[cell] += ph.c_an_map * sq[3].x * lamB.x;   // c_an_map = 2 / Ms
      a.m_out[cell] = lamB.x; a.m_out[cell + N] = lamB.y; a.m_out[cell + 2 * N] = lamB.z;
      return lamB;
    }
    a.adj_lam_m[cell] = lm.x; a.adj_lam_m[cell + N] = lm.y; a.adj_lam_m[cell + 2 * N] = lm.z;
    const float3 lk = make_float3(a.adj_lk[cell] + a.adj_c * ls.x, a.adj_lk[cell + N] + a.adj_c * ls.y,
                                  a.adj_lk[cell + 2 * N] + a.adj_c * ls.z);
    a.adj_lk[cell] = lk.x; a.adj_lk[cell + N] = lk.y; a.adj_lk[cell + 2 * N] = lk.z;
    // open the next stage: the VJP of eq. 2 at its recorded state and field
    const float3 sv = make_float3(a.adj_s[cell], a.adj_s[cell + N], a.adj_s[cell + 2 * N]);
    const float3 Bv = make_float3(a.adj_B[cell], a.adj_B[cell + N], a.adj_B[cell + 2 * N]);
    float3 lamB, loc;
    llg_vjp(ph.g1, ph.g2, can, sv, Bv, lk, lamB, loc);
    a.adj_loc[cell] = loc.x; a.adj_loc[cell + N] = loc.y; a.adj_loc[cell + 2 * N] = loc.z;
    a.adj_gh[cell] += lamB.x; a.adj_gh[cell + N] += lamB.y; a.adj_gh[cell + 2 * N] += lamB.z;
    a.adj_gku[cell] += ph.c_an_map * sv.x * lamB.x;   // c_an_map = 2 / Ms
    a.m_out[cell] = lamB.x; a.m_out[cell + N] = lamB.y; a.m_out[cell + 2 * N] = lamB.z;
    return lamB;   // transformed along x by the caller for the next application of L
  }
  const float3 B = make_float3(bex.x + ban + bd.x + bz.x, bex.y + bd.y + bz.y, bex.z + bd.z + bz.z);
  if (a.B_out) {   // recorded for the adjoint sweep
    a.B_out[cell] = B.x;
    a.B_out[cell + N] = B.y;
    a.B_out[cell + 2 * N] = B.z;
  }
  float3 m0 = m, accv = m;
  if (a.mode == 1) {
    m0 = make_float3(ld_rw<PC>(a.m0 + cell), ld_rw<PC>(a.m0 + cell + N), ld_rw<PC>(a.m0 + cell + 2 * N));
    if (a.stage > 0)
      accv = make_float3(ld_rw<PC>(a.acc + cell), ld_rw<PC>(a.acc + cell + N), ld_rw<PC>(a.acc + cell + 2 * N));
  }
  float3 acc_out;
  const float3 nm = llg_stage(a, ph, m, B, m0, accv, &acc_out, kmag);
  if (a.mode == 1 && a.stage < 3) {
    a.acc[cell] = acc_out.x; a.acc[cell + N] = acc_out.y; a.acc[cell + 2 * N] = acc_out.z;
  }
  a.m_out[cell] = nm.x;
  a.m_out[cell + N] = nm.y;
  a.m_out[cell + 2 * N] = nm.z;
  return nm;
}

// V (2 or 4) consecutive cells x0 .. x0+V-1 of row (y, z) in modes 1/2 (nx a
// multiple of V, so every row and plane offset keeps the vector alignment):
// the same arithmetic as cell_update, with V-wide loads and stores.  The x
// neighbours inside the group come from the group's own load; the two outside
// it are scalar loads (clamped at the film edge by eq. 7).
template <int V> struct VecOf;
template <> struct VecOf<2> {
  using T = float2;
  __device__ static void get(const T& v, float* o) { o[0] = v.x; o[1] = v.y; }
  __device__ static T make(const float* o) { return make_float2(o[0], o[1]); }
};
template <> struct VecOf<4> {
  using T = float4;
  __device__ static void get(const T& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  __device__ static T make(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};

template <int V, bool PC = false>
__device__ __forceinline__ void cell_updateV(const StageArgs& a, const Phys& ph, const Dims& d, int x0, int y,
                                             int z, const float3 (&bd)[V], float3 (&nm)[V], float* kmag) {
  using Vec = VecOf<V>;
  using T = typename Vec::T;
  const long long N = d.N;
  const long long cell = ((long long)z * d.ny + y) * d.nx + x0;
  if (!MM_BC(x0 + V <= d.nx && y < d.ny && z < d.nz)) {
#pragma unroll
    for (int j = 0; j < V; ++j) nm[j] = make_float3(0.f, 0.f, 0.f);
    return;
  }
  const long long row = d.nx, pl = (long long)d.nx * d.ny;
  const long long oym = y > 0 ? -row : 0, oyp = y < d.ny - 1 ? row : 0;
  const long long ozm = z > 0 ? -pl : 0, ozp = z < d.nz - 1 ? pl : 0;
  float mv[3][V], lap[3][V];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* b = a.m_in + cell + c * N;
    float sv[V + 2], vym[V], vyp[V], vzm[V], vzp[V];
    Vec::get(ld_ro<PC>(reinterpret_cast<const T*>(b)), sv + 1);
    sv[0] = x0 > 0 ? ld_ro<PC>(b - 1) : sv[1];
    sv[V + 1] = x0 + V < d.nx ? ld_ro<PC>(b + V) : sv[V];
    Vec::get(ld_ro<PC>(reinterpret_cast<const T*>(b + oym)), vym);
    Vec::get(ld_ro<PC>(reinterpret_cast<const T*>(b + oyp)), vyp);
    Vec::get(ld_ro<PC>(reinterpret_cast<const T*>(b + ozm)), vzm);
    Vec::get(ld_ro<PC>(reinterpret_cast<const T*>(b + ozp)), vzp);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const float m = sv[j + 1];
      mv[c][j] = m;
      lap[c][j] = ((sv[j] - m) + (sv[j + 2] - m)) + ((vym[j] - m) + (vyp[j] - m)) + ((vzm[j] - m) + (vzp[j] - m));
    }
  }
  float can[V];
#pragma unroll
  for (int j = 0; j < V; ++j) can[j] = ph.c_an;
  if (a.kumap) {
    float ku[V];
    Vec::get(__ldg(reinterpret_cast<const T*>(a.kumap + cell)), ku);
#pragma unroll
    for (int j = 0; j < V; ++j) can[j] = ph.c_an_map * ku[j];
  }
  float hz[3][V];
#pragma unroll
  for (int j = 0; j < V; ++j) { hz[0][j] = ph.bx; hz[1][j] = ph.by; hz[2][j] = ph.bz; }
  if (a.hmap) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float h[V];
      Vec::get(__ldg(reinterpret_cast<const T*>(a.hmap + cell + c * N)), h);
#pragma unroll
      for (int j = 0; j < V; ++j) hz[c][j] += h[j];
    }
  }
  float m0v[3][V], accv[3][V];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int j = 0; j < V; ++j) { m0v[c][j] = mv[c][j]; accv[c][j] = mv[c][j]; }
    if (a.mode == 1) {
      Vec::get(ld_rw<PC>(reinterpret_cast<const T*>(a.m0 + cell + c * N)), m0v[c]);
      if (a.stage > 0) Vec::get(ld_rw<PC>(reinterpret_cast<const T*>(a.acc + cell + c * N)), accv[c]);
    }
  }
  float Bv[3][V], ao[3][V], no[3][V];
  float km = 0.f;
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const float3 m = make_float3(mv[0][j], mv[1][j], mv[2][j]);
    const float bex_x = ph.c_ex * lap[0][j], bex_y = ph.c_ex * lap[1][j], bex_z = ph.c_ex * lap[2][j];
    const float ban = can[j] * m.x;
    const float3 B = make_float3(bex_x + ban + bd[j].x + hz[0][j], bex_y + bd[j].y + hz[1][j],
                                 bex_z + bd[j].z + hz[2][j]);
    Bv[0][j] = B.x; Bv[1][j] = B.y; Bv[2][j] = B.z;
    float3 acc_out = make_float3(0.f, 0.f, 0.f);
    float kj = 0.f;
    nm[j] = llg_stage(a, ph, m, B, make_float3(m0v[0][j], m0v[1][j], m0v[2][j]),
                      make_float3(accv[0][j], accv[1][j], accv[2][j]), &acc_out, kmag ? &kj : nullptr);
    km = fmaxf(km, kj);
    ao[0][j] = acc_out.x; ao[1][j] = acc_out.y; ao[2][j] = acc_out.z;
    no[0][j] = nm[j].x; no[1][j] = nm[j].y; no[2][j] = nm[j].z;
  }
  if (kmag) *kmag = km;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (a.B_out) *reinterpret_cast<T*>(a.B_out + cell + c * N) = Vec::make(Bv[c]);
    if (a.mode == 1 && a.stage < 3) *reinterpret_cast<T*>(a.acc + cell + c * N) = Vec::make(ao[c]);
    *reinterpret_cast<T*>(a.m_out + cell + c * N) = Vec::make(no[c]);
  }
}

// The adjoint modes (3-5) of cell_update for V consecutive cells x0 .. x0+V-1
// (nx a multiple of V): the same per-cell arithmetic, with V-wide loads and
// stores of every field it touches.  m_in holds lam_B; nm returns what the
// scalar form returns (lam_B of the next application of L, or, in mode 4, the
// cells' own input).
template <int V, bool PC = false>
__device__ __forceinline__ void cell_adjV(const StageArgs& a, const Phys& ph, const Dims& d, int x0, int y, int z,
                                          const float3 (&bd)[V], float3 (&nm)[V]) {
  using Vec = VecOf<V>;
  using T = typename Vec::T;
  const long long N = d.N;
  const long long cell = ((long long)z * d.ny + y) * d.nx + x0;
  if (!MM_BC(x0 + V <= d.nx && y < d.ny && z < d.nz)) {
#pragma unroll
    for (int j = 0; j < V; ++j) nm[j] = make_float3(0.f, 0.f, 0.f);
    return;
  }
  auto ld3 = [&](const float* p, float (&o)[3][V]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) Vec::get(ld_rw<PC>(reinterpret_cast<const T*>(p + cell + c * N)), o[c]);
  };
  auto st3 = [&](float* p, const float (&v)[3][V]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) *reinterpret_cast<T*>(p + cell + c * N) = Vec::make(v[c]);
  };
  const long long row = d.nx, pl = (long long)d.nx * d.ny;
  const long long oym = y > 0 ? -row : 0, oyp = y < d.ny - 1 ? row : 0;
  const long long ozm = z > 0 ? -pl : 0, ozp = z < d.nz - 1 ? pl : 0;
  float mv[3][V], L[3][V];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* b = a.m_in + cell + c * N;
    float sv[V + 2], vym[V], vyp[V], vzm[V], vzp[V];
    Vec::get(ld_ro<PC>(reinterpret_cast<const T*>(b)), sv + 1);
    sv[0] = x0 > 0 ? ld_ro<PC>(b - 1) : sv[1];
    sv[V + 1] = x0 + V < d.nx ? ld_ro<PC>(b + V) : sv[V];
    Vec::get(ld_ro<PC>(reinterpret_cast<const T*>(b + oym)), vym);
    Vec::get(ld_ro<PC>(reinterpret_cast<const T*>(b + oyp)), vyp);
    Vec::get(ld_ro<PC>(reinterpret_cast<const T*>(b + ozm)), vzm);
    Vec::get(ld_ro<PC>(reinterpret_cast<const T*>(b + ozp)), vzp);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const float m = sv[j + 1];
      mv[c][j] = m;
      const float lap = ((sv[j] - m) + (sv[j + 2] - m)) + ((vym[j] - m) + (vyp[j] - m)) + ((vzm[j] - m) + (vzp[j] - m));
      L[c][j] = ph.c_ex * lap + (c == 0 ? bd[j].x : c == 1 ? bd[j].y : bd[j].z);
    }
  }
  float can[V];
#pragma unroll
  for (int j = 0; j < V; ++j) can[j] = ph.c_an;
  if (a.kumap) {
    float ku[V];
    Vec::get(__ldg(reinterpret_cast<const T*>(a.kumap + cell)), ku);
#pragma unroll
    for (int j = 0; j < V; ++j) can[j] = ph.c_an_map * ku[j];
  }
  // ls = loc + L lam_B closes the stage; lm = lam_m + ls
  float ls[3][V], lm[3][V];
  ld3(a.adj_loc, ls);
  ld3(a.adj_lam_m, lm);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int j = 0; j < V; ++j) {
      ls[c][j] = ls[c][j] + L[c][j];
      lm[c][j] = lm[c][j] + ls[c][j];
    }
  if (a.mode == 4) {
    st3(a.adj_lam, lm);
#pragma unroll
    for (int j = 0; j < V; ++j) nm[j] = make_float3(mv[0][j], mv[1][j], mv[2][j]);
    return;
  }
  float lamB[3][V], loc[3][V];
  if (a.mode == 5) {   // lm is the cotangent of the previous step's end state: start its sweep
    float lu[3][V], sx3[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      float3 sq[4], Bq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float s3[3][V], b3[3][V];
        ld3(a.adj_sq[q], s3);
        ld3(a.adj_Bq[q], b3);
        sq[q] = make_float3(s3[0][j], s3[1][j], s3[2][j]);
        Bq[q] = make_float3(b3[0][j], b3[1][j], b3[2][j]);
      }
      float3 u, lb, lc;
      adj_step_start(ph.g1, ph.g2, can[j], a.adj_dt, sq, Bq, make_float3(lm[0][j], lm[1][j], lm[2][j]), u, lb, lc);
      lu[0][j] = u.x; lu[1][j] = u.y; lu[2][j] = u.z;
      lamB[0][j] = lb.x; lamB[1][j] = lb.y; lamB[2][j] = lb.z;
      loc[0][j] = lc.x; loc[1][j] = lc.y; loc[2][j] = lc.z;
      sx3[j] = sq[3].x;
    }
    const float h = a.adj_dt * (1.0f / 6.0f);
    st3(a.adj_lam_m, lu);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float f = q == 0 ? h : 2.f * h;   // lk_1 = dt/6 lu, lk_2 = lk_3 = dt/3 lu
      float lk[3][V];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < V; ++j) lk[c][j] = f * lu[c][j];
      st3(a.adj_lk0 + 3 * N * q, lk);
    }
    st3(a.adj_loc, loc);
    float gh[3][V], gk[V];
    ld3(a.adj_gh, gh);
    Vec::get(ld_rw<PC>(reinterpret_cast<const T*>(a.adj_gku + cell)), gk);
#pragma unroll
    for (int j = 0; j < V; ++j) {
#pragma unroll
      for (int c = 0; c < 3; ++c) gh[c][j] += lamB[c][j];
      gk[j] += ph.c_an_map * sx3[j] * lamB[0][j];   // c_an_map = 2 / Ms
    }
    st3(a.adj_gh, gh);
    *reinterpret_cast<T*>(a.adj_gku + cell) = Vec::make(gk);
  } else {             // mode 3: close this stage, open the next one
    st3(a.adj_lam_m, lm);
    float lk[3][V], sv[3][V], Bv[3][V];
    ld3(a.adj_lk, lk);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int j = 0; j < V; ++j) lk[c][j] = lk[c][j] + a.adj_c * ls[c][j];
    st3(a.adj_lk, lk);
    // the VJP of eq. 2 at the next stage's recorded state and field
    ld3(a.adj_s, sv);
    ld3(a.adj_B, Bv);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      float3 lb, lc;
      llg_vjp(ph.g1, ph.g2, can[j], make_float3(sv[0][j], sv[1][j], sv[2][j]),
              make_float3(Bv[0][j], Bv[1][j], Bv[2][j]), make_float3(lk[0][j], lk[1][j], lk[2][j]), lb, lc);
      lamB[0][j] = lb.x; lamB[1][j] = lb.y; lamB[2][j] = lb.z;
      loc[0][j] = lc.x; loc[1][j] = lc.y; loc[2][j] = lc.z;
    }
    st3(a.adj_loc, loc);
    float gh[3][V], gk[V];
    ld3(a.adj_gh, gh);
    Vec::get(ld_rw<PC>(reinterpret_cast<const T*>(a.adj_gku + cell)), gk);
#pragma unroll
    for (int j = 0; j < V; ++j) {
#pragma unroll
      for (int c = 0; c < 3; ++c) gh[c][j] += lamB[c][j];
      gk[j] += ph.c_an_map * sv[0][j] * lamB[0][j];   // c_an_map = 2 / Ms
    }
    st3(a.adj_gh, gh);
    *reinterpret_cast<T*>(a.adj_gku + cell) = Vec::make(gk);
  }
  st3(a.m_out, lamB);
#pragma unroll
  for (int j = 0; j < V; ++j) nm[j] = make_float3(lamB[0][j], lamB[1][j], lamB[2][j]);
}

// ---------------------------------------------------------------------------
// k_x: CTA = (tile of TY rows along y, plane z), all three components.
// Inverse x transform of the field (complex-to-real, first nx points), the
// per-cell update, and -- when `fwd` is set -- the forward x transform of the
// state just written, stored back into the same tile of S for the next field
// evaluation (so a stage needs only k_yz + k_x).
// ---------------------------------------------------------------------------
// Rows per tile of the x kernels.
template <int HALF>
struct XTile {
  static constexpr int v = HALF <= 256 ? 8 : (HALF <= 512 ? 4 : 2);
};

template <int PADS>
__device__ __forceinline__ float& rowf(float2* row, int x) {
  float2& e = row[pidx<PADS>(x >> 1)];
  return (x & 1) ? e.y : e.x;
}

// The x transforms of a k_x tile at HALF = 256 with the TMA staging area
// (TY = 8: 24 rows [c][r], 384 threads), as two register passes of 16
// (256 = 16 x 16, fft.cuh reg_fft).  Thread t takes row rr = t % 24 and lane
// l = t / 24: rows fastest, so the 24 rows' reads of one staged kx are
// contiguous.  Pass 1 of lane l transforms the 16 values l + 16 j, multiplies
// output k1 by W_256^(l k1) and stores it at k1 17 + l, which is pidx<4>(16 k1
// + l) (the rows' padded layout); pass 2 of lane k1 transforms the 16 values
// k1 17 + l and stores X[k1 + 16 k2] at pidx<4>(k1 + 16 k2).  tws is the
// table exp(-2 pi i m / 512).
static constexpr int kXFusedHalf = 256;

template <int DIR>
__device__ __forceinline__ void x16_pass2(float2* row, int k1, int nout) {
  float2 u[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) u[q] = row[k1 * 17 + q];
  __syncthreads();   // every thread has read its pass-2 inputs before any output lands
  reg_fft<16, DIR>(u);
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const int n = k1 + 16 * k2;
    if (n < nout && MM_BC_SMEM(&row[pidx<4>(n)], sizeof(float2))) row[pidx<4>(n)] = u[brev(k2, 4)];
  }
}

// Inverse, with the complex-to-real pre-processing in pass 1: Z[k] =
// (X[k] + conj X[256-k]) + i W_512^-k (X[k] - conj X[256-k]) straight from the
// staged spectrum (stg0: kx 0..128, stg1: kx 129..257, [kx][c][TY]).  Only the
// first nout outputs are stored.
template <int TY>
__device__ __forceinline__ void x16_inverse_c2r(const float2* stg0, const float2* stg1, float2* rows, int RS,
                                                const float2* tws, int nout) {
  constexpr int H = kXFusedHalf, XB = 129, NR = 3 * TY;
  const int rr = threadIdx.x % NR, l = threadIdx.x / NR;
  const int c = rr / TY, r = rr % TY;
  float2* row = rows + rr * RS;
  auto stg = [&](int k) { return k < XB ? stg0[(k * 3 + c) * TY + r] : stg1[((k - XB) * 3 + c) * TY + r]; };
  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int k = l + 16 * j;
    const float2 Xa = stg(k), Xb = cconj(stg(H - k));
    v[j] = cadd(cadd(Xa, Xb), cmuli(cmul(csub(Xa, Xb), cconj(tws[k]))));
  }
  reg_fft<16, 1>(v);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    const float2 x = v[brev(k1, 4)];
    if (MM_BC_SMEM(&row[k1 * 17 + l], sizeof(float2))) row[k1 * 17 + l] = k1 ? cmul(x, cconj(tws[2 * ((l * k1) & (H - 1))])) : x;
  }
  __syncthreads();
  x16_pass2<1>(row, l, nout);
}

// Forward of the rows whose y is inside the film; only the first nin inputs
// are read (the rest are zeros: the upper half of every pass-1 sequence).
template <int TY>
__device__ __forceinline__ void x16_forward(float2* rows, int RS, const float2* tws, int nin, bool act) {
  constexpr int H = kXFusedHalf, NR = 3 * TY;
  const int rr = threadIdx.x % NR, l = threadIdx.x / NR;
  float2* row = rows + rr * RS;
  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int n = l + 16 * j;
    v[j] = (j < 8 && act && n < nin) ? row[pidx<4>(n)] : make_float2(0.f, 0.f);
  }
  reg_fft<16, -1, true>(v);
  if (act) {   // in place: thread (l, rr) overwrites only the slots it has read
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
      const float2 x = v[brev(k1, 4)];
      if (MM_BC_SMEM(&row[k1 * 17 + l], sizeof(float2))) row[k1 * 17 + l] = k1 ? cmul(x, tws[2 * ((l * k1) & (H - 1))]) : x;
    }
  }
  __syncthreads();
  x16_pass2<-1>(row, l, act ? H : 0);
}

// TMA: the S tile arrives as two tiled tensor copies (kx 0..128 and 129..257)
// into a staging area [kx][c][TY] (xmap: the tensor map of S), instead of
// per-thread copies; the C2R pre-processing then reads the staging area.
template <int HALF, int TYV = XTile<HALF>::v, bool TMA = false, bool PC = false, bool ADJ = false>
__device__ __forceinline__ void body_x(const StageArgs& a, const Phys& ph, float2* __restrict__ S,
                                       const float2* __restrict__ twP, const Dims& d, int TY, int fwd, int z,
                                       int y0, const CUtensorMap* xmap = nullptr) {
  if constexpr (HALF == 0) {
    float kmax = 0.f;
    for (int r = threadIdx.x; r < TY; r += blockDim.x) {
      const int y = y0 + r;
      if (y >= d.ny) continue;
      float2* s0 = S + ((long long)0 * d.nz + z) * d.ny + y;
      float2* s1 = S + ((long long)1 * d.nz + z) * d.ny + y;
      float2* s2 = S + ((long long)2 * d.nz + z) * d.ny + y;
      const float3 bd = make_float3(ph.c_d * s0->x, ph.c_d * s1->x, ph.c_d * s2->x);
      float km = 0.f;
      const float3 nm = cell_update<PC>(a, ph, d, 0, y, z, bd, a.maxdmdt ? &km : nullptr);
      kmax = fmaxf(kmax, km);
      if (fwd) {
        *s0 = make_float2(nm.x, 0.f);
        *s1 = make_float2(nm.y, 0.f);
        *s2 = make_float2(nm.z, 0.f);
      }
    }
    if (a.maxdmdt) {
      const unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(kmax));
      if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned*>(a.maxdmdt), v);
    }
  } else {
    constexpr int T = TeamOf<HALF>::v;
    constexpr int P = 2 * HALF;
    constexpr int PADS = 4;
    constexpr int RS = HALF + (HALF + 1) / 16 + 2;
    constexpr int TY = TYV;   // rows per tile (the launcher uses the same value)
    constexpr int XV = 2;                 // cells per thread of the vector update
    extern __shared__ float2 sm[];
    float2* tws = sm;
    float2* rows = sm + P;   // [3][TY] rows, element k at pidx(k), k <= HALF
    const int total = (HALF + 1) * 3 * TY;
    const int NR = 3 * TY;
    const int npair = HALF / 2 + 1;
    // Z[k] = (X[k] + conj X[HALF-k]) + i W_P^{-k} (X[k] - conj X[HALF-k]), k < HALF,
    // for the pair (k, HALF - k) of row rr
    auto pre_pair = [&](int rr, int k, float2 Xa, float2 Xb) {
      float2* row = rows + rr * RS;
      const int k2 = HALF - k;
      const float2 w = tws[k];
      const float2 wm = make_float2(w.x, -w.y);
      const float2 Za = cadd(cadd(Xa, cconj(Xb)), cmuli(cmul(csub(Xa, cconj(Xb)), wm)));
      if (!MM_BC_SMEM(&row[pidx<PADS>(k2)], sizeof(float2)) || !MM_BC_SMEM(&row[pidx<PADS>(k)], sizeof(float2))) {
      } else if (k == 0 || k == k2) {
        row[pidx<PADS>(k)] = Za;
      } else {
        const float2 wm2 = make_float2(-w.x, -w.y);
        const float2 Zb = cadd(cadd(Xb, cconj(Xa)), cmuli(cmul(csub(Xb, cconj(Xa)), wm2)));
        row[pidx<PADS>(k)] = Za;
        row[pidx<PADS>(k2)] = Zb;
      }
    };
    if constexpr (TMA) {
      static_assert(HALF >= 4 && HALF <= 256, "two boxes of 129 kx");
      constexpr int XB = 129;   // kx per tensor copy (two cover hx <= 257)
      constexpr uint32_t box_bytes = XB * 3 * TY * sizeof(float2);
      // two staging boxes [kx][c][TY] after the rows, each on a 128-byte boundary
      float2* rend = rows + 3 * TY * RS;
      const uint32_t s0 = (smem_u32(rend) + 127u) & ~127u;
      const uint32_t s1 = (s0 + box_bytes + 127u) & ~127u;
      float2* stg0 = rend + (s0 - smem_u32(rend)) / sizeof(float2);
      float2* stg1 = stg0 + (s1 - s0) / sizeof(float2);
      __shared__ __align__(8) uint64_t xbar;
      if (threadIdx.x == 0) {
        mbar_init(&xbar, 1);
        mbar_fence_init();
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&xbar, 2 * box_bytes);
        tma_load_4d(stg0, xmap, 2 * y0, z, 0, 0, &xbar);    // x: float index of y0 (a multiple of 16)
        tma_load_4d(stg1, xmap, 2 * y0, z, 0, XB, &xbar);
      }
      for (int i = threadIdx.x; i < P; i += blockDim.x) tws[i] = twP[i];
      const bool ok = mbar_wait_bounded(&xbar, 0);
      if (!__syncthreads_and(ok)) {   // uniform exit; copies in flight get one more bounded wait
        if (threadIdx.x == 0 && a.flag) atomicOr(a.flag + 1, 1);
        mbar_wait_bounded(&xbar, 0);
        return;
      }
      // rows fastest: the staging reads are contiguous across lanes (at HALF =
      // 256 the inverse transform's first pass reads the staging area itself)
      if constexpr (HALF != kXFusedHalf)
      for (int i = threadIdx.x; i < NR * npair; i += blockDim.x) {
        const int r = i % TY, c = (i / TY) % 3, k = i / (3 * TY), kb = HALF - k;
        const float2 Xa = k < XB ? stg0[(k * 3 + c) * TY + r] : stg1[((k - XB) * 3 + c) * TY + r];
        const float2 Xb = kb < XB ? stg0[(kb * 3 + c) * TY + r] : stg1[((kb - XB) * 3 + c) * TY + r];
        pre_pair(c * TY + r, k, Xa, Xb);
      }
    } else {
      // the tile of S arrives by asynchronous copies (all in flight at once)
      for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int r = i % TY, rest = i / TY;
        const int c = rest % 3, k = rest / 3;
        const int y = y0 + r;
        float2* dst = rows + (c * TY + r) * RS + pidx<PADS>(k);
        const float2* src = S + (((long long)k * 3 + c) * d.nz + z) * d.ny + y;
        if (y >= d.ny) *dst = make_float2(0.f, 0.f);
        else if constexpr (PC) *dst = __ldcg(src);
        else cp_async8(dst, src);
      }
      cp_async_commit();
      for (int i = threadIdx.x; i < P; i += blockDim.x) tws[i] = twP[i];
      cp_async_wait_all();
      __syncthreads();
      for (int i = threadIdx.x; i < NR * npair; i += blockDim.x) {
        const int rr = i / npair, k = i % npair;
        pre_pair(rr, k, rows[rr * RS + pidx<PADS>(k)], rows[rr * RS + pidx<PADS>(HALF - k)]);
      }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int team = threadIdx.x / T, t = threadIdx.x % T, nteams = blockDim.x / T;
    const unsigned mask = team_mask<T>(lane);
    if constexpr (TMA && HALF == kXFusedHalf) {
      static_assert(TY == 8, "24 rows x 16 lanes = 384 threads");
      constexpr uint32_t box_bytes = 129 * 3 * TY * sizeof(float2);
      float2* rend = rows + 3 * TY * RS;
      const uint32_t s0 = (smem_u32(rend) + 127u) & ~127u;
      const uint32_t s1 = (s0 + box_bytes + 127u) & ~127u;
      float2* stg0 = rend + (s0 - smem_u32(rend)) / sizeof(float2);
      x16_inverse_c2r<TY>(stg0, stg0 + (s1 - s0) / sizeof(float2), rows, RS, tws, (d.nx + 1) / 2);
    } else {
      for (int rr = team; rr < NR; rr += nteams) team_fft<HALF, T, 1, 2, PADS>(rows + rr * RS, t, mask, tws);
    }
    __syncthreads();
    float kmax = 0.f;
    if ((a.mode == 1 || a.mode == 2 || (ADJ && a.mode >= 3)) && (d.nx % XV) == 0) {
      // XV consecutive cells per thread (vector loads and stores); in the
      // adjoint instances (ADJ) the adjoint modes 3-5 through cell_adjV
      constexpr int Q = HALF / XV;
      for (int i = threadIdx.x; i < TY * Q; i += blockDim.x) {
        const int r = i / Q, x0 = (i % Q) * XV;
        if (x0 >= d.nx) continue;
        const int y = y0 + r;
        if (y >= d.ny) continue;
        float2* rw[3] = {rows + (0 * TY + r) * RS, rows + (1 * TY + r) * RS, rows + (2 * TY + r) * RS};
        float3 bd[XV], nm[XV];
#pragma unroll
        for (int h = 0; h < XV / 2; ++h) {
          const float2 p0 = rw[0][pidx<PADS>((x0 >> 1) + h)], p1 = rw[1][pidx<PADS>((x0 >> 1) + h)],
                       p2 = rw[2][pidx<PADS>((x0 >> 1) + h)];
          bd[2 * h] = make_float3(ph.c_d * p0.x, ph.c_d * p1.x, ph.c_d * p2.x);
          bd[2 * h + 1] = make_float3(ph.c_d * p0.y, ph.c_d * p1.y, ph.c_d * p2.y);
        }
        float km = 0.f;
        if constexpr (ADJ) {
          if (a.mode >= 3) cell_adjV<XV, PC>(a, ph, d, x0, y, z, bd, nm);
          else cell_updateV<XV, PC>(a, ph, d, x0, y, z, bd, nm, a.maxdmdt ? &km : nullptr);
        } else {
          cell_updateV<XV, PC>(a, ph, d, x0, y, z, bd, nm, a.maxdmdt ? &km : nullptr);
        }
        kmax = fmaxf(kmax, km);
        if (fwd) {
#pragma unroll
          for (int h = 0; h < XV / 2; ++h) {
            rw[0][pidx<PADS>((x0 >> 1) + h)] = make_float2(nm[2 * h].x, nm[2 * h + 1].x);
            rw[1][pidx<PADS>((x0 >> 1) + h)] = make_float2(nm[2 * h].y, nm[2 * h + 1].y);
            rw[2][pidx<PADS>((x0 >> 1) + h)] = make_float2(nm[2 * h].z, nm[2 * h + 1].z);
          }
        }
      }
    } else
    for (int i = threadIdx.x; i < TY * HALF; i += blockDim.x) {
      const int r = i / HALF, x = i % HALF;   // nx <= HALF
      if (x >= d.nx) continue;
      const int y = y0 + r;
      if (y >= d.ny) continue;
      float& f0 = rowf<PADS>(rows + (0 * TY + r) * RS, x);
      float& f1 = rowf<PADS>(rows + (1 * TY + r) * RS, x);
      float& f2 = rowf<PADS>(rows + (2 * TY + r) * RS, x);
      const float3 bd = make_float3(ph.c_d * f0, ph.c_d * f1, ph.c_d * f2);
      float km = 0.f;
      const float3 nm = cell_update<PC>(a, ph, d, x, y, z, bd, a.maxdmdt ? &km : nullptr);
      kmax = fmaxf(kmax, km);
      if (fwd) { f0 = nm.x; f1 = nm.y; f2 = nm.z; }
    }
    if (a.maxdmdt) {   // max |dm/dt| of the tile (non-negative floats order like their bit patterns)
      const unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(kmax));
      if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned*>(a.maxdmdt), v);
    }
    if (!fwd) return;
    __syncthreads();
    // zero padding nx..P-1 of every valid row, then the forward half-length transform
    // zero padding nx..P-1: the first pass reads only the (nx+1)/2 packed samples;
    // for odd nx the partner of the last sample is cleared below
    if (d.nx & 1) {
      for (int rr = threadIdx.x; rr < NR; rr += blockDim.x) rowf<PADS>(rows + rr * RS, d.nx) = 0.f;
    }
    __syncthreads();
    const int nin = (d.nx + 1) / 2;
    if constexpr (TMA && HALF == kXFusedHalf) {
      x16_forward<TY>(rows, RS, tws, nin, y0 + (int)(threadIdx.x % NR) % TY < d.ny);
    } else {
      for (int rr = team; rr < NR; rr += nteams) {
        if (y0 + rr % TY >= d.ny) continue;
        team_fft_io<HALF, T, -1, 2, PADS, PADS, PADS>(rows + rr * RS, t, mask, tws, nin, HALF);
      }
    }
    __syncthreads();
    // X[k] = 1/2 (Z[k] + conj Z[-k]) - i/2 W_P^k (Z[k] - conj Z[-k]), by pairs (k, HALF-k)
    if constexpr (TMA) {
      // into the staging boxes (rows fastest), then two tensor stores of the tile
      constexpr int XB = 129;
      constexpr uint32_t box_bytes = XB * 3 * TY * sizeof(float2);
      float2* rend = rows + 3 * TY * RS;
      const uint32_t s0 = (smem_u32(rend) + 127u) & ~127u;
      const uint32_t s1 = (s0 + box_bytes + 127u) & ~127u;
      float2* stg0 = rend + (s0 - smem_u32(rend)) / sizeof(float2);
      float2* stg1 = stg0 + (s1 - s0) / sizeof(float2);
      auto put = [&](int k, int c, int r, float2 v) {
        if (k < XB) stg0[(k * 3 + c) * TY + r] = v;
        else stg1[((k - XB) * 3 + c) * TY + r] = v;
      };
      for (int i = threadIdx.x; i < NR * npair; i += blockDim.x) {
        const int r = i % TY, c = (i / TY) % 3, k = i / (3 * TY);
        const float2* row = rows + (c * TY + r) * RS;
        const int k2 = HALF - k;
        if (k == 0) {
          const float2 z0 = row[pidx<PADS>(0)];
          put(0, c, r, make_float2(z0.x + z0.y, 0.f));
          put(HALF, c, r, make_float2(z0.x - z0.y, 0.f));
        } else if (k == k2) {
          put(k, c, r, cconj(row[pidx<PADS>(k)]));
        } else {
          const float2 zk = row[pidx<PADS>(k)], zc = row[pidx<PADS>(k2)];
          const float2 w = tws[k];
          const float2 d1 = csub(zk, cconj(zc));
          put(k, c, r, cscale(cadd(cadd(zk, cconj(zc)), cmul(make_float2(d1.y, -d1.x), w)), 0.5f));
          const float2 w2 = make_float2(-w.x, w.y);            // W_P^{HALF-k} = -conj W_P^k
          const float2 d2 = csub(zc, cconj(zk));
          put(k2, c, r, cscale(cadd(cadd(zc, cconj(zk)), cmul(make_float2(d2.y, -d2.x), w2)), 0.5f));
        }
      }
      fence_proxy_async_smem();   // the tensor stores read the staging area (async proxy)
      __syncthreads();
      if (threadIdx.x == 0) {
        tma_store_4d(xmap, stg0, 2 * y0, z, 0, 0);
        tma_store_4d(xmap, stg1, 2 * y0, z, 0, XB);
        bulk_commit();
        bulk_wait_read_all();   // the staging area stays valid until the stores have read it
      }
      return;
    }
    for (int i = threadIdx.x; i < NR * npair; i += blockDim.x) {
      const int rr = i / npair, k = i % npair;
      float2* row = rows + rr * RS;
      const int k2 = HALF - k;
      if (k == 0) {
        const float2 z0 = row[pidx<PADS>(0)];
        row[pidx<PADS>(0)] = make_float2(z0.x + z0.y, 0.f);
        row[pidx<PADS>(HALF)] = make_float2(z0.x - z0.y, 0.f);
      } else if (k == k2) {
        row[pidx<PADS>(k)] = cconj(row[pidx<PADS>(k)]);
      } else {
        const float2 zk = row[pidx<PADS>(k)], zc = row[pidx<PADS>(k2)];
        const float2 w = tws[k];
        const float2 d1 = csub(zk, cconj(zc));
        const float2 Xk = cscale(cadd(cadd(zk, cconj(zc)), cmul(make_float2(d1.y, -d1.x), w)), 0.5f);
        const float2 w2 = make_float2(-w.x, w.y);            // W_P^{HALF-k} = -conj W_P^k
        const float2 d2 = csub(zc, cconj(zk));
        const float2 Xc = cscale(cadd(cadd(zc, cconj(zk)), cmul(make_float2(d2.y, -d2.x), w2)), 0.5f);
        row[pidx<PADS>(k)] = Xk;
        row[pidx<PADS>(k2)] = Xc;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int r = i % TY, rest = i / TY;
      const int c = rest % 3, k = rest / 3;
      const int y = y0 + r;
      if (y < d.ny && MM_BC(k < d.hx && z < d.nz))
        S[(((long long)k * 3 + c) * d.nz + z) * d.ny + y] = rows[(c * TY + r) * RS + pidx<PADS>(k)];
    }
  }
}

// DRIVE: the applied field and LLG prefactors of this stage come from the field
// program's drive slot (a.drive, device memory) instead of the kernel parameters
// (a separate instantiation, so the constant-field kernel keeps them as
// constant-bank operands).
template <int HALF, bool DRIVE, int TYV, bool TMA, bool ADJ = false>
// At most 384 threads (3 TY / 2 teams of 32 lanes for 8-row tiles); two CTAs
// per SM up to px = 512 (the long rows beyond need the registers, and so does
// the adjoint sweep's two-cell epilogue)
__global__ void __launch_bounds__(384, (HALF >= 512 || ADJ) ? 1 : 2) k_x(StageArgs a, Phys ph, float2* __restrict__ S,
                                           const float2* __restrict__ twP, Dims d, int TY, int fwd,
                                           const __grid_constant__ CUtensorMap xmap) {
  MM_BC_ENTER(d.flag);
  grid_dep_wait();     // S, the stage states and the drive slots: written by the kernels before
  grid_dep_launch();
  if constexpr (DRIVE) {
    ph.bx = a.drive[0]; ph.by = a.drive[1]; ph.bz = a.drive[2];
    ph.g1 = a.drive[3]; ph.g2 = a.drive[4];
  }
  body_x<HALF, TYV, TMA, false, ADJ>(a, ph, S, twP, d, TY, fwd, blockIdx.y, blockIdx.x * TY, &xmap);
}

// ---------------------------------------------------------------------------
// launch geometry and dispatch
// ---------------------------------------------------------------------------
static inline int pow2_ceil(int v) {
  int p = 1;
  while (p < v) p *= 2;
  return p;
}

static inline int nzm_of(int nz) { return pow2_ceil(nz); }

static inline int xtile(int half) { return half <= 256 ? 16 : (half <= 512 ? 8 : 4); }
static inline int x_tile(int half) { return half <= 256 ? 8 : (half <= 512 ? 4 : 2); }
static inline int x_rs(int half) { return half + (half + 1) / 16 + 2; }

static inline int yz_rs(int py) { return py + (py >= 32 ? py / 16 : 0) + 2; }
// Does a column of the thinnest film of this plane class (nz = NZM / 2 + 1)
// fit one CTA's shared memory?  (yz_smem at that nz, FP32 path, plus the
// static shared memory.)
__host__ __device__ constexpr bool yz_col_fits(int PY, int NZM) {
  return 8ull * ((unsigned long long)PY + 3ull * (NZM > 1 ? NZM / 2 + 1 : 1) *
                                              (PY + (PY >= 32 ? PY / 16 : 0) + 2)) + 64 <= 227ull * 1024;
}
static inline size_t yz_smem(const Dims& d) {
  size_t b = sizeof(float2) * ((size_t)d.py + 3ull * d.nz * yz_rs(d.py));
  if (d.prec) b += mm_nzm(d.nz) == 8 ? zs::Dft<8>::bytes : zs::Dft<16>::bytes;
  return b;
}
static inline size_t x_smem(int half, int ty = 0, bool tma = false) {
  if (half == 0) return 0;
  const int t = ty ? ty : x_tile(half);
  return sizeof(float2) * ((size_t)2 * half + 3ull * t * x_rs(half) + (tma ? 2ull * 129 * 3 * t + 32 : 0));
}

static constexpr size_t kMaxSmem = 227 * 1024;

// Raise a kernel's dynamic shared-memory limit to everything its static shared
// memory leaves free (once per kernel; a host attribute, not a stream operation).
template <typename K>
static inline cudaError_t allow_max_smem(K kernel, bool& done) {
  if (done) return cudaSuccess;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxSmem - fa.sharedSizeBytes));
  if (e == cudaSuccess) done = true;
  return e;
}

static constexpr size_t kZtBudget = 200 * 1024;   // shared memory of one k_zt CTA (its ky block)

// shared memory of a k_zt CTA with a block of kb ky: the data plus, at most,
// the tensor rows of kb + 1 folded ky (a block that straddles py/2 folds onto
// fewer rows)
static inline size_t zt_smem(const Dims& d, int kb) {
  return sizeof(float2) * 3ull * d.nz * kb + sizeof(float) * 6ull * (d.nz + 4) * (kb + 1);
}

// ky block the split pass uses: the tuned value, else what a CTA's shared
// memory holds (mm_zt_kb_max), halved while the launch would not fill two
// waves of the 148 SMs
static inline int zt_kb(const Dims& d) {
  const int kmax = mm_zt_kb_max(d);
  if (d.ztkb > 0) return d.ztkb < kmax ? d.ztkb : kmax;   // tuned
  int kb = kmax;
  while (kb >= 16 && (long long)d.hx * ((d.py + kb - 1) / kb) < 2 * 148) kb /= 2;
  return kb;
}

// Launch with programmatic stream serialization (when d.pdl): the kernel's
// blocks may start while the kernel before it in the stream drains, and wait
// (grid_dep_wait) before they touch anything that kernel writes.
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(const Dims& d, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = d.pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// --- x forward (prologue: S <- transform of a state) ------------------------
template <int HALF>
static cudaError_t run_xfwd(const Dims& d, const float* m, const float2* tw, float2* S, cudaStream_t s) {
  const int P = HALF == 0 ? 1 : 2 * HALF;
  const int TY = HALF == 0 ? 32 : xtile(HALF);
  const int T = HALF == 0 ? 1 : TeamOf<(HALF > 0 ? HALF : 1)>::v;
  int threads = HALF == 0 ? 32 : TY * T;
  if (threads < 32) threads = 32;
  if (threads > 512) threads = 512;
  const size_t smem = HALF == 0 ? 0 : sizeof(float2) * ((size_t)P + (size_t)TY * (HALF + 1));
  static bool attr = false;
  if (cudaError_t e = allow_max_smem(k_xfwd<HALF>, attr)) return e;
  dim3 grid((d.ny + TY - 1) / TY, d.nz, 3);
  k_xfwd<HALF><<<grid, threads, smem, s>>>(m, S, tw + P, d, TY);
  return cudaGetLastError();
}

// --- x inverse + update (+ forward of the new state) -------------------------
template <int HALF, int TYV, bool TMA>
static cudaError_t run_x_ty(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                            cudaStream_t s, int fwd) {
  const int P = HALF == 0 ? 1 : 2 * HALF;
  const int TY = HALF == 0 ? 32 : TYV;
  const int T = HALF == 0 ? 1 : TeamOf<(HALF > 0 ? HALF : 1)>::v;
  int threads = HALF == 0 ? 32 : ((3 * TY + 1) / 2) * T;
  threads = (threads + 31) / 32 * 32;
  if (threads < 128) threads = 128;
  if (threads > 512) threads = 512;
  static bool attr = false, attr_d = false, attr_a = false;
  dim3 grid((d.ny + TY - 1) / TY, d.nz, 1);
  const size_t sm = x_smem(HALF, HALF == 0 ? 0 : TY, TMA);
  alignas(64) CUtensorMap map;
  if (TMA) map = *a.xmap;
  else memset(&map, 0, sizeof map);
  const float2* twP = tw + P;
  if (a.drive) {
    if (cudaError_t e = allow_max_smem(k_x<HALF, true, TYV, TMA>, attr_d)) return e;
    return launch_pdl(d, k_x<HALF, true, TYV, TMA>, grid, dim3(threads), sm, s, a, ph, S, twP, d, TY, fwd, map);
  }
  if (a.mode >= 3) {   // the adjoint sweep: its own instance, so the others keep their registers
    if (cudaError_t e = allow_max_smem(k_x<HALF, false, TYV, TMA, true>, attr_a)) return e;
    return launch_pdl(d, k_x<HALF, false, TYV, TMA, true>, grid, dim3(threads), sm, s, a, ph, S, twP, d, TY, fwd,
                      map);
  }
  if (cudaError_t e = allow_max_smem(k_x<HALF, false, TYV, TMA>, attr)) return e;
  return launch_pdl(d, k_x<HALF, false, TYV, TMA>, grid, dim3(threads), sm, s, a, ph, S, twP, d, TY, fwd, map);
}

// Rows per tile: the default, or 2 / 1 while fewer tiles than SMs would leave
// most of them idle (small films such as the paper's 166 x 42 x 1 run: 6 tiles
// of 8 rows, 42 of 1)
template <int HALF>
static cudaError_t run_x(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                         cudaStream_t s, int fwd) {
  constexpr int TD = XTile<HALF>::v;
  if constexpr (HALF >= 4 && HALF <= 256) {
    if ((long long)((d.ny + TD - 1) / TD) * d.nz < 148) {
      if ((long long)((d.ny + 1) / 2) * d.nz >= 148) return run_x_ty<HALF, 2, false>(d, ph, a, tw, S, s, fwd);
      return run_x_ty<HALF, 1, false>(d, ph, a, tw, S, s, fwd);
    }
    if (a.xmap) return run_x_ty<HALF, TD, true>(d, ph, a, tw, S, s, fwd);
  }
  return run_x_ty<HALF, TD, false>(d, ph, a, tw, S, s, fwd);
}

// --- y/z pass ------------------------------------------------------------------
template <int PY, int NZM>
static cudaError_t run_yz_t(const Dims& d, const float2* tw, float2* S, const float* Kh, int* flag, const Tick& tk,
                            cudaStream_t s) {
  // only the instances whose smallest column (nz = NZM / 2 + 1 planes) fits a
  // CTA exist; mm_yz_fits never routes a larger column here
  if constexpr (!yz_col_fits(PY, NZM)) {
    return cudaErrorInvalidValue;
  } else {
    if constexpr (PY >= 128 && (NZM == 8 || NZM == 16)) {
      if (d.prec == MM_SPLIT_BF16 || d.prec == MM_SPLIT_FP16) {
        static bool attr1 = false, attr2 = false;
        if (d.prec == MM_SPLIT_BF16) {
          if (cudaError_t e = allow_max_smem(k_yz<PY, NZM, MM_SPLIT_BF16>, attr1)) return e;
          return launch_pdl(d, k_yz<PY, NZM, MM_SPLIT_BF16>, dim3(d.hx), dim3(512), yz_smem(d), s, S, Kh, tw + PY, d,
                            flag, tk);
        }
        if (cudaError_t e = allow_max_smem(k_yz<PY, NZM, MM_SPLIT_FP16>, attr2)) return e;
        return launch_pdl(d, k_yz<PY, NZM, MM_SPLIT_FP16>, dim3(d.hx), dim3(512), yz_smem(d), s, S, Kh, tw + PY, d,
                          flag, tk);
      }
    }
    if (d.prec) return cudaErrorInvalidValue;
    static bool attr = false;
    if (cudaError_t e = allow_max_smem(k_yz<PY, NZM, 0>, attr)) return e;
    return launch_pdl(d, k_yz<PY, NZM, 0>, dim3(d.hx), dim3(512), yz_smem(d), s, S, Kh, tw + PY, d, flag, tk);
  }
}

#define MM_NZ_SWITCH(nz, CALL)          \
  switch (nzm_of(nz)) {                 \
    case 1: return CALL(1);             \
    case 2: return CALL(2);             \
    case 4: return CALL(4);             \
    case 8: return CALL(8);             \
    case 16: return CALL(16);           \
  }                                     \
  return cudaErrorInvalidValue;

template <int PY>
static cudaError_t run_yz_nz(const Dims& d, const float2* tw, float2* S, const float* Kh, int* flag, const Tick& tk,
                             cudaStream_t s) {
  // thick films (33..64 and 17..32 planes): the chunked z product
  if (nzm_of(d.nz) == 64) return run_yz_t<PY, 64>(d, tw, S, Kh, flag, tk, s);
  if (nzm_of(d.nz) == 32) return run_yz_t<PY, 32>(d, tw, S, Kh, flag, tk, s);
#define MM_CALL_YZ(Z) run_yz_t<PY, Z>(d, tw, S, Kh, flag, tk, s)
  MM_NZ_SWITCH(d.nz, MM_CALL_YZ)
#undef MM_CALL_YZ
}

template <int PY>
static cudaError_t run_yt(const Dims& d, const float2* tw, float2* S, int dir, const Tick& tk, cudaStream_t s) {
  constexpr int TM = TeamOf<PY>::v;
  const int threads = 256, nrows = threads / TM;
  const size_t smem = sizeof(float2) * ((size_t)PY + (size_t)nrows * YzLayout<PY>::RS);
  dim3 grid(d.hx, (3 * d.nz + nrows - 1) / nrows);
  if (dir < 0) {
    static bool attr = false;
    if (cudaError_t e = allow_max_smem(k_yt<PY, -1>, attr)) return e;
    return launch_pdl(d, k_yt<PY, -1>, grid, dim3(threads), smem, s, S, d.T, tw + PY, d, tk);
  } else {
    static bool attr = false;
    if (cudaError_t e = allow_max_smem(k_yt<PY, 1>, attr)) return e;
    return launch_pdl(d, k_yt<PY, 1>, grid, dim3(threads), smem, s, S, d.T, tw + PY, d, Tick{});
  }
}

template <int NZM>
static cudaError_t run_zt(const Dims& d, const float* Kh, cudaStream_t s) {
  const int kb = zt_kb(d);
  // one warp per task (10 positions, or one position per 3 NZM/16 lanes for
  // NZM > 16), at most 16 warps
  const int per_warp = NZM > 16 ? 32 / (3 * (NZM / 16)) : 10;
  int warps = (kb + per_warp - 1) / per_warp;
  if (warps > 16) warps = 16;
  static bool attr = false;
  if (cudaError_t e = allow_max_smem(k_zt<NZM>, attr)) return e;
  dim3 grid(d.hx, (d.py + kb - 1) / kb);
  return launch_pdl(d, k_zt<NZM>, grid, dim3(32 * warps), zt_smem(d, kb), s, d.T, Kh, d, kb);
}

// ---------------------------------------------------------------------------
// Batched launches: CTA i works on film map[i].x, tile map[i].y.  All films of
// a launch share the padded sizes (the template parameters); their other sizes,
// buffers and parameters come from the BatchFilm array.
// ---------------------------------------------------------------------------
template <int HALF>
__global__ void __launch_bounds__(512) kb_xfwd(const BatchFilm* __restrict__ F, const int2* __restrict__ map,
                                               int TY) {
  const int2 ft = map[blockIdx.x];
  const BatchFilm& f = F[ft.x];
  MM_BC_ENTER(f.d.flag);
  if (!f.active) return;
  const int ntyl = (f.d.ny + TY - 1) / TY;
  const int c = ft.y / (f.d.nz * ntyl), rem = ft.y % (f.d.nz * ntyl);
  constexpr int P = HALF == 0 ? 1 : 2 * HALF;
  body_xfwd<HALF>(f.m0, f.S, f.tw + P, f.d, TY, c, rem / ntyl, (rem % ntyl) * TY);
}

template <int PY, int NZM>
__global__ void __launch_bounds__(512, 1) kb_yz(const BatchFilm* __restrict__ F, const int2* __restrict__ map,
                                                 int* flag) {
  const int2 ft = map[blockIdx.x];
  const BatchFilm& f = F[ft.x];
  MM_BC_ENTER(f.d.flag);
  if (!f.active) return;
  body_yz<PY, NZM>(f.S, f.Kh, f.tw + PY, f.d, flag, ft.y);
}

template <int HALF>
__global__ void __launch_bounds__(512) kb_x(const BatchFilm* __restrict__ F, const int2* __restrict__ map, int TY,
                                            int stage, float dt) {
  const int2 ft = map[blockIdx.x];
  const BatchFilm& f = F[ft.x];
  MM_BC_ENTER(f.d.flag);
  if (!f.active) return;
  const int ntyl = (f.d.ny + TY - 1) / TY;
  StageArgs a = {};
  a.mode = 1;
  a.stage = stage;
  a.dt = dt;
  a.m0 = f.m0;
  a.acc = f.acc;
  a.hmap = f.hmap;
  a.kumap = f.kumap;
  a.m_in = stage == 0 ? f.m0 : (stage == 2 ? f.stB : f.stA);
  a.m_out = stage == 0 ? f.stA : (stage == 1 ? f.stB : (stage == 2 ? f.stA : f.m0));
  a.maxdmdt = stage == 0 ? f.maxdmdt : nullptr;
  constexpr int P = HALF == 0 ? 1 : 2 * HALF;
  body_x<HALF>(a, f.ph, f.S, f.tw + P, f.d, TY, 1, ft.y / ntyl, (ft.y % ntyl) * TY);
}

template <int HALF>
static cudaError_t run_bx(const BatchFilm* F, const int2* map, int nblocks, int kind, int stage, float dt,
                          cudaStream_t s) {
  const int T = HALF == 0 ? 1 : TeamOf<(HALF > 0 ? HALF : 1)>::v;
  if (kind == 0) {
    const int TY = HALF == 0 ? 32 : xtile(HALF);
    int threads = HALF == 0 ? 32 : TY * T;
    threads = threads < 32 ? 32 : (threads > 512 ? 512 : threads);
    const size_t smem = HALF == 0 ? 0 : sizeof(float2) * ((size_t)2 * HALF + (size_t)TY * (HALF + 1));
    static bool attr = false;
    if (cudaError_t e = allow_max_smem(kb_xfwd<HALF>, attr)) return e;
    kb_xfwd<HALF><<<nblocks, threads, smem, s>>>(F, map, TY);
  } else {
    const int TY = HALF == 0 ? 32 : x_tile(HALF);
    int threads = HALF == 0 ? 32 : ((3 * TY + 1) / 2) * T;
    threads = (threads + 31) / 32 * 32;
    threads = threads < 128 ? 128 : (threads > 512 ? 512 : threads);
    static bool attr = false;
    if (cudaError_t e = allow_max_smem(kb_x<HALF>, attr)) return e;
    kb_x<HALF><<<nblocks, threads, x_smem(HALF), s>>>(F, map, TY, stage, dt);
  }
  return cudaGetLastError();
}

template <int PY, int NZM>
static cudaError_t run_byz_t(const BatchFilm* F, const int2* map, int nblocks, size_t smem, int* flag,
                             cudaStream_t s) {
  if constexpr (!yz_col_fits(PY, NZM)) {
    return cudaErrorInvalidValue;
  } else {
    static bool attr = false;
    if (cudaError_t e = allow_max_smem(kb_yz<PY, NZM>, attr)) return e;
    kb_yz<PY, NZM><<<nblocks, 512, smem, s>>>(F, map, flag);
    return cudaGetLastError();
  }
}

template <int PY>
static cudaError_t run_byz(const BatchFilm* F, const int2* map, int nblocks, size_t smem, int nzm, int* flag,
                           cudaStream_t s) {
#define MM_CALL_BYZ(Z) run_byz_t<PY, Z>(F, map, nblocks, smem, flag, s)
  MM_NZ_SWITCH(nzm, MM_CALL_BYZ)
#undef MM_CALL_BYZ
}

// ---------------------------------------------------------------------------
// Per-size entry points.  Declared here for the dispatch in field.cu; defined
// and explicitly instantiated only in the field_inst_*.cu units (which define
// FIELD_INSTANTIATE), one unit per class of padded sizes, so that every kernel
// instance is compiled in exactly one translation unit.
// ---------------------------------------------------------------------------
template <int HALF>
cudaError_t fk_xfwd(const Dims& d, const float* m, const float2* tw, float2* S, cudaStream_t s);
template <int HALF>
cudaError_t fk_x(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S, cudaStream_t s,
                 int fwd);
template <int PY>
cudaError_t fk_yz(const Dims& d, const float2* tw, float2* S, const float* Kh, int* flag, const Tick& tk,
                  cudaStream_t s);
template <int PY>
cudaError_t fk_yt(const Dims& d, const float2* tw, float2* S, int dir, const Tick& tk, cudaStream_t s);
template <int NZM>
cudaError_t fk_zt(const Dims& d, const float* Kh, cudaStream_t s);
template <int HALF>
cudaError_t fk_bx(const BatchFilm* F, const int2* map, int nblocks, int kind, int stage, float dt, cudaStream_t s);
template <int PY>
cudaError_t fk_byz(const BatchFilm* F, const int2* map, int nblocks, size_t smem, int nzm, int* flag,
                   cudaStream_t s);

#ifdef FIELD_INSTANTIATE
template <int HALF>
cudaError_t fk_xfwd(const Dims& d, const float* m, const float2* tw, float2* S, cudaStream_t s) {
  return run_xfwd<HALF>(d, m, tw, S, s);
}
template <int HALF>
cudaError_t fk_x(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S, cudaStream_t s,
                 int fwd) {
  return run_x<HALF>(d, ph, a, tw, S, s, fwd);
}
template <int PY>
cudaError_t fk_yz(const Dims& d, const float2* tw, float2* S, const float* Kh, int* flag, const Tick& tk,
                  cudaStream_t s) {
  return run_yz_nz<PY>(d, tw, S, Kh, flag, tk, s);
}
template <int PY>
cudaError_t fk_yt(const Dims& d, const float2* tw, float2* S, int dir, const Tick& tk, cudaStream_t s) {
  return run_yt<PY>(d, tw, S, dir, tk, s);
}
template <int NZM>
cudaError_t fk_zt(const Dims& d, const float* Kh, cudaStream_t s) {
  return run_zt<NZM>(d, Kh, s);
}
template <int HALF>
cudaError_t fk_bx(const BatchFilm* F, const int2* map, int nblocks, int kind, int stage, float dt, cudaStream_t s) {
  return run_bx<HALF>(F, map, nblocks, kind, stage, dt, s);
}
template <int PY>
cudaError_t fk_byz(const BatchFilm* F, const int2* map, int nblocks, size_t smem, int nzm, int* flag,
                   cudaStream_t s) {
  return run_byz<PY>(F, map, nblocks, smem, nzm, flag, s);
}
// the x-pass entry points of one padded x size (HALF = px / 2, 0 for px = 1)
#define FK_INSTANTIATE_X(H)                                                                                     \
  template cudaError_t fk_xfwd<H>(const Dims&, const float*, const float2*, float2*, cudaStream_t);             \
  template cudaError_t fk_x<H>(const Dims&, const Phys&, const StageArgs&, const float2*, float2*,              \
                               cudaStream_t, int);                                                              \
  template cudaError_t fk_bx<H>(const BatchFilm*, const int2*, int, int, int, float, cudaStream_t);
// the y/z-pass entry points of one padded y size
#define FK_INSTANTIATE_YZ(P)                                                                                    \
  template cudaError_t fk_yz<P>(const Dims&, const float2*, float2*, const float*, int*, const Tick&,           \
                                cudaStream_t);                                                                  \
  template cudaError_t fk_yt<P>(const Dims&, const float2*, float2*, int, const Tick&, cudaStream_t);           \
  template cudaError_t fk_byz<P>(const BatchFilm*, const int2*, int, size_t, int, int*, cudaStream_t);
#define FK_INSTANTIATE_ZT(Z) template cudaError_t fk_zt<Z>(const Dims&, const float*, cudaStream_t);
#endif
