// FP32 FFT building blocks for the demagnetising convolution (eq. 14).
//
// A "team" of T lanes (T a power of two, T <= 32, all in one warp) transforms
// one power-of-two row of length L held in shared memory, in place, with the
// Stockham auto-sort formulation: pass by pass every lane loads R values at
// stride L/R into registers, applies the twiddles of the pass, does a radix-R
// DFT in registers and stores the R results at their auto-sorted places.
// Radices 8, then 4 or 2 for the remainder.  Results are in natural order.
// DIR = -1 is the forward transform exp(-2 pi i nk/L), DIR = +1 the
// unnormalised inverse.  Twiddles come from a table tw[m] = exp(-2 pi i m/LT)
// of length LT = L * TWS (TWS a power-of-two stride), so one table serves a
// transform and its half-length sub-transforms.  With PADS > 0 element e of a
// row is stored at e + (e >> PADS) (one spare slot every 2^PADS elements),
// which spreads the radix-8 stores of the first passes over all banks.
#pragma once
#include <cuda_runtime.h>

#ifndef MM_BC_SMEM
#define MM_BC_SMEM(p, n) true   // bounds checks: see common.cuh
#endif

// Complex arithmetic on the packed FP32 pair instructions of sm_100+ (one
// instruction per complex add; two per complex product), rounding per
// component exactly as the scalar forms.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return __ffma2_rn(make_float2(a.x, a.x), b, __fmul2_rn(make_float2(a.y, a.y), make_float2(-b.y, b.x)));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by i
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }
// multiply by the quarter-turn of direction DIR: -i (forward) or +i (inverse)
template <int DIR>
__device__ __forceinline__ float2 cquarter(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int DIR>
__device__ __forceinline__ void dft2(float2* v) {
  float2 t = v[0];
  v[0] = cadd(t, v[1]);
  v[1] = csub(t, v[1]);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2* v) {
  float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  float2 b0 = cadd(v[1], v[3]), b1 = cquarter<DIR>(csub(v[1], v[3]));
  v[0] = cadd(a0, b0);
  v[2] = csub(a0, b0);
  v[1] = cadd(a1, b1);
  v[3] = csub(a1, b1);
}

template <int DIR>
__device__ __forceinline__ void dft8(float2* v) {
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4<DIR>(e);
  dft4<DIR>(o);
  const float r = 0.70710678118654752440f;
  // o[k] *= exp(DIR * 2 pi i k / 8)
  if (DIR < 0) {
    o[1] = make_float2((o[1].x + o[1].y) * r, (o[1].y - o[1].x) * r);
    o[3] = make_float2((o[3].y - o[3].x) * r, -(o[3].x + o[3].y) * r);
  } else {
    o[1] = make_float2((o[1].x - o[1].y) * r, (o[1].x + o[1].y) * r);
    o[3] = make_float2(-(o[3].x + o[3].y) * r, (o[3].x - o[3].y) * r);
  }
  o[2] = cquarter<DIR>(o[2]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = cadd(e[k], o[k]);
    v[k + 4] = csub(e[k], o[k]);
  }
}

template <int R, int DIR>
__device__ __forceinline__ void dftR(float2* v) {
  if (R == 2) dft2<DIR>(v);
  else if (R == 4) dft4<DIR>(v);
  else dft8<DIR>(v);
}

// Lane mask of the team that lane `lane` belongs to.
template <int T>
__device__ __forceinline__ unsigned team_mask(int lane) {
  if (T >= 32) return 0xffffffffu;
  unsigned m = (T == 32) ? 0xffffffffu : ((1u << T) - 1u);
  return m << (lane & ~(T - 1));
}

template <int PADS>
__device__ __forceinline__ int pidx(int e) {
  return PADS > 0 ? e + (e >> PADS) : e;
}

// One pass.  PADR / PADW: padding of the layout read / written (they differ
// only when a transform converts between a dense and a padded row).  Inputs at
// positions >= nin are taken as zero without being read, outputs at positions
// >= nout are not written (zero padding and truncation of eq. 14).
template <int L, int R, int NS, int T, int DIR, int TWS, int PADR, int PADW>
__device__ __forceinline__ void stockham_pass(float2* x, int t, unsigned mask, const float2* tw, int nin,
                                              int nout) {
  constexpr int NB = L / R;                 // butterflies in this pass
  constexpr int PER = (NB + T - 1) / T;     // butterflies per lane
  float2 v[PER][R];
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = t + b * T;
    if (NB % T == 0 || j < NB) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = j + r * NB;
        v[b][r] = (e < nin) ? x[pidx<PADR>(e)] : make_float2(0.f, 0.f);
      }
    }
  }
  __syncwarp(mask);
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = t + b * T;
    if (NB % T == 0 || j < NB) {
      const int k = j & (NS - 1);
      if (NS > 1) {
        // w^r for r = 1..R-1 from one table entry (powers by multiplication:
        // one shared-memory load per butterfly instead of R-1)
        float2 wp[8];
        wp[1] = tw[(k * (L / (NS * R))) * TWS];
        if (DIR > 0) wp[1].y = -wp[1].y;
        if (R > 2) { wp[2] = cmul(wp[1], wp[1]); wp[3] = cmul(wp[2], wp[1]); }
        if (R > 4) {
          wp[4] = cmul(wp[2], wp[2]);
          wp[5] = cmul(wp[4], wp[1]);
          wp[6] = cmul(wp[4], wp[2]);
          wp[7] = cmul(wp[4], wp[3]);
        }
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], wp[r]);
      }
      dftR<R, DIR>(v[b]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = base + r * NS;
        if (e < nout && MM_BC_SMEM(&x[pidx<PADW>(e)], sizeof(float2))) x[pidx<PADW>(e)] = v[b][r];
      }
    }
  }
  __syncwarp(mask);
}

// Passes from sub-length NS on.  PIN: padding of the input layout (first pass),
// PMID: between passes, POUT: of the output layout (last pass).
template <int L, int NS, int T, int DIR, int TWS, int PIN, int PMID, int POUT>
struct FftPasses {
  __device__ __forceinline__ static void run(float2* x, int t, unsigned mask, const float2* tw, int nin, int nout) {
    constexpr int REM = L / NS;
    constexpr int R = (REM % 8 == 0) ? 8 : ((REM % 4 == 0) ? 4 : 2);
    constexpr bool first = (NS == 1), last = (NS * R == L);
    stockham_pass<L, R, NS, T, DIR, TWS, first ? PIN : PMID, last ? POUT : PMID>(x, t, mask, tw,
                                                                                 first ? nin : L, last ? nout : L);
    FftPasses<L, NS * R, T, DIR, TWS, PIN, PMID, POUT>::run(x, t, mask, tw, L, nout);
  }
};
template <int L, int T, int DIR, int TWS, int PIN, int PMID, int POUT>
struct FftPasses<L, L, T, DIR, TWS, PIN, PMID, POUT> {
  __device__ __forceinline__ static void run(float2*, int, unsigned, const float2*, int, int) {}
};

// Transform one row of length L in place; t = lane index within the team.
template <int L, int T, int DIR, int TWS, int PADS = 0>
__device__ __forceinline__ void team_fft(float2* x, int t, unsigned mask, const float2* tw) {
  FftPasses<L, 1, T, DIR, TWS, PADS, PADS, PADS>::run(x, t, mask, tw, L, L);
}

// Same, with a dense (PIN) / padded (PMID) / dense (POUT) choice of layouts, only
// the first nin inputs read (the rest are zeros) and only the first nout outputs
// written.  A row of length 1 is copied from the input to the output layout.
template <int L, int T, int DIR, int TWS, int PIN, int PMID, int POUT>
__device__ __forceinline__ void team_fft_io(float2* x, int t, unsigned mask, const float2* tw, int nin, int nout) {
  FftPasses<L, 1, T, DIR, TWS, PIN, PMID, POUT>::run(x, t, mask, tw, nin, nout);
}

// Team size used for a row of length L.
template <int L>
struct TeamOf {
  static constexpr int v = (L / 8) >= 32 ? 32 : ((L / 8) >= 1 ? (L / 8) : 1);
};

// ---------------------------------------------------------------------------
// Register-resident transforms.  One lane holds N <= 32 values of a sequence in
// registers; reg_fft is an in-place radix-2 decimation-in-frequency transform
// whose twiddles are compile-time powers of W_32, leaving X[k] in v[brev(k)].
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int brev(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// cos(2 pi k / 32) and sin(2 pi k / 32) for an integer k (quarter-wave values)
__host__ __device__ constexpr float cos32(int k) {
  const float q[9] = {1.0f, 0.980785280403230449f, 0.923879532511286756f, 0.831469612302545237f,
                      0.707106781186547524f, 0.555570233019602225f, 0.382683432365089772f,
                      0.195090322016128268f, 0.0f};
  k &= 31;
  return k <= 8 ? q[k] : (k <= 16 ? -q[16 - k] : (k <= 24 ? -q[k - 16] : q[32 - k]));
}
__host__ __device__ constexpr float sin32(int k) { return cos32(k - 8); }

// x * exp(DIR 2 pi i k / 32); k is a compile-time constant after unrolling, so the
// quarter turns cost no multiplication
template <int DIR>
__device__ __forceinline__ float2 mul_w32(float2 x, int k) {
  k &= 31;
  if (k == 0) return x;
  if (k == 16) return make_float2(-x.x, -x.y);
  if (k == 8) return cquarter<DIR>(x);
  if (k == 24) return cquarter<-DIR>(x);
  return cmul(x, make_float2(cos32(k), DIR < 0 ? -sin32(k) : sin32(k)));
}

// ZH: the upper half of the input is zero (the first stage then only twiddles).
template <int N, int DIR, bool ZH = false>
__device__ __forceinline__ void reg_fft(float2 (&v)[N]) {
  static_assert(N >= 2 && N <= 32 && (N & (N - 1)) == 0, "register transform of 2..32 values");
#pragma unroll
  for (int len = N; len >= 2; len >>= 1) {
    const int h = len >> 1;
#pragma unroll
    for (int s = 0; s < N; s += len) {
#pragma unroll
      for (int j = 0; j < h; ++j) {
        const float2 a = v[s + j], b = v[s + j + h];
        if (ZH && len == N) {
          v[s + j + h] = mul_w32<DIR>(a, j * (32 / len));
        } else {
          v[s + j] = cadd(a, b);
          v[s + j + h] = mul_w32<DIR>(csub(a, b), j * (32 / len));
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Two-pass transform of a row of L = 16 R2 values in shared memory (R2 = 16 or
// 32), Cooley-Tukey with L = 16 x R2:
//   pass 1: lane l (0 <= l < R2) transforms x[l + R2 j], j < 16, in registers,
//           multiplies result k1 by W_L^(l k1) and stores it at k1 (R2 + 1) + l
//           (one spare slot per R2 values: the reads of pass 2 hit 16
//           different banks);
//   pass 2: lane k1 (0 <= k1 < 16) transforms the R2 values k1 (R2 + 1) + l
//           and stores X[k1 + 16 k2] at its natural position.
// Two shared-memory round trips instead of log8(L); every access is free of
// bank conflicts.  In place: the lanes of a row read everything before any of
// them writes (__syncwarp).  Inputs at positions >= nin are zeros (not read),
// outputs at positions >= nout are not written; ZH: nin <= L / 2 (the upper
// half of every pass-1 sequence is zero).
// ---------------------------------------------------------------------------
template <int R2, int DIR, bool ZH, int NR = 1>
__device__ __forceinline__ void fft2_pass1(float2* const (&row)[NR], const bool (&act)[NR], int l, int nin,
                                           const float2 (&tw)[16]) {
  float2 v[NR][16];   // NR rows at once (independent chains)
#pragma unroll
  for (int r = 0; r < NR; ++r) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = l + R2 * j;
      v[r][j] = make_float2(0.f, 0.f);
      if (!(ZH && j >= 8) && act[r] && n < nin) v[r][j] = row[r][n];
    }
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < NR; ++r) reg_fft<16, DIR, ZH>(v[r]);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (act[r]) {
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) {
        const float2 x = v[r][brev(k1, 4)];
        if (MM_BC_SMEM(&row[r][k1 * (R2 + 1) + l], sizeof(float2))) row[r][k1 * (R2 + 1) + l] = k1 ? cmul(x, tw[k1]) : x;
      }
    }
  }
}

template <int R2, int DIR>
__device__ __forceinline__ void fft2_pass2(float2* row, bool act, int k1, int nout) {
  float2 v[R2];
#pragma unroll
  for (int l = 0; l < R2; ++l) v[l] = act ? row[k1 * (R2 + 1) + l] : make_float2(0.f, 0.f);
  __syncwarp();
  reg_fft<R2, DIR>(v);
  if (act) {
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int n = k1 + 16 * k2;
      if (n < nout && MM_BC_SMEM(&row[n], sizeof(float2))) row[n] = v[brev(k2, ilog2c(R2))];
    }
  }
}

// Pass-1 twiddles of lane l: tw[k] = W_L^(l k) (forward table twL[m] =
// exp(-2 pi i m / L)), conjugated for the inverse.
template <int L, int DIR>
__device__ __forceinline__ void fft2_twiddles(float2 (&tw)[16], int l, const float2* __restrict__ twL) {
  tw[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int k = 1; k < 16; ++k) {
    const float2 w = __ldg(twL + ((l * k) & (L - 1)));
    tw[k] = DIR < 0 ? w : cconj(w);
  }
}
