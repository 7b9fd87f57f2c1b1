// Effective field and LLG stage kernels (FP32): launch dispatch.  The device
// code and the template launchers live in field_kernels.cuh; each padded size
// class is instantiated in its own field_inst_*.cu unit (fk_* entry points).
#include <stdio.h>
#include <string.h>

#include <type_traits>
#include <utility>

#include "field_kernels.cuh"

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

// k_normalise_from: dst <- src / |src|, four cells per thread; src may be page-
// locked host memory that the kernel reads over the bus (the SMs' many
// outstanding loads, instead of one copy engine).  A zero or non-finite vector
// is flagged and passed through unchanged, as k_normalise leaves it.
__global__ void k_normalise_from(const float4* __restrict__ src, float4* __restrict__ dst, long long N4, int* flag) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N4) return;
  const float4 x = src[i], y = src[i + N4], z = src[i + 2 * N4];
  float4 o[3];
  const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w}, zs[4] = {z.x, z.y, z.z, z.w};
  float r[3][4];
  bool bad = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float n2 = xs[j] * xs[j] + ys[j] * ys[j] + zs[j] * zs[j];
    if (!(n2 > 0.f) || !isfinite(n2)) {
      bad = true;
      r[0][j] = xs[j]; r[1][j] = ys[j]; r[2][j] = zs[j];
      continue;
    }
    const float inv = rsqrtf(n2);
    r[0][j] = xs[j] * inv; r[1][j] = ys[j] * inv; r[2][j] = zs[j] * inv;
  }
  if (bad) atomicOr(flag, 1);
#pragma unroll
  for (int c = 0; c < 3; ++c) o[c] = make_float4(r[c][0], r[c][1], r[c][2], r[c][3]);
  dst[i] = o[0];
  dst[i + N4] = o[1];
  dst[i + 2 * N4] = o[2];
}

// ---------------------------------------------------------------------------
// launch geometry
// ---------------------------------------------------------------------------
int mm_nzm(int nz) { return nzm_of(nz); }

// ky block of one k_zt CTA: what its shared memory holds, at most 128
int mm_zt_kb_max(const Dims& d) {
  int kb = (int)(kZtBudget / (sizeof(float2) * 3ull * d.nz + sizeof(float) * 6ull * (d.nz + 4))) - 1;
  return kb > 128 ? 128 : kb;
}
int mm_zt_kb(const Dims& d) { return zt_kb(d); }

// The fused kernel needs the column in one CTA; thick samples with fewer kx
// columns than SMs also take the split pass, which spreads the z product (the
// bulk of their work, O(nz^2) per column) over ky blocks.
int mm_yz_fits(const Dims& d) { return nzm_of(d.nz) <= 64 && yz_smem(d) + 64 <= kMaxSmem; }

int mm_yz_fused(const Dims& d) {
  if (!mm_yz_fits(d)) return 0;
  if (d.route == 1) return 1;   // tuned
  if (d.route == 2) return d.prec ? 1 : 0;
  if (nzm_of(d.nz) >= 32 && d.hx < 148) return 0;
  return 1;
}
int mm_yz_launches(const Dims& d) { return mm_yz_fused(d) ? 1 : 3; }

int mm_supported(const Dims& d, char* why, int nwhy) {
  if (d.px > 2048 || d.py > 2048) {
    snprintf(why, nwhy, "padded size %dx%d exceeds 2048 (nx, ny <= 1024 supported)", d.px, d.py);
    return 0;
  }
  if (d.nz > 128) {
    snprintf(why, nwhy, "nz = %d > 128 is not supported by the z Toeplitz product of this build", d.nz);
    return 0;
  }
  if (d.prec) {
    if (d.nz < 5 || d.nz > 16 || d.py < 128) {
      snprintf(why, nwhy, "split precision needs 5 <= nz <= 16 and ny >= 33 (grid %d x %d x %d)", d.nx, d.ny, d.nz);
      return 0;
    }
  }
  if (!mm_yz_fused(d)) {
    // the split y/z pass: a ky block of the z product and a row group of the y transforms
    if (d.prec) {
      snprintf(why, nwhy, "split precision needs a kx column in one CTA (3 x %d x %d complex too large)", d.nz, d.py);
      return 0;
    }
    if (zt_kb(d) < 8) {
      snprintf(why, nwhy, "nz = %d: a block of 8 ky of the z product exceeds shared memory", d.nz);
      return 0;
    }
  }
  return 1;
}

#define MM_HALF_SWITCH(px, CALL)              \
  switch ((px) == 1 ? 0 : (px) / 2) {         \
    case 0: return CALL(0);                   \
    case 2: return CALL(2);                   \
    case 4: return CALL(4);                   \
    case 8: return CALL(8);                   \
    case 16: return CALL(16);                 \
    case 32: return CALL(32);                 \
    case 64: return CALL(64);                 \
    case 128: return CALL(128);               \
    case 256: return CALL(256);               \
    case 512: return CALL(512);               \
    case 1024: return CALL(1024);             \
  }                                           \
  return cudaErrorInvalidValue;

static cudaError_t dispatch_xfwd(const Dims& d, const float* m, const float2* tw, float2* S, cudaStream_t s) {
#define MM_CALL_XFWD(H) fk_xfwd<H>(d, m, tw, S, s)
  MM_HALF_SWITCH(d.px, MM_CALL_XFWD)
#undef MM_CALL_XFWD
}

static cudaError_t dispatch_x(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                              cudaStream_t s, int fwd) {
#define MM_CALL_X(H) fk_x<H>(d, ph, a, tw, S, s, fwd)
  MM_HALF_SWITCH(d.px, MM_CALL_X)
#undef MM_CALL_X
}

static cudaError_t dispatch_yt(const Dims& d, const float2* tw, float2* S, int dir, const Tick& tk, cudaStream_t s) {
  switch (d.py) {
    case 1: return fk_yt<1>(d, tw, S, dir, tk, s);
    case 4: return fk_yt<4>(d, tw, S, dir, tk, s);
    case 8: return fk_yt<8>(d, tw, S, dir, tk, s);
    case 16: return fk_yt<16>(d, tw, S, dir, tk, s);
    case 32: return fk_yt<32>(d, tw, S, dir, tk, s);
    case 64: return fk_yt<64>(d, tw, S, dir, tk, s);
    case 128: return fk_yt<128>(d, tw, S, dir, tk, s);
    case 256: return fk_yt<256>(d, tw, S, dir, tk, s);
    case 512: return fk_yt<512>(d, tw, S, dir, tk, s);
    case 1024: return fk_yt<1024>(d, tw, S, dir, tk, s);
    case 2048: return fk_yt<2048>(d, tw, S, dir, tk, s);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t dispatch_zt(const Dims& d, const float* Kh, cudaStream_t s) {
  switch (nzm_of(d.nz)) {
    case 1: return fk_zt<1>(d, Kh, s);
    case 2: return fk_zt<2>(d, Kh, s);
    case 4: return fk_zt<4>(d, Kh, s);
    case 8: return fk_zt<8>(d, Kh, s);
    case 16: return fk_zt<16>(d, Kh, s);
    case 32: return fk_zt<32>(d, Kh, s);
    case 64: return fk_zt<64>(d, Kh, s);
    case 128: return fk_zt<128>(d, Kh, s);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t dispatch_yz(const Dims& d, const float2* tw, float2* S, const float* Kh, int* flag, const Tick& tk,
                               cudaStream_t s) {
  if (!mm_yz_fused(d)) {
    if (!d.T) return cudaErrorInvalidValue;
    if (cudaError_t e = dispatch_yt(d, tw, S, -1, tk, s)) return e;
    if (cudaError_t e = dispatch_zt(d, Kh, s)) return e;
    return dispatch_yt(d, tw, S, 1, Tick{}, s);
  }
  switch (d.py) {
    case 1: return fk_yz<1>(d, tw, S, Kh, flag, tk, s);
    case 4: return fk_yz<4>(d, tw, S, Kh, flag, tk, s);
    case 8: return fk_yz<8>(d, tw, S, Kh, flag, tk, s);
    case 16: return fk_yz<16>(d, tw, S, Kh, flag, tk, s);
    case 32: return fk_yz<32>(d, tw, S, Kh, flag, tk, s);
    case 64: return fk_yz<64>(d, tw, S, Kh, flag, tk, s);
    case 128: return fk_yz<128>(d, tw, S, Kh, flag, tk, s);
    case 256: return fk_yz<256>(d, tw, S, Kh, flag, tk, s);
    case 512: return fk_yz<512>(d, tw, S, Kh, flag, tk, s);
    case 1024: return fk_yz<1024>(d, tw, S, Kh, flag, tk, s);
    case 2048: return fk_yz<2048>(d, tw, S, Kh, flag, tk, s);
  }
  return cudaErrorInvalidValue;
}

// Field evaluation from scratch (mode 0): x forward of a.m_in, y/z, x inverse.
int launch_field_eval(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                      const float* Kh, int* flag, cudaStream_t s) {
  StageArgs ax = a;
  ax.flag = flag;
  if (dispatch_xfwd(d, a.m_in, tw, S, s) != cudaSuccess) return -1;
  if (dispatch_yz(d, tw, S, Kh, flag, Tick{}, s) != cudaSuccess) return -2;
  if (dispatch_x(d, ph, ax, tw, S, s, a.mode != 0) != cudaSuccess) return -3;
  return 2 + mm_yz_launches(d);
}

// One stage when S already holds the x transform of a.m_in: y/z, then x inverse
// + update + x forward of the new state (S then holds the transform of a.m_out).
int launch_stage(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                 const float* Kh, int* flag, cudaStream_t s) {
  StageArgs ax = a;
  ax.flag = flag;
  if (dispatch_yz(d, tw, S, Kh, flag, a.tick, s) != cudaSuccess) return -2;
  if (dispatch_x(d, ph, ax, tw, S, s, 1) != cudaSuccess) return -3;
  return 1 + mm_yz_launches(d);
}

int launch_xfwd(const Dims& d, const float* m, const float2* tw, float2* S, cudaStream_t s) {
  return dispatch_xfwd(d, m, tw, S, s) == cudaSuccess ? 1 : -1;
}

int launch_field_part(const Dims& d, const Phys& ph, const StageArgs& a, const float2* tw, float2* S,
                      const float* Kh, int* flag, cudaStream_t s, int part) {
  cudaError_t e = cudaErrorInvalidValue;
  if (part == 0) e = dispatch_xfwd(d, a.m_in, tw, S, s);
  else if (part == 1) e = dispatch_yz(d, tw, S, Kh, flag, a.tick, s);
  else if (part == 2) {
    StageArgs ax = a;
    ax.flag = flag;
    // modes 1, 2 (a stage), 3 and 5 (adjoint stages) transform their output along x for the next pass
    e = dispatch_x(d, ph, ax, tw, S, s, a.mode != 0 && a.mode != 4);
  }
  if (e != cudaSuccess) return -1;
  return part == 1 ? mm_yz_launches(d) : 1;
}

int launch_normalise_from(const Dims& d, const float* src, float* dst, int* flag, cudaStream_t s) {
  const long long N4 = d.N / 4;
  k_normalise_from<<<(unsigned)((N4 + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float4*>(src),
                                                                 reinterpret_cast<float4*>(dst), N4, flag);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_normalise(const Dims& d, float* m, int* flag, cudaStream_t s) {
  k_normalise<<<(unsigned)((d.N + 255) / 256), 256, 0, s>>>(m, d.N, flag);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

// ---------------------------------------------------------------------------
// Batched launches (kernels kb_xfwd, kb_yz, kb_x in field_kernels.cuh): CTA i
// works on film map[i].x, tile map[i].y; the films of a launch share the padded
// sizes.
// ---------------------------------------------------------------------------
int x_batch_tile(int px, int kind) {
  const int half = px == 1 ? 0 : px / 2;
  if (kind == 0) return half == 0 ? 32 : xtile(half);
  return half == 0 ? 32 : x_tile(half);
}

int launch_batch(const BatchFilm* F, int px, int py, int nzm, const int2* map, int nblocks, size_t smem_yz,
                 int kind, int stage, float dt, int* flag, cudaStream_t s) {
  if (nblocks <= 0) return 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (kind == 1) {
    switch (py) {
      case 1: e = fk_byz<1>(F, map, nblocks, smem_yz, nzm, flag, s); break;
      case 4: e = fk_byz<4>(F, map, nblocks, smem_yz, nzm, flag, s); break;
      case 8: e = fk_byz<8>(F, map, nblocks, smem_yz, nzm, flag, s); break;
      case 16: e = fk_byz<16>(F, map, nblocks, smem_yz, nzm, flag, s); break;
      case 32: e = fk_byz<32>(F, map, nblocks, smem_yz, nzm, flag, s); break;
      case 64: e = fk_byz<64>(F, map, nblocks, smem_yz, nzm, flag, s); break;
      case 128: e = fk_byz<128>(F, map, nblocks, smem_yz, nzm, flag, s); break;
      case 256: e = fk_byz<256>(F, map, nblocks, smem_yz, nzm, flag, s); break;
      case 512: e = fk_byz<512>(F, map, nblocks, smem_yz, nzm, flag, s); break;
      case 1024: e = fk_byz<1024>(F, map, nblocks, smem_yz, nzm, flag, s); break;
      case 2048: e = fk_byz<2048>(F, map, nblocks, smem_yz, nzm, flag, s); break;
    }
  } else {
    const int k = kind;
    auto go = [&](auto half_tag) { return fk_bx<decltype(half_tag)::value>(F, map, nblocks, k, stage, dt, s); };
    switch (px == 1 ? 0 : px / 2) {
      case 0: e = go(std::integral_constant<int, 0>()); break;
      case 2: e = go(std::integral_constant<int, 2>()); break;
      case 4: e = go(std::integral_constant<int, 4>()); break;
      case 8: e = go(std::integral_constant<int, 8>()); break;
      case 16: e = go(std::integral_constant<int, 16>()); break;
      case 32: e = go(std::integral_constant<int, 32>()); break;
      case 64: e = go(std::integral_constant<int, 64>()); break;
      case 128: e = go(std::integral_constant<int, 128>()); break;
      case 256: e = go(std::integral_constant<int, 256>()); break;
      case 512: e = go(std::integral_constant<int, 512>()); break;
      case 1024: e = go(std::integral_constant<int, 1024>()); break;
    }
  }
  return e == cudaSuccess ? 1 : -1;
}

size_t mm_yz_smem(const Dims& d) { return yz_smem(d); }
