// Split-precision product of eq. 14 along z on the tensor cores (tcgen05).
//
// For one kx column whose y transform sits in shared memory (rows b*nz + z,
// position ky), the Toeplitz sum along z is taken through a length-PZ = 2 NZ
// DFT (circular embedding, PZ >= 2 nz - 1):
//   M^_b(kz)  = sum_z m_b(z) e^{-2 pi i kz z / PZ}             (GEMM 1)
//   H^_a(kz)  = sum_b s_ab Kt_ab(kz) M^_b(kz)                    (FP32, per cell)
//   H_a(z)    = sum_kz H^_a(kz) e^{+2 pi i kz z / PZ}            (GEMM 2)
// Kt is the tensor (already transformed along x and y) transformed along z, real
// for every pair, with the 1/PZ of the inverse folded in (setup.cu); s_ab is
// the y-parity sign at mirrored ky.
//
// GEMM operands are split into a high and a low part of the 16-bit type
// (x = hi + lo), and each product is hi*hi + hi*lo + lo*hi with FP32
// accumulation in tensor memory.  A operands (the data) are written to tensor
// memory by the threads (one row per lane); B operands (the DFT matrices) sit in
// shared memory in the canonical no-swizzle K-major layout: core matrices of 8
// rows x 16 bytes, element (n, k) of an N x K matrix at
//   ((k/8) * (N/8) + n/8) * 128 + (n%8) * 16 + (k%8) * 2,
// so a K step of 16 starts 2 (N/8) 128 bytes further, LBO = (N/8) 128 (between
// the two core matrices along K) and SBO = 128 (between 8-row groups).
//
// The ky positions are processed in chunks of 128 (one MMA M tile per lane
// block of tensor memory).  Per chunk: one thread issues GEMM 1 on the A1 rows
// written before, all wait on an mbarrier (bounded; the product's tensor loads
// go out first), threads form H^ and write A2, one thread issues GEMM 2, the
// threads write the next chunk's A1 while it runs, then read H back into
// shared memory.  Tensor memory columns (512 allocated per CTA):
//   [0, 6 PZ)             D1: 3 b x 2 PZ  (re kz | im kz)
//                         D2: 3 a x 2 NZ (re z | im z), in D1's first columns
//                         (D1 has been read into registers when GEMM 2 starts)
//   [6 PZ, 6 PZ + 6 NZ)   A1: 3 b x {hi, lo} x NZ columns (K = 2 NZ: re z | im z)
//   [6 PZ + 6 NZ, ...)    A2: 3 a x {hi, lo} x PZ columns (K = 2 PZ: re kz | im kz)
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "bulk.cuh"

namespace zs {

// --- tcgen05 wrappers (one CTA, cta_group::1) --------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// D (+)= A(tmem) * B(smem descriptor)
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}

// 32 lanes x N 32-bit columns (this thread's lane), N = 2, 4, 8, 16
template <int N> struct TmemIO;
template <> struct TmemIO<2> {
  __device__ static void ld(uint32_t t, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(t));
  }
  __device__ static void st(uint32_t t, const uint32_t* r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(t), "r"(r[0]), "r"(r[1]));
  }
};
template <> struct TmemIO<4> {
  __device__ static void ld(uint32_t t, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(t));
  }
  __device__ static void st(uint32_t t, const uint32_t* r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(t), "r"(r[0]), "r"(r[1]),
                 "r"(r[2]), "r"(r[3]));
  }
};
template <> struct TmemIO<8> {
  __device__ static void ld(uint32_t t, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(t));
  }
  __device__ static void st(uint32_t t, const uint32_t* r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(t), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]));
  }
};
template <> struct TmemIO<16> {
  __device__ static void ld(uint32_t t, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(t));
  }
  __device__ static void st(uint32_t t, const uint32_t* r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(t),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
  }
};

// --- the 16-bit split x = hi + lo -------------------------------------------
// PREC 1: bfloat16; PREC 2: float16 with the data scaled by 2^-12 (the y
// transforms of unit vectors reach nx ny, beyond the float16 range).
template <int PREC> struct Split;
template <> struct Split<1> {
  static constexpr float scale = 1.f, unscale = 1.f;
  __device__ static void split(float x, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
  }
  static constexpr uint32_t fmt = 1;   // instruction-descriptor A/B format
};
template <> struct Split<2> {
  static constexpr float scale = 1.f / 4096.f, unscale = 4096.f;
  __device__ static void split(float x, uint16_t& hi, uint16_t& lo) {
    const __half h = __float2half_rn(x);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
  }
  static constexpr uint32_t fmt = 0;
};

// instruction descriptor: D F32, A/B format, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// shared-memory descriptor of a canonical no-swizzle K-major operand with N rows
// (version 1 for this architecture in bits 46-47)
__device__ __forceinline__ uint64_t bdesc(uint32_t saddr, int N) {
  const uint32_t lbo = (uint32_t)(N / 8) * 128u, sbo = 128u;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__host__ __device__ constexpr int canon_off(int n, int k, int N) {
  return ((k / 8) * (N / 8) + n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
}

// Byte sizes of the two DFT operands (hi and lo each): B1 = 2 PZ x 2 NZ, B2 = 2 NZ x 2 PZ.
template <int NZ>
struct Dft {
  static constexpr int PZ = 2 * NZ;
  static constexpr int N1 = 2 * PZ, K1 = 2 * NZ;   // GEMM 1: N x K
  static constexpr int N2 = 2 * NZ, K2 = 2 * PZ;   // GEMM 2
  static constexpr int B1 = N1 * K1 * 2, B2 = N2 * K2 * 2;
  static constexpr int bytes = 2 * B1 + 2 * B2;   // B1 hi, B1 lo, B2 hi, B2 lo
  static constexpr int KW = PZ / 4;               // kz values per thread in the product
  static constexpr uint32_t D1 = 0, A1 = 6 * PZ, D2 = 0, A2 = 6 * PZ + 6 * NZ;
};

// Wait for phase `ph` of bar (bounded); false when it gave up.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t ph) { return mbar_wait_bounded(bar, ph); }

// The split z product of one kx column.  buf: rows b*nz + z of stride rs
// (position ky at pidx<PADS>(ky)), PY positions, PY % 128 == 0.  Kt: this
// column's [PZ/2 + 1][6][hy] transformed tensor.  Bsm: the DFT operands in
// shared memory.  tb: the CTA's tensor-memory base; bar/phase: the MMA
// completion barrier.  512 threads.  Returns false after a wait gave up (flag set).
template <int PY, int NZ, int PREC, int PADS>
__device__ __forceinline__ bool zprod_split(float2* buf, int rs, int nz, int py, int hy, const float* __restrict__ Kt,
                                            const unsigned char* Bsm, uint32_t tb, uint64_t* bar, uint32_t& phase,
                                            int* flag) {
  using G = Dft<NZ>;
  using S = Split<PREC>;
  constexpr int PZ = G::PZ, KW = G::KW;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, g = warp >> 2;               // lane block, warp group
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;  // this warp's tensor-memory lanes
  const uint32_t b1h = smem_u32(Bsm), b1l = b1h + G::B1, b2h = b1l + G::B1, b2l = b2h + G::B2;
  constexpr uint32_t id1 = idesc_f16(S::fmt, 128, G::N1), id2 = idesc_f16(S::fmt, 128, G::N2);
  // 1. A1 rows of the chunk at ky0: (b = g, ky) -> K = 2 NZ reals (re z | im z),
  //    split, packed 2 per column
  auto fill_a1 = [&](int ky0) {
    if (g < 3) {
      const int pos = pidx<PADS>(ky0 + 32 * q + lane);
      uint32_t hi[NZ], lo[NZ];
#pragma unroll
      for (int c = 0; c < NZ; ++c) {
        float v[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int k = 2 * c + e;
          const int z = k < NZ ? k : k - NZ;
          float x = 0.f;
          if (z < nz) {
            const float2 m = buf[(g * nz + z) * rs + pos];
            x = (k < NZ ? m.x : m.y) * S::scale;
          }
          v[e] = x;
        }
        uint16_t h0, l0, h1, l1;
        S::split(v[0], h0, l0);
        S::split(v[1], h1, l1);
        hi[c] = (uint32_t)h0 | ((uint32_t)h1 << 16);
        lo[c] = (uint32_t)l0 | ((uint32_t)l1 << 16);
      }
      const uint32_t ta = tb + lane_off + G::A1 + (uint32_t)(g * 2) * NZ;
      TmemIO<NZ>::st(ta, hi);
      TmemIO<NZ>::st(ta + NZ, lo);
      wait_st();
    }
  };
  fill_a1(0);
  fence_before();
  __syncthreads();
  for (int ky0 = 0; ky0 < PY; ky0 += 128) {
    const int ky = ky0 + 32 * q + lane;
    const int pos = pidx<PADS>(ky);
    // 2. GEMM 1: D1_b = A1_b * B1 (3 split terms per K step)
    if (tid == 0) {
      fence_after();
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const uint32_t d = tb + G::D1 + (uint32_t)b * G::N1;
        const uint32_t ah = tb + G::A1 + (uint32_t)(b * 2) * NZ, al = ah + NZ;
#pragma unroll
        for (int ks = 0; ks < G::K1 / 16; ++ks) {
          const uint32_t koff = (uint32_t)ks * 2u * (G::N1 / 8) * 128u;
          mma_ts(d, ah + 8 * ks, bdesc(b1h + koff, G::N1), id1, ks > 0);
          mma_ts(d, ah + 8 * ks, bdesc(b1l + koff, G::N1), id1, 1);
          mma_ts(d, al + 8 * ks, bdesc(b1h + koff, G::N1), id1, 1);
        }
      }
      mma_commit(bar);
    }
    // the tensor values of this thread's ky and kz range (step 3) do not depend on
    // GEMM 1: their loads go out before its completion wait and land under it; Kt is
    // [kz][pair][ky] per column, so a warp's loads are contiguous
    const int kz0 = KW * g;
    const bool mir = ky > py / 2;
    const int kyf = mir ? py - ky : ky;
    float2 kv[KW][3];
#pragma unroll
    for (int j = 0; j < KW; ++j) {
      const int kz = kz0 + j;
      const int kzf = kz > PZ / 2 ? PZ - kz : kz;
      const float* kp = Kt + (long long)kzf * 6 * hy + kyf;
#pragma unroll
      for (int u = 0; u < 3; ++u) kv[j][u] = make_float2(__ldg(kp + (2 * u) * hy), __ldg(kp + (2 * u + 1) * hy));
    }
    if (!wait_phase(bar, phase)) {
      if (tid == 0) atomicOr(flag + 1, 1);
      return false;
    }
    phase ^= 1;
    fence_after();
    // 3. H^_a(kz) for this thread's ky and kz in [KW g, KW g + KW)
    {
      float re[3][KW], im[3][KW];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        uint32_t r[KW], i[KW];
        const uint32_t t = tb + lane_off + G::D1 + (uint32_t)b * G::N1;
        TmemIO<KW>::ld(t + kz0, r);
        TmemIO<KW>::ld(t + PZ + kz0, i);
        wait_ld();
#pragma unroll
        for (int j = 0; j < KW; ++j) { re[b][j] = __uint_as_float(r[j]); im[b][j] = __uint_as_float(i[j]); }
      }
      uint32_t hr[3][KW / 2], lr[3][KW / 2], hm[3][KW / 2], lm[3][KW / 2];
#pragma unroll
      for (int j = 0; j < KW; ++j) {
        const int kz = kz0 + j;
        const bool up = kz > PZ / 2;   // Kt(kz) = +-Kt(PZ - kz): cosine pairs even, sine pairs odd
        const float2 k01 = kv[j][0], k23 = kv[j][1], k45 = kv[j][2];   // xx yy | zz xy | xz yz
        const float ys = mir ? -1.f : 1.f;
        const float zsg = up ? -1.f : 1.f;
        const float kxx = k01.x, kyy = k01.y, kzz = k23.x, kxy = ys * k23.y;
        const float kxz = zsg * k45.x, kyz = ys * zsg * k45.y;
        float hre[3], him[3];
        hre[0] = kxx * re[0][j] + kxy * re[1][j] + kxz * re[2][j];
        him[0] = kxx * im[0][j] + kxy * im[1][j] + kxz * im[2][j];
        hre[1] = kxy * re[0][j] + kyy * re[1][j] + kyz * re[2][j];
        him[1] = kxy * im[0][j] + kyy * im[1][j] + kyz * im[2][j];
        hre[2] = kxz * re[0][j] + kyz * re[1][j] + kzz * re[2][j];
        him[2] = kxz * im[0][j] + kyz * im[1][j] + kzz * im[2][j];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          uint16_t h0, l0, h1, l1;
          S::split(hre[a], h0, l0);
          S::split(him[a], h1, l1);
          const int c = j >> 1, s = (j & 1) * 16;
          if ((j & 1) == 0) { hr[a][c] = 0; lr[a][c] = 0; hm[a][c] = 0; lm[a][c] = 0; }
          hr[a][c] |= (uint32_t)h0 << s; lr[a][c] |= (uint32_t)l0 << s;
          hm[a][c] |= (uint32_t)h1 << s; lm[a][c] |= (uint32_t)l1 << s;
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        // A2_a: K = 2 PZ (re kz | im kz), 2 per column: re at kz/2, im at (PZ + kz)/2
        const uint32_t th = tb + lane_off + G::A2 + (uint32_t)(a * 2) * PZ, tl = th + PZ;
        TmemIO<KW / 2>::st(th + kz0 / 2, hr[a]);
        TmemIO<KW / 2>::st(th + (PZ + kz0) / 2, hm[a]);
        TmemIO<KW / 2>::st(tl + kz0 / 2, lr[a]);
        TmemIO<KW / 2>::st(tl + (PZ + kz0) / 2, lm[a]);
      }
      wait_st();
    }
    fence_before();
    __syncthreads();
    // 4. GEMM 2: D2_a = A2_a * B2
    if (tid == 0) {
      fence_after();
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const uint32_t d = tb + G::D2 + (uint32_t)a * G::N2;
        const uint32_t ah = tb + G::A2 + (uint32_t)(a * 2) * PZ, al = ah + PZ;
#pragma unroll
        for (int ks = 0; ks < G::K2 / 16; ++ks) {
          const uint32_t koff = (uint32_t)ks * 2u * (G::N2 / 8) * 128u;
          mma_ts(d, ah + 8 * ks, bdesc(b2h + koff, G::N2), id2, ks > 0);
          mma_ts(d, ah + 8 * ks, bdesc(b2l + koff, G::N2), id2, 1);
          mma_ts(d, al + 8 * ks, bdesc(b2h + koff, G::N2), id2, 1);
        }
      }
      mma_commit(bar);
    }
    // the next chunk's A1 while GEMM 2 runs: GEMM 1 has completed (A1 is free) and
    // GEMM 2 reads A2 and writes D2 in D1's columns, neither of which A1 overlaps
    if (ky0 + 128 < PY) fill_a1(ky0 + 128);
    if (!wait_phase(bar, phase)) {
      if (tid == 0) atomicOr(flag + 1, 1);
      return false;
    }
    phase ^= 1;
    fence_after();
    // 5. H_a(z) back into the rows (a = g)
    if (g < 3) {
      uint32_t r[NZ], i[NZ];
      const uint32_t t = tb + lane_off + G::D2 + (uint32_t)g * G::N2;
      TmemIO<NZ>::ld(t, r);
      TmemIO<NZ>::ld(t + NZ, i);
      wait_ld();
#pragma unroll
      for (int z = 0; z < NZ; ++z)
        if (z < nz)
          buf[(g * nz + z) * rs + pos] =
              make_float2(__uint_as_float(r[z]) * S::unscale, __uint_as_float(i[z]) * S::unscale);
    }
    fence_before();
    __syncthreads();
  }
  return true;
}

}  // namespace zs
