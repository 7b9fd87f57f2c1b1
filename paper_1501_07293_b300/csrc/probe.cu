// Peak-rate probe of the FP32 pipes (measurement only; the paper has no
// counterpart).  The roofline of the y/z kernel is reported against the FP32
// rate this kernel reaches on the device at hand, rather than against a figure
// derived from unit counts and a nominal clock.
//
// Every thread runs NCHAIN independent fused multiply-add chains for `iters`
// iterations with its operands in registers (no memory traffic inside the
// loop); the result is stored only if it equals a value it cannot reach, so
// the compiler keeps the work.  The packed form issues the FP32 pair FMA of
// sm_100+ (__ffma2_rn: two FMAs per instruction).
#include "common.cuh"

static constexpr int kProbeChains = 8;
static constexpr int kProbeThreads = 256;
static constexpr int kProbeBlocksPerSM = 4;

// where a result would go if it ever reached the unreachable value (never written)
static __device__ float g_probe_sink[kProbeThreads];

template <bool PACKED>
__global__ void __launch_bounds__(kProbeThreads) k_fp32_probe(float a, float b, int iters) {
  if constexpr (PACKED) {
    float2 acc[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc[c] = make_float2(threadIdx.x * 1e-7f + c, c * 1e-3f);
    const float2 av = make_float2(a, a), bv = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) acc[c] = __ffma2_rn(acc[c], av, bv);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += acc[c].x + acc[c].y;
    if (s == -1.2345e30f) g_probe_sink[threadIdx.x] = s;
  } else {
    float acc[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc[c] = threadIdx.x * 1e-7f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) acc[c] = fmaf(acc[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += acc[c];
    if (s == -1.2345e30f) g_probe_sink[threadIdx.x] = s;
  }
}

extern "C" int mm_fp32_probe(int packed, int iters, void* stream, double* flops) {
  if (!flops || iters < 1 || iters > (1 << 24)) return MM_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return MM_ECUDA;
  }
  const int blocks = sms * kProbeBlocksPerSM;
  cudaStream_t s = (cudaStream_t)stream;
  // a = 1 - 2^-20, b = 2^-30: the chains decay slowly and stay finite and normal
  const float a = 1.0f - 9.5367431640625e-07f, b = 9.313225746154785e-10f;
  if (packed) k_fp32_probe<true><<<blocks, kProbeThreads, 0, s>>>(a, b, iters);
  else k_fp32_probe<false><<<blocks, kProbeThreads, 0, s>>>(a, b, iters);
  if (cudaGetLastError() != cudaSuccess) return MM_ECUDA;
  *flops = 2.0 * (packed ? 2.0 : 1.0) * kProbeChains * (double)iters * kProbeThreads * (double)blocks;
  return MM_OK;
}
