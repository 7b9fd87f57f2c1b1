// Demagnetising kernel setup (once per geometry), FP64 on the device.
//
// 1. k_tensor: the tensor of eq. 10/11 for every offset |I| < nx, |J| < ny,
//    0 <= K < nz, placed on the padded px x py plane at the wrap position
//    (I mod px, J mod py), one plane per K.  Offsets are in units of delta
//    (the tensor is scale free).  log(z + r) is evaluated as
//    log((x^2 + y^2) / (r - z)) when z < 0, the same number without the
//    cancellation of z + r.
// 2. k_fft64: FP64 radix-2 Stockham transforms along x, then y, of every plane
//    (the convolution theorem of eq. 14 along x and y; z stays in real space).
// 3. k_extract: keeps kx in [0, px/2], ky in [0, py/2] (the rest follows from
//    the tensor's parity) and stores float32 Kh[kx][ky][pair][K].  Pairs xx, yy,
//    zz, xy transform to real numbers, xz and yz to imaginary ones (they are odd
//    in exactly one of x, y); the imaginary part is stored for those two.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

__device__ __forceinline__ double log_z_plus_r(double x, double y, double z) {
  const double rho2 = x * x + y * y;
  const double r = sqrt(rho2 + z * z);
  return z >= 0.0 ? log(z + r) : log(rho2 / (r - z));
}

__global__ void k_tensor(double2* __restrict__ Kc, Dims d, int self_term) {
  const long long plane = (long long)d.px * d.py;
  const long long total = plane * d.nz;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int x = (int)(idx % d.px);
  const int y = (int)((idx / d.px) % d.py);
  const int kz = (int)(idx / plane);
  int I = 0, J = 0;
  bool ok = true;
  if (x < d.nx) I = x;
  else if (x > d.px - d.nx) I = x - d.px;
  else ok = false;
  if (y < d.ny) J = y;
  else if (y > d.py - d.ny) J = y - d.py;
  else ok = false;
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (ok && (self_term || I != 0 || J != 0 || kz != 0)) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const double s = ((i + j + k) & 1) ? -1.0 : 1.0;
          const double X = I + i - 0.5, Y = J + j - 0.5, Z = kz + k - 0.5;
          const double r = sqrt(X * X + Y * Y + Z * Z);
          v[0] += s * atan(Y * Z / (X * r));
          v[1] += s * atan(X * Z / (Y * r));
          v[2] += s * atan(Y * X / (Z * r));
          v[3] += s * log_z_plus_r(X, Y, Z);  // log(z + r)
          v[4] += s * log_z_plus_r(X, Z, Y);  // log(y + r)
          v[5] += s * log_z_plus_r(Y, Z, X);  // log(x + r)
        }
    const double pref = 1.0 / (4.0 * MM_PI);
    v[0] *= pref; v[1] *= pref; v[2] *= pref;
    v[3] *= -pref; v[4] *= -pref; v[5] *= -pref;
  }
  for (int p = 0; p < 6; ++p)
    Kc[((long long)p * d.nz + kz) * plane + (long long)y * d.px + x] = make_double2(v[p], 0.0);
}

// One CTA per line of length L (power of two), radix-2 Stockham, ping-pong in shared memory.
// Line l starts at (l / inner) * outer + (l % inner) * inner_step; elements are estride apart.
__global__ void k_fft64(double2* __restrict__ data, int L, long long inner, long long inner_step,
                        long long outer, long long estride) {
  extern __shared__ double2 sh64[];
  double2* a = sh64;
  double2* b = sh64 + L;
  const long long l = blockIdx.x;
  const long long base = (l / inner) * outer + (l % inner) * inner_step;
  for (int i = threadIdx.x; i < L; i += blockDim.x) a[i] = data[base + i * estride];
  __syncthreads();
  const int half = L / 2;
  for (int ns = 1; ns < L; ns *= 2) {
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
      const int k = j & (ns - 1);
      double2 u = a[j], v = a[j + half];
      double sn, cs;
      sincospi(-(double)k / (double)ns, &sn, &cs);   // exp(-2 pi i k / (2 ns))
      const double2 w = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
      const int o = (j - k) * 2 + k;
      b[o] = make_double2(u.x + w.x, u.y + w.y);
      b[o + ns] = make_double2(u.x - w.x, u.y - w.y);
    }
    __syncthreads();
    double2* t = a; a = b; b = t;
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) data[base + i * estride] = a[i];
}

__global__ void k_extract(const double2* __restrict__ Kc, float* __restrict__ Kh, Dims d) {
  const long long total = (long long)d.hx * 6 * d.nz * d.hy;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  // Kh[kx][ky][pair][K]: the nz values one (kx, ky, pair) needs are contiguous
  const int kz = (int)(idx % d.nz);
  long long r = idx / d.nz;
  const int p = (int)(r % 6);
  r /= 6;
  const int ky = (int)(r % d.hy);
  const int kx = (int)(r / d.hy);
  const long long plane = (long long)d.px * d.py;
  const double2 v = Kc[((long long)p * d.nz + kz) * plane + (long long)ky * d.px + kx];
  Kh[idx] = (float)(p < 4 ? v.x : v.y);
}

int mm_build_kernel(mm_ctx* c) {
  const Dims& d = c->d;
  const long long plane = (long long)d.px * d.py;
  const size_t kc_bytes = sizeof(double2) * 6 * (size_t)d.nz * plane;
  double2* Kc = nullptr;
  if (cudaMalloc(&Kc, kc_bytes) != cudaSuccess) {
    cudaGetLastError();
    return mm_fail(c, MM_ENOMEM, "tensor setup: cannot allocate %zu bytes", kc_bytes);
  }
  int rc = MM_OK;
  do {
    const long long total = plane * d.nz;
    k_tensor<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(Kc, d, c->opts.self_term);
    if (cudaGetLastError() != cudaSuccess) { rc = mm_fail(c, MM_ECUDA, "k_tensor launch failed"); break; }
    c->launches++;
    // x lines: 6*nz*py lines of px contiguous elements
    if (d.px > 1) {
      const size_t sm = 2 * sizeof(double2) * d.px;
      if (sm > 48 * 1024) cudaFuncSetAttribute(k_fft64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      const long long lines = 6LL * d.nz * d.py;
      k_fft64<<<(unsigned)lines, d.px / 2 < 256 ? d.px / 2 : 256, sm, c->stream>>>(Kc, d.px, 1, 0, d.px, 1);
      if (cudaGetLastError() != cudaSuccess) { rc = mm_fail(c, MM_ECUDA, "k_fft64(x) launch failed"); break; }
      c->launches++;
    }
    // y lines: for every plane and x, py elements px apart
    if (d.py > 1) {
      const size_t sm = 2 * sizeof(double2) * d.py;
      if (sm > 48 * 1024) cudaFuncSetAttribute(k_fft64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      const long long lines = 6LL * d.nz * d.px;
      k_fft64<<<(unsigned)lines, d.py / 2 < 256 ? d.py / 2 : 256, sm, c->stream>>>(Kc, d.py, d.px, 1, plane, d.px);
      if (cudaGetLastError() != cudaSuccess) { rc = mm_fail(c, MM_ECUDA, "k_fft64(y) launch failed"); break; }
      c->launches++;
    }
    const long long tot = (long long)d.hx * 6 * d.nz * d.hy;
    k_extract<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(Kc, c->Kh, d);
    if (cudaGetLastError() != cudaSuccess) { rc = mm_fail(c, MM_ECUDA, "k_extract launch failed"); break; }
    c->launches++;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
      rc = mm_fail(c, MM_ECUDA, "tensor setup failed: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
  } while (0);
  cudaFree(Kc);
  if (rc != MM_OK) return rc;

  // Twiddle tables exp(-2 pi i m / L) for L = 1, 2, 4, ..., Lmax at offset L (computed in double).
  std::vector<float2> tw(2 * (size_t)c->Lmax);
  for (int L = 1; L <= c->Lmax; L *= 2)
    for (int m = 0; m < L; ++m) {
      const double ang = -2.0 * MM_PI * (double)m / (double)L;
      tw[L + m] = make_float2((float)cos(ang), (float)sin(ang));
    }
  tw[0] = make_float2(0.f, 0.f);
  MM_CK(c, cudaMemcpy(c->tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice));
  return MM_OK;
}

// Tensor set-up into caller-provided buffers (no allocation, no host copy):
// Kc = 6 nz px py double2 of scratch, Kh = the output table.  Same kernels as
// mm_build_kernel.
int mm_setup_kernel_into(const Dims& d, int self_term, double2* Kc, float* Kh, cudaStream_t s) {
  const long long plane = (long long)d.px * d.py;
  const long long total = plane * d.nz;
  k_tensor<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Kc, d, self_term);
  if (cudaGetLastError() != cudaSuccess) return -1;
  int n = 1;
  if (d.px > 1) {
    const size_t sm = 2 * sizeof(double2) * d.px;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_fft64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_fft64<<<(unsigned)(6LL * d.nz * d.py), d.px / 2 < 256 ? d.px / 2 : 256, sm, s>>>(Kc, d.px, 1, 0, d.px, 1);
    if (cudaGetLastError() != cudaSuccess) return -1;
    ++n;
  }
  if (d.py > 1) {
    const size_t sm = 2 * sizeof(double2) * d.py;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_fft64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_fft64<<<(unsigned)(6LL * d.nz * d.px), d.py / 2 < 256 ? d.py / 2 : 256, sm, s>>>(Kc, d.py, d.px, 1, plane, d.px);
    if (cudaGetLastError() != cudaSuccess) return -1;
    ++n;
  }
  const long long tot = (long long)d.hx * 6 * d.nz * d.hy;
  k_extract<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Kc, Kh, d);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return n + 1;
}

// ---------------------------------------------------------------------------
// Split-precision operands (zsplit.cuh).
// Kt[kx][kz][pair][ky], kz = 0 .. PZ/2 (ky fastest, so the lanes of a warp,
// which hold consecutive ky, read consecutive words): the x/y-transformed tensor Kh
// transformed along z with a length-PZ DFT of its offsets -(nz-1) .. nz-1,
// scaled by 1/PZ.  Pairs even in z (xx yy zz xy) give the cosine sum
// K(0) + 2 sum_d K(d) cos(2 pi kz d / PZ); pairs odd in z (xz yz, stored as
// the imaginary part of their x/y transform, acting as i Kt) give
// 2 sum_d K(d) sin(2 pi kz d / PZ), the real factor left after i (-2i) = 2.
// FP64 arithmetic on the FP32 Kh values.
// ---------------------------------------------------------------------------
__global__ void k_ktz(const float* __restrict__ Kh, float* __restrict__ Kt, Dims d, int PZ) {
  const int nkz = PZ / 2 + 1;
  const long long total = (long long)d.hx * d.hy * nkz;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int ky = (int)(idx % d.hy);
  const int kz = (int)((idx / d.hy) % nkz);
  const int kx = (int)(idx / ((long long)d.hy * nkz));
  const long long col = (long long)kx * d.hy + ky;
  for (int p = 0; p < 6; ++p) {
    const float* k = Kh + (col * 6 + p) * d.nz;
    double s;
    if (p < 4) {
      s = k[0];
      for (int dz = 1; dz < d.nz; ++dz) s += 2.0 * k[dz] * cospi(2.0 * kz * dz / PZ);
    } else {
      s = 0.0;
      for (int dz = 1; dz < d.nz; ++dz) s += 2.0 * k[dz] * sinpi(2.0 * kz * dz / PZ);
    }
    Kt[(((long long)kx * nkz + kz) * 6 + p) * d.hy + ky] = (float)(s / PZ);
  }
}

// hi/lo parts of v in the 16-bit type of the split (1: bfloat16, 2: float16)
static void split16(double v, int prec, uint16_t* hi, uint16_t* lo) {
  if (prec == MM_SPLIT_BF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
    const __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
    memcpy(hi, &h, 2);
    memcpy(lo, &l, 2);
  } else {
    const __half h = __float2half_rn((float)v);
    const __half l = __float2half_rn((float)(v - (double)__half2float(h)));
    memcpy(hi, &h, 2);
    memcpy(lo, &l, 2);
  }
}

// byte offset of element (n, k) of an N x K operand in the canonical
// no-swizzle K-major layout (core matrices of 8 rows x 16 bytes)
static size_t canon(int n, int k, int N) { return ((size_t)(k / 8) * (N / 8) + n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2; }

int mm_build_split(mm_ctx* c) {
  Dims& d = c->d;
  const int NZ = mm_nzm(d.nz), PZ = 2 * NZ;
  const long long nkt = (long long)d.hx * d.hy * (PZ / 2 + 1) * 6;
  if (cudaMalloc(&c->Kt, sizeof(float) * nkt) != cudaSuccess) {
    cudaGetLastError();
    return mm_fail(c, MM_ENOMEM, "split precision: cannot allocate the z-transformed tensor");
  }
  // GEMM 1 operand B1 (2 PZ x 2 NZ): rows re kz | im kz, columns re z | im z of
  //   sum_z m(z) e^{-2 pi i kz z / PZ}:  re = sum re cos + im sin,  im = sum im cos - re sin
  // GEMM 2 operand B2 (2 NZ x 2 PZ): rows re z | im z, columns re kz | im kz of
  //   sum_kz h(kz) e^{+2 pi i kz z / PZ}: re = sum re cos - im sin,  im = sum re sin + im cos
  const int N1 = 2 * PZ, K1 = 2 * NZ, N2 = 2 * NZ, K2 = 2 * PZ;
  const size_t B1 = (size_t)N1 * K1 * 2, B2 = (size_t)N2 * K2 * 2;
  std::vector<unsigned char> h(2 * B1 + 2 * B2, 0);
  auto put = [&](size_t base_hi, size_t base_lo, int n, int k, int N, double v) {
    uint16_t hi, lo;
    split16(v, d.prec, &hi, &lo);
    memcpy(&h[base_hi + canon(n, k, N)], &hi, 2);
    memcpy(&h[base_lo + canon(n, k, N)], &lo, 2);
  };
  for (int n = 0; n < N1; ++n)
    for (int k = 0; k < K1; ++k) {
      const int kz = n % PZ, z = k % NZ;
      const double th = 2.0 * MM_PI * kz * z / PZ;
      const bool out_im = n >= PZ, in_im = k >= NZ;
      const double v = !out_im ? (!in_im ? cos(th) : sin(th)) : (!in_im ? -sin(th) : cos(th));
      put(0, B1, n, k, N1, v);
    }
  for (int n = 0; n < N2; ++n)
    for (int k = 0; k < K2; ++k) {
      const int z = n % NZ, kz = k % PZ;
      const double th = 2.0 * MM_PI * kz * z / PZ;
      const bool out_im = n >= NZ, in_im = k >= PZ;
      const double v = !out_im ? (!in_im ? cos(th) : -sin(th)) : (!in_im ? sin(th) : cos(th));
      put(2 * B1, 2 * B1 + B2, n, k, N2, v);
    }
  if (cudaMalloc(&c->Bdft, h.size()) != cudaSuccess) {
    cudaGetLastError();
    return mm_fail(c, MM_ENOMEM, "split precision: cannot allocate the DFT operands");
  }
  MM_CK(c, cudaMemcpy(c->Bdft, h.data(), h.size(), cudaMemcpyHostToDevice));
  const long long tot = (long long)d.hx * d.hy * (PZ / 2 + 1);
  k_ktz<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(c->Kh, c->Kt, d, PZ);
  MM_CK(c, cudaGetLastError());
  c->launches++;
  MM_CK(c, cudaStreamSynchronize(c->stream));
  d.Kt = c->Kt;
  d.Bdft = c->Bdft;
  return MM_OK;
}
