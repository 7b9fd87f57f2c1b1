// Demagnetising kernel setup (once per geometry), FP64 on the device.
//
// 1. k_tensor: the tensor of eq. 10/11 for every offset 0 <= I < nx,
//    0 <= J < ny, 0 <= K < nz, written with the tensor's parities to the up to
//    four positions (+-I mod px, +-J mod py) of the padded plane of K (the
//    padding is cleared first).  Offsets are in units of delta (the tensor is
//    scale free).  Near the source (|n| < 9 cells) the eight-corner sums of
//    eq. 10/11, with log(z + r) evaluated as log((x^2 + y^2) / (r - z)) when
//    z < 0 (the same number without the cancellation of z + r).  Farther out
//    the corner sums cancel to ~eps |n|^3 relative (a few 1e-8 at 500 cells),
//    so the tensor is taken from its multipole series instead (tensor_series):
//    eq. 10/11 is the field at a cell centre of a uniformly magnetised cube,
//    i.e. K = grad grad G with G the cube's Newtonian potential
//        G(R) = 1/(4 pi) int_cube d^3r' / |R - r'|
//             = 1/(4 pi) prod_i [sinh(d_i / 2) / (d_i / 2)] 1/|R|
//    (the cube's moments factorise; only even powers of each derivative
//    remain), truncated after the terms of total derivative order 2 Kmax + 2,
//    Kmax chosen per distance for a truncation error below ~1e-15 relative.
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

// Eq. 10/11 at offset (I, J, K): the sums over the eight corners.  v: xx yy zz xy xz yz.
__device__ __forceinline__ void tensor_exact(double I, double J, double K, double (&v)[6]) {
#pragma unroll
  for (int p = 0; p < 6; ++p) v[p] = 0.0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double s = ((i + j + k) & 1) ? -1.0 : 1.0;
        const double X = I + i - 0.5, Y = J + j - 0.5, Z = K + k - 0.5;
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

// Far field: K_ij = 1/(4 pi) sum_{a,b,c even, a+b+c <= 2 Kmax} c_a c_b c_c
//                  d^(a,b,c) d_i d_j (1/R),   c_a = 1 / ((a + 1)! 2^a)
// (the series of the cube's sinh(d/2)/(d/2) factors).  The derivatives of 1/R
// come from its Taylor coefficients t_k = d^k (1/R) / k! (k a multi-index;
// here only even total orders |k| are used, where the expansion of 1/|R - h|
// in h has the same coefficients), which obey for |k| >= 1
//   |k| R^2 t_k = (2|k| - 1) sum_l R_l t_{k - e_l} - (|k| - 1) sum_l t_{k - 2 e_l},
// t_0 = 1/R, t of a negative index = 0.
static constexpr int kSeriesMaxOrder = 12;   // 2 Kmax + 2 for Kmax = 5

// position of multi-index (a, b, n - a - b) of total order n in the table
__device__ __forceinline__ int tidx(int n, int a, int b) {
  return n * (n + 1) * (n + 2) / 6 + a * (n + 1) - a * (a - 1) / 2 + b;
}

__device__ void tensor_series(double x, double y, double z, int kmax, double (&v)[6]) {
  double t[(kSeriesMaxOrder + 1) * (kSeriesMaxOrder + 2) * (kSeriesMaxOrder + 3) / 6];
  const double r2 = x * x + y * y + z * z;
  const int P = 2 * kmax + 2;
  t[0] = 1.0 / sqrt(r2);
  for (int n = 1; n <= P; ++n) {
    const double inv = 1.0 / (n * r2);
    for (int a = 0; a <= n; ++a)
      for (int b = 0; b <= n - a; ++b) {
        const int c = n - a - b;
        double s1 = 0.0, s2 = 0.0;
        if (a >= 1) s1 += x * t[tidx(n - 1, a - 1, b)];
        if (b >= 1) s1 += y * t[tidx(n - 1, a, b - 1)];
        if (c >= 1) s1 += z * t[tidx(n - 1, a, b)];
        if (n >= 2) {
          if (a >= 2) s2 += t[tidx(n - 2, a - 2, b)];
          if (b >= 2) s2 += t[tidx(n - 2, a, b - 2)];
          if (c >= 2) s2 += t[tidx(n - 2, a, b)];
        }
        t[tidx(n, a, b)] = ((2 * n - 1) * s1 - (n - 1) * s2) * inv;
      }
  }
  // (2a)! c_{2a} = 1 / ((2a + 1) 4^a) is folded with the factorials of the pair below
  const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
  for (int p = 0; p < 6; ++p) {
    double sum = 0.0;
    for (int k = 0; k <= kmax; ++k)
      for (int a2 = 0; a2 <= k; ++a2)
        for (int b2 = 0; b2 <= k - a2; ++b2) {
          const int c2 = k - a2 - b2;
          int e[3] = {2 * a2, 2 * b2, 2 * c2};
          e[pi[p]] += 1;
          e[pj[p]] += 1;
          // c_{2a} (beta_x)! etc.: beta! / ((2a + 1)! 4^a) per axis
          double w = 1.0;
          const int h[3] = {a2, b2, c2};
          for (int ax = 0; ax < 3; ++ax) {
            double f = 1.0;   // beta_ax! / (2 h + 1)!
            for (int q = 2 * h[ax] + 2; q <= e[ax]; ++q) f *= q;
            for (int q = e[ax] + 1; q <= 2 * h[ax] + 1; ++q) f /= q;
            w *= f / (double)(1 << (2 * h[ax]));
          }
          sum += w * t[tidx(e[0] + e[1] + e[2], e[0], e[1])];
        }
    v[p] = sum / (4.0 * MM_PI);
  }
}

// Truncation order of the far-field series by distance |n| (cells): a relative
// truncation error below ~3e-14 at 9 cells and ~1e-15 beyond 12 (measured
// against a 50-digit evaluation of eq. 10/11), where the FP64 corner sums are
// off by up to ~6e-13 at 9 cells; 0 = use the corner sums.
__device__ __forceinline__ int series_order(double n2) {
  if (n2 < 81.0) return 0;         // |n| < 9
  if (n2 < 400.0) return 5;        // < 20
  if (n2 < 2500.0) return 4;       // < 50
  if (n2 < 25600.0) return 3;      // < 160
  return 2;
}

__device__ __forceinline__ void tensor_eval(int I, int J, int K, double (&v)[6]) {
  const double n2 = (double)I * I + (double)J * J + (double)K * K;
  const int ord = series_order(n2);
  if (ord == 0) tensor_exact(I, J, K, v);
  else tensor_series(I, J, K, ord, v);
}

// One thread per offset I, J, K >= 0; the tensor at (+-I, +-J) follows from its
// parities (xy odd in I and J, xz odd in I, yz odd in J; all even in K here).
__global__ void k_tensor(double2* __restrict__ Kc, Dims d, int self_term) {
  const long long total = (long long)d.nx * d.ny * d.nz;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int I = (int)(idx % d.nx);
  const int J = (int)((idx / d.nx) % d.ny);
  const int kz = (int)(idx / ((long long)d.nx * d.ny));
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (self_term || I != 0 || J != 0 || kz != 0) tensor_eval(I, J, kz, v);
  const long long plane = (long long)d.px * d.py;
  for (int sj = 0; sj < (J ? 2 : 1); ++sj)
    for (int si = 0; si < (I ? 2 : 1); ++si) {
      const int x = si ? d.px - I : I, y = sj ? d.py - J : J;
      const double fI = si ? -1.0 : 1.0, fJ = sj ? -1.0 : 1.0;
      const double w[6] = {v[0], v[1], v[2], fI * fJ * v[3], fI * v[4], fJ * v[5]};
      for (int p = 0; p < 6; ++p)
        Kc[((long long)p * d.nz + kz) * plane + (long long)y * d.px + x] = make_double2(w[p], 0.0);
    }
}

// The tensor at given offsets, as k_tensor evaluates it (mm_tensor_eval).
__global__ void k_tensor_at(const int* __restrict__ off, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v[6];
  tensor_eval(off[3 * i], off[3 * i + 1], off[3 * i + 2], v);
  for (int p = 0; p < 6; ++p) out[6 * i + p] = v[p];
}

// One CTA per line of length L (power of two), radix-2 Stockham, ping-pong in
// shared memory; the twiddles exp(-2 pi i k / L), k < L/2, are tabulated once
// per CTA (one sincospi per thread instead of one per butterfly and stage).
// Line l starts at (l / inner) * outer + (l % inner) * inner_step; elements are estride apart.
__global__ void k_fft64(double2* __restrict__ data, int L, long long inner, long long inner_step,
                        long long outer, long long estride) {
  extern __shared__ double2 sh64[];
  double2* a = sh64;
  double2* b = sh64 + L;
  double2* w = sh64 + 2 * L;
  const long long l = blockIdx.x;
  const long long base = (l / inner) * outer + (l % inner) * inner_step;
  const int half = L / 2;
  for (int k = threadIdx.x; k < half; k += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)L, &sn, &cs);
    w[k] = make_double2(cs, sn);
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) a[i] = data[base + i * estride];
  __syncthreads();
  for (int ns = 1; ns < L; ns *= 2) {
    const int step = L / (2 * ns);   // exp(-2 pi i k / (2 ns)) = w[k step]
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
      const int k = j & (ns - 1);
      const double2 u = a[j], v = a[j + half];
      const double2 tw = w[k * step];
      const double2 t = make_double2(v.x * tw.x - v.y * tw.y, v.x * tw.y + v.y * tw.x);
      const int o = (j - k) * 2 + k;
      b[o] = make_double2(u.x + t.x, u.y + t.y);
      b[o + ns] = make_double2(u.x - t.x, u.y - t.y);
    }
    __syncthreads();
    double2* tmp = a; a = b; b = tmp;
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

// Tensor set-up into caller-provided buffers (no allocation, no host copy):
// Kc = 6 nz px py double2 of scratch, Kh = the output table.  Returns the
// kernels launched (not counting the clearing of Kc) or < 0.
int mm_setup_kernel_into(const Dims& d, int self_term, double2* Kc, float* Kh, cudaStream_t s) {
  const long long plane = (long long)d.px * d.py;
  if (cudaMemsetAsync(Kc, 0, sizeof(double2) * 6 * (size_t)d.nz * plane, s) != cudaSuccess) return -1;
  const long long offsets = (long long)d.nx * d.ny * d.nz;
  k_tensor<<<(unsigned)((offsets + 127) / 128), 128, 0, s>>>(Kc, d, self_term);
  if (cudaGetLastError() != cudaSuccess) return -1;
  int n = 1;
  // x lines: 6 nz py lines of px contiguous elements; y lines: for every plane
  // and x, py elements px apart
  if (d.px > 1) {
    const size_t sm = sizeof(double2) * (2 * (size_t)d.px + d.px / 2);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_fft64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_fft64<<<(unsigned)(6LL * d.nz * d.py), d.px / 2 < 256 ? d.px / 2 : 256, sm, s>>>(Kc, d.px, 1, 0, d.px, 1);
    if (cudaGetLastError() != cudaSuccess) return -1;
    ++n;
  }
  if (d.py > 1) {
    const size_t sm = sizeof(double2) * (2 * (size_t)d.py + d.py / 2);
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
  const int k = mm_setup_kernel_into(d, c->opts.self_term, Kc, c->Kh, c->stream);
  if (k < 0) rc = mm_fail(c, MM_ECUDA, "tensor setup launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  else c->launches += k;
  if (rc == MM_OK && cudaStreamSynchronize(c->stream) != cudaSuccess)
    rc = mm_fail(c, MM_ECUDA, "tensor setup failed: %s", cudaGetErrorString(cudaGetLastError()));
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

extern "C" int mm_tensor_eval(const int* offsets, int n, double* out) {
  if (!offsets || !out || n < 1 || n > (1 << 20)) return MM_EINVAL;
  int* d_off = nullptr;
  double* d_out = nullptr;
  int rc = MM_OK;
  if (cudaMalloc(&d_off, sizeof(int) * 3 * (size_t)n) != cudaSuccess ||
      cudaMalloc(&d_out, sizeof(double) * 6 * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    rc = MM_ENOMEM;
  } else if (cudaMemcpy(d_off, offsets, sizeof(int) * 3 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = MM_ECUDA;
  } else {
    k_tensor_at<<<(n + 127) / 128, 128>>>(d_off, n, d_out);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(out, d_out, sizeof(double) * 6 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = MM_ECUDA;
  }
  cudaGetLastError();
  cudaFree(d_off);
  cudaFree(d_out);
  return rc;
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
  // one thread per (kx, ky); cos / sin (2 pi kz dz / PZ) tabulated once per block
  // (kz <= PZ / 2, dz < nz <= PZ / 2) instead of one sincospi per term
  __shared__ double cs[33 * 32], sn[33 * 32];
  const int nkz = PZ / 2 + 1;
  for (int i = threadIdx.x; i < nkz * d.nz; i += blockDim.x) {
    const int kz = i / d.nz, dz = i % d.nz;
    sincospi(2.0 * ((kz * dz) % PZ) / PZ, &sn[i], &cs[i]);
  }
  __syncthreads();
  const long long total = (long long)d.hx * d.hy;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int ky = (int)(idx % d.hy);
  const int kx = (int)(idx / d.hy);
  for (int p = 0; p < 6; ++p) {
    const float* k = Kh + (idx * 6 + p) * d.nz;
    float kv[32];
    for (int dz = 0; dz < d.nz; ++dz) kv[dz] = k[dz];
    for (int kz = 0; kz < nkz; ++kz) {
      const double* t = (p < 4 ? cs : sn) + kz * d.nz;
      double s = p < 4 ? (double)kv[0] : 0.0;
      for (int dz = 1; dz < d.nz; ++dz) s += 2.0 * (double)kv[dz] * t[dz];
      Kt[(((long long)kx * nkz + kz) * 6 + p) * d.hy + ky] = (float)(s / PZ);
    }
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

// Kt from Kh (above), PZ = 2 * NZM; synchronises the context's stream.
static int build_kt(mm_ctx* c) {
  Dims& d = c->d;
  const int PZ = 2 * mm_nzm(d.nz);
  const long long nkt = (long long)d.hx * d.hy * (PZ / 2 + 1) * 6;
  if (!c->Kt && cudaMalloc(&c->Kt, sizeof(float) * nkt) != cudaSuccess) {
    cudaGetLastError();
    c->Kt = nullptr;
    return mm_fail(c, MM_ENOMEM, "cannot allocate the z-transformed tensor");
  }
  const long long tot = (long long)d.hx * d.hy;
  k_ktz<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(c->Kh, c->Kt, d, PZ);
  MM_CK(c, cudaGetLastError());
  c->launches++;
  MM_CK(c, cudaStreamSynchronize(c->stream));
  d.Kt = c->Kt;
  return MM_OK;
}

// FP32 path: the z product as a length-32 transform (field_kernels.cuh
// zprod_fft_column) needs Kt with PZ = 32.
int mm_build_kz(mm_ctx* c) {
  const int rc = build_kt(c);
  if (rc == MM_OK) c->d.zfft = 1;
  return rc;
}

int mm_build_split(mm_ctx* c) {
  Dims& d = c->d;
  const int NZ = mm_nzm(d.nz), PZ = 2 * NZ;
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
  d.Bdft = c->Bdft;
  return build_kt(c);
}
