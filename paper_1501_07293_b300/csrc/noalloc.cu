// mm_heff_noalloc: the effective field of a given state without any device
// allocation.  Every intermediate buffer (the FP64 tensor planes, the
// transformed tensor, the x-transformed field and the twiddle tables) is carved
// out of one file-scope static device array, so the call needs no context and
// never calls cudaMalloc or cudaFree.  mm_noalloc_status reads back the error
// flags its kernels set.  See include/mm_b300.h for the contract.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>
#include <string.h>

#include "common.cuh"

#define MM_NOALLOC_MAX_DEVICES 64

// The shared scratch.  Every GPU that loads the library holds it until exit.
// Its first 256 bytes are the kernels' error flags ([0] non-finite, [1] a
// bounded wait gave up); static storage starts zeroed, and only
// mm_noalloc_status clears them again.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MM_NOALLOC_SCRATCH_BYTES];

// Host-side device address of g_noalloc_scratch per device (the symbol itself
// is only a host stand-in and must never be passed to a kernel), with the CUDA
// context that was current when it was looked up: a different context on the
// same device (after cudaDeviceReset, the module is loaded anew) looks it up
// again.
struct ScratchSlot {
  void* addr;
  void* ctx;
};
static ScratchSlot g_slot[MM_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mutex;
static thread_local char g_noalloc_err[512] = "";

static int noalloc_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_noalloc_err, sizeof g_noalloc_err, fmt, ap);
  va_end(ap);
  return code;
}

extern "C" const char* mm_noalloc_last_error(void) { return g_noalloc_err; }

// The driver's cuCtxGetCurrent, taken through the runtime (the library does not
// link the driver library itself); null if unavailable.
typedef int (*CtxGetCurrentFn)(void**);
static CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
    else
      cudaGetLastError();
    tried = true;
  }
  return fn;
}

// Set-up: the device address of the scratch on the current device, looked up
// (cudaGetSymbolAddress, with that device current) on the first call in each
// CUDA context and cached.  Returns MM_OK or MM_ECUDA (message set).
int mm_noalloc_scratch(unsigned char** base) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MM_NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return noalloc_fail(MM_ECUDA, "mm_heff_noalloc: no usable current device");
  }
  CtxGetCurrentFn cur = ctx_get_current();
  void* ctx = nullptr;
  if (cur) cur(&ctx);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchSlot& sl = g_slot[dev];
  if (!sl.addr || !ctx || sl.ctx != ctx) {
    // (the lookup also makes the device's primary context current if none was)
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(MM_ECUDA, "mm_heff_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    }
    ctx = nullptr;
    if (cur) cur(&ctx);
    sl.addr = p;
    sl.ctx = ctx;
  }
  *base = (unsigned char*)sl.addr;
  return MM_OK;
}

// Twiddle tables exp(-2 pi i m / L), L = 1, 2, ..., Lmax, at offset L (double, rounded to float).
__global__ void k_noalloc_twiddles(float2* tw, int Lmax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * Lmax) return;
  if (i == 0) { tw[0] = make_float2(0.f, 0.f); return; }
  int L = 1;
  while (2 * L <= i) L *= 2;
  const int m = i - L;
  double s, c;
  sincospi(-2.0 * (double)m / (double)L, &s, &c);
  tw[i] = make_float2((float)c, (float)s);
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static int pow2_ge(int v) {
  int p = 1;
  while (p < v) p *= 2;
  return p;
}

extern "C" int mm_heff_noalloc(const int grid[3], double delta, double Ms, double A, double Ku,
                               const double b_ext[3], int self_term, const float* m_dev, float* H_dev,
                               unsigned term_mask, void* stream) {
  if (!grid || !b_ext || !m_dev || !H_dev) return noalloc_fail(MM_EINVAL, "mm_heff_noalloc: NULL argument");
  if (grid[0] < 1 || grid[1] < 1 || grid[2] < 1)
    return noalloc_fail(MM_EINVAL, "mm_heff_noalloc: grid %d x %d x %d has a size < 1", grid[0], grid[1], grid[2]);
  if (!(delta > 0) || !(Ms > 0) || !(A >= 0))
    return noalloc_fail(MM_EINVAL, "mm_heff_noalloc: need delta > 0, Ms > 0, A >= 0");
  if (term_mask & ~(unsigned)MM_TERM_ALL)
    return noalloc_fail(MM_EINVAL, "mm_heff_noalloc: bad term mask 0x%x", term_mask);

  Dims d;
  memset(&d, 0, sizeof d);
  d.nx = grid[0]; d.ny = grid[1]; d.nz = grid[2];
  d.px = d.nx == 1 ? 1 : pow2_ge(2 * d.nx - 1);
  d.py = d.ny == 1 ? 1 : pow2_ge(2 * d.ny - 1);
  d.hx = d.px == 1 ? 1 : d.px / 2 + 1;
  d.hy = d.py == 1 ? 1 : d.py / 2 + 1;
  d.N = (long long)d.nx * d.ny * d.nz;
  char why[256];
  if (!mm_supported(d, why, sizeof why)) return noalloc_fail(MM_EUNSUPPORTED, "mm_heff_noalloc: %s", why);
  if (!mm_yz_fused(d))
    return noalloc_fail(MM_EUNSUPPORTED, "mm_heff_noalloc: a kx column (3 x %d x %d complex) exceeds one CTA", d.nz, d.py);
  int Lmax = d.px > d.py ? d.px : d.py;
  if (Lmax < 2) Lmax = 2;

  // Scratch layout: [flags][Kh][twiddles][Kc during set-up, then S]  (S reuses Kc's bytes).
  const size_t fl_b = 256;
  const size_t kh_b = align256(sizeof(float) * (size_t)d.hx * 6 * d.nz * d.hy);
  const size_t tw_b = align256(sizeof(float2) * 2 * (size_t)Lmax);
  const size_t kc_b = align256(sizeof(double2) * 6 * (size_t)d.nz * d.px * d.py);
  const size_t s_b = align256(sizeof(float2) * (size_t)d.hx * 3 * d.nz * d.ny);
  const size_t need = fl_b + kh_b + tw_b + (kc_b > s_b ? kc_b : s_b);
  if (need > (size_t)MM_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(MM_EUNSUPPORTED,
                        "mm_heff_noalloc: grid %d x %d x %d needs %zu bytes of scratch, the static array holds %zu",
                        d.nx, d.ny, d.nz, need, (size_t)MM_NOALLOC_SCRATCH_BYTES);

  // Set-up (the scratch's device address), once per device and context.
  unsigned char* base = nullptr;
  if (int rc = mm_noalloc_scratch(&base)) return rc;
  int* flags = (int*)base;   // kernels' error flags, read by mm_noalloc_status
  d.flag = flags;
  float* Kh = (float*)(base + fl_b);
  float2* tw = (float2*)(base + fl_b + kh_b);
  double2* Kc = (double2*)(base + fl_b + kh_b + tw_b);
  float2* S = (float2*)(base + fl_b + kh_b + tw_b);
  cudaStream_t s = (cudaStream_t)stream;

  k_noalloc_twiddles<<<(2 * Lmax + 255) / 256, 256, 0, s>>>(tw, Lmax);
  if (cudaGetLastError() != cudaSuccess) return noalloc_fail(MM_ECUDA, "mm_heff_noalloc: twiddle launch failed");
  if (mm_setup_kernel_into(d, self_term ? 1 : 0, Kc, Kh, s) < 0)
    return noalloc_fail(MM_ECUDA, "mm_heff_noalloc: tensor set-up launch failed: %s", cudaGetErrorString(cudaGetLastError()));

  Phys ph;
  ph.c_ex = (float)(2.0 * A / (Ms * delta * delta));
  ph.c_an = (float)(2.0 * Ku / Ms);
  ph.c_an_map = (float)(2.0 / Ms);
  ph.c_d = (float)(MM_MU0 * Ms / ((double)d.px * (double)d.py));
  ph.bx = (float)b_ext[0];
  ph.by = (float)b_ext[1];
  ph.bz = (float)b_ext[2];
  ph.g1 = 0.f;
  ph.g2 = 0.f;
  ph.inv_mu0 = (float)(1.0 / MM_MU0);
  StageArgs a;
  memset(&a, 0, sizeof a);
  a.m_in = m_dev;
  a.H_out = H_dev;
  a.mode = 0;
  a.mask = term_mask;
  if (launch_field_eval(d, ph, a, tw, S, Kh, flags, s) < 0)
    return noalloc_fail(MM_ECUDA, "mm_heff_noalloc: field kernels failed to launch: %s",
                        cudaGetErrorString(cudaGetLastError()));
  return MM_OK;
}

extern "C" int mm_noalloc_status(void* stream) {
  unsigned char* base = nullptr;
  if (int rc = mm_noalloc_scratch(&base)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int h[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(h, base, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    return noalloc_fail(MM_ECUDA, "mm_noalloc_status: reading the flags failed: %s", cudaGetErrorString(e));
  }
  if (h[0] || h[1]) {
    if (cudaMemsetAsync(base, 0, sizeof h, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      const cudaError_t e = cudaGetLastError();
      return noalloc_fail(MM_ECUDA, "mm_noalloc_status: clearing the flags failed: %s", cudaGetErrorString(e));
    }
    if (h[1]) return noalloc_fail(MM_ETIMEOUT, "mm_heff_noalloc: a bounded wait inside a kernel gave up");
    return noalloc_fail(MM_ENONFINITE, "mm_heff_noalloc: a kernel flagged a non-finite value");
  }
  return MM_OK;
}
