// C ABI of libmm_b300 (declared in include/mm_b300.h): context life cycle,
// state and field set-up, the captured step graph, energies and observables.
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

// NVTX range around an entry point (visible in Nsight timelines; free when no
// tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

static char g_create_err[512] = "";

int mm_fail(mm_ctx* c, int code, const char* fmt, ...) {
  char* dst = c ? c->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

static int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p *= 2;
  return p;
}

Phys mm_make_phys(const mm_ctx* c) {
  Phys ph;
  const double Ms = c->Ms, dl = c->delta;
  ph.c_ex = (float)(2.0 * c->A / (Ms * dl * dl));
  ph.c_an = (float)(2.0 * c->Ku / Ms);
  ph.c_an_map = (float)(2.0 / Ms);
  ph.c_d = (float)(MM_MU0 * Ms / ((double)c->d.px * (double)c->d.py));
  ph.bx = (float)c->b_ext[0];
  ph.by = (float)c->b_ext[1];
  ph.bz = (float)c->b_ext[2];
  const double g = c->gamma / (1.0 + c->alpha * c->alpha);
  ph.g1 = (float)(-g);
  ph.g2 = (float)(-c->alpha * g);
  ph.inv_mu0 = (float)(1.0 / MM_MU0);
  return ph;
}

// The tensor map of S for the x kernel's tiled loads: a 4-D float view
// {2 ny, nz, 3, hx} of S[kx][c][z][y] (float2), tile {2 TY, 1, 3, 129}.  Needs
// ny even (16-byte row strides) and 8 <= px <= 512 (two tiles of 129 kx, 8
// rows per tile); otherwise, or if the driver has no encoder, the kernel keeps
// its per-thread copies.  The encoder is taken from the driver through the
// runtime, so the library does not link the driver library itself.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static void make_xmap(mm_ctx* c) {
  const Dims& d = c->d;
  if (d.ny % 2 != 0 || d.px < 8 || d.px > 512) return;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return;
  }
  CUtensorMap* m = (CUtensorMap*)aligned_alloc(64, sizeof(CUtensorMap));
  if (!m) return;
  const cuuint64_t dims[4] = {2ull * d.ny, (cuuint64_t)d.nz, 3ull, (cuuint64_t)d.hx};
  const cuuint64_t strides[3] = {8ull * d.ny, 8ull * d.ny * d.nz, 24ull * d.ny * d.nz};
  const cuuint32_t box[4] = {16u, 1u, 3u, 129u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUresult r = ((EncodeTiledFn)fn)(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)c->S, dims, strides, box, estr,
                                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    free(m);
    return;
  }
  c->xmap = m;
}

static void drop_graphs(mm_ctx* c) {
  for (int i = 0; i < 4; ++i)
    if (c->graph[i]) {
      cudaGraphExecDestroy(c->graph[i]);
      c->graph[i] = nullptr;
    }
  c->graph_valid = 0;
}

extern "C" void mm_default_opts(mm_opts* o) {
  if (!o) return;
  o->precision = MM_FP32;
  o->integrator = MM_RK4;
  o->self_term = 1;
  o->obs_every = 0;
  o->stream = nullptr;
  o->tune_cache = nullptr;
  o->zform = MM_ZFORM_AUTO;
}

static void free_ctx(mm_ctx* c) {
  if (!c) return;
  drop_graphs(c);
  cudaFree(c->m0); cudaFree(c->stA); cudaFree(c->stB); cudaFree(c->acc); cudaFree(c->Hs);
  cudaFree(c->hmap); cudaFree(c->kumap); cudaFree(c->S); cudaFree(c->Kh); cudaFree(c->tw);
  cudaFree(c->red); cudaFree(c->red_out); cudaFree(c->dflag); cudaFree(c->prog);
  cudaFree(c->Kt); cudaFree(c->Bdft); cudaFree(c->series); cudaFree(c->T);
  free(c->xmap);
  mm_adjoint_free(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->ev) cudaEventDestroy(c->ev);
  free(c);
}

extern "C" void mm_destroy(mm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

// Launch shape recorded for this context in a tune cache (JSON written by the
// Python autotuner): the record under "<px>x<py>x<nz>:<precision>" holds integer
// fields "yz_route" and "zt_block".  Returns 1 and the values if found.
static int read_tune_cache(const char* path, const mm_ctx* c, int* route, int* block) {
  FILE* f = fopen(path, "rb");
  if (!f) return 0;
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, n);
  fclose(f);
  const char* prec = c->d.prec == MM_SPLIT_BF16 ? "split_bf16" : (c->d.prec == MM_SPLIT_FP16 ? "split_fp16" : "fp32");
  char key[96];
  snprintf(key, sizeof key, "\"%dx%dx%d:%s\"", c->d.px, c->d.py, c->d.nz, prec);
  size_t at = txt.find(key);
  if (at == std::string::npos) return 0;
  at = txt.find('{', at);
  if (at == std::string::npos) return 0;
  size_t end = at;
  for (int depth = 0; end < txt.size(); ++end) {   // the record's closing brace
    if (txt[end] == '{') ++depth;
    else if (txt[end] == '}' && --depth == 0) break;
  }
  const std::string rec = txt.substr(at, end - at);
  auto field = [&](const char* name, int* out) {
    const size_t k = rec.find(name);
    if (k == std::string::npos) return false;
    const size_t colon = rec.find(':', k);
    return colon != std::string::npos && sscanf(rec.c_str() + colon + 1, "%d", out) == 1;
  };
  return field("\"yz_route\"", route) && field("\"zt_block\"", block) ? 1 : 0;
}

#define ALLOC(ptr, bytes)                                                                       \
  do {                                                                                          \
    if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) {                                   \
      cudaGetLastError();                                                                       \
      rc = mm_fail(nullptr, MM_ENOMEM, "cannot allocate %zu bytes of device memory", (size_t)(bytes)); \
      goto fail;                                                                                \
    }                                                                                           \
  } while (0)

extern "C" int mm_create(mm_ctx** out, const int grid[3], double delta, double Ms, double A, double Ku,
                         double alpha, double gamma, const mm_opts* opts) {
  NvtxRange nvtx_("mm_create");
  if (!out) return mm_fail(nullptr, MM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grid) return mm_fail(nullptr, MM_EINVAL, "grid is NULL");
  if (grid[0] < 1 || grid[1] < 1 || grid[2] < 1)
    return mm_fail(nullptr, MM_EINVAL, "grid %d x %d x %d: every size must be >= 1", grid[0], grid[1], grid[2]);
  if (!(delta > 0) || !(Ms > 0) || !(A >= 0) || !(Ku >= 0 || Ku < 0) || !(alpha >= 0) || !(gamma > 0))
    return mm_fail(nullptr, MM_EINVAL, "material parameters out of range (delta, Ms, gamma > 0; A, alpha >= 0)");
  mm_opts o;
  mm_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision != MM_FP32 && o.precision != MM_SPLIT_BF16 && o.precision != MM_SPLIT_FP16)
    return mm_fail(nullptr, MM_EINVAL, "unknown precision mode %d", o.precision);
  if (o.integrator != MM_RK4 && o.integrator != MM_EULER)
    return mm_fail(nullptr, MM_EINVAL, "unknown integrator %d", o.integrator);
  if (o.obs_every < 0) return mm_fail(nullptr, MM_EINVAL, "obs_every = %d < 0", o.obs_every);
  if (o.zform != MM_ZFORM_AUTO && o.zform != MM_ZFORM_DIRECT)
    return mm_fail(nullptr, MM_EINVAL, "unknown zform %d", o.zform);

  int rc = MM_OK;
  mm_ctx* c = (mm_ctx*)calloc(1, sizeof(mm_ctx));
  if (!c) return mm_fail(nullptr, MM_ENOMEM, "host allocation failed");
  c->d.nx = grid[0]; c->d.ny = grid[1]; c->d.nz = grid[2];
  c->d.px = grid[0] == 1 ? 1 : pow2_at_least(2 * grid[0] - 1);
  c->d.py = grid[1] == 1 ? 1 : pow2_at_least(2 * grid[1] - 1);
  c->d.hx = c->d.px == 1 ? 1 : c->d.px / 2 + 1;
  c->d.hy = c->d.py == 1 ? 1 : c->d.py / 2 + 1;
  c->d.N = (long long)grid[0] * grid[1] * grid[2];
  c->d.prec = o.precision;
  // Programmatic serialization lets a stage kernel's blocks start while the one
  // before drains; it pays on large grids and costs a few microseconds a step on
  // small, launch-bound ones (166 x 42 x 1 film: 15.9 -> 20.0 us, measured)
  c->d.pdl = (long long)c->d.px * c->d.py * grid[2] >= (1LL << 20);
  c->delta = delta; c->Ms = Ms; c->A = A; c->Ku = Ku; c->alpha = alpha; c->gamma = gamma;
  c->opts = o;
  c->stream = (cudaStream_t)o.stream;
  c->Lmax = c->d.px > c->d.py ? c->d.px : c->d.py;
  if (c->Lmax < 2) c->Lmax = 2;
  {
    char why[256];
    if (!mm_supported(c->d, why, sizeof why)) {
      rc = mm_fail(nullptr, MM_EUNSUPPORTED, "grid %d x %d x %d: %s", grid[0], grid[1], grid[2], why);
      goto fail;
    }
  }
  {
    const size_t v3 = sizeof(float) * 3 * (size_t)c->d.N;
    ALLOC(c->m0, v3);
    ALLOC(c->stA, v3);
    ALLOC(c->stB, v3);
    ALLOC(c->acc, v3);
    ALLOC(c->Hs, v3);
    ALLOC(c->S, sizeof(float2) * (size_t)c->d.hx * 3 * c->d.nz * c->d.ny);
    ALLOC(c->Kh, sizeof(float) * (size_t)c->d.hx * 6 * c->d.nz * c->d.hy);
    ALLOC(c->tw, sizeof(float2) * 2 * (size_t)c->Lmax);
    long long nb = (c->d.N + 255) / 256;
    if (nb > 1184) nb = 1184;
    if (nb < 1) nb = 1;
    c->red_blocks = (int)nb;
    ALLOC(c->red, sizeof(double) * 9 * (size_t)nb);
    ALLOC(c->red_out, sizeof(double) * 16);
    ALLOC(c->dflag, sizeof(int) * 4);
    c->d.flag = c->dflag;
    ALLOC(c->prog, sizeof(ProgState));
    if (!mm_yz_fused(c->d)) {   // the split y/z pass meets in a global buffer
      ALLOC(c->T, sizeof(float2) * (size_t)c->d.hx * 3 * c->d.nz * c->d.py);
      c->d.T = c->T;
    }
    if (o.obs_every > 0) {
      c->series_cap = MM_SERIES_CAP;
      ALLOC(c->series, sizeof(double) * 6 * (size_t)c->series_cap);
    }
  }
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    rc = mm_fail(nullptr, MM_ECUDA, "stream/event creation failed");
    goto fail;
  }
  if (cudaMemsetAsync(c->dflag, 0, sizeof(int) * 4, c->stream) != cudaSuccess) {
    rc = mm_fail(nullptr, MM_ECUDA, "memset failed");
    goto fail;
  }
  make_xmap(c);
  if (c->series && cudaMemsetAsync(c->series, 0, sizeof(double) * 6 * (size_t)c->series_cap, c->stream) != cudaSuccess) {
    rc = mm_fail(nullptr, MM_ECUDA, "memset failed");
    goto fail;
  }
  if (mm_prog_init(c) != MM_OK) {
    rc = mm_fail(nullptr, MM_ECUDA, "field program initialisation failed");
    goto fail;
  }
  rc = mm_build_kernel(c);
  if (rc == MM_OK && c->d.prec != MM_FP32) rc = mm_build_split(c);
  // the transform form of the z product: 9..16 planes, py = 256 / 512, fused y/z kernel
  if (rc == MM_OK && c->d.prec == MM_FP32 && o.zform == MM_ZFORM_AUTO && mm_nzm(c->d.nz) == 16 &&
      (c->d.py == 256 || c->d.py == 512) && mm_yz_fused(c->d))
    rc = mm_build_kz(c);
  if (rc != MM_OK) {
    snprintf(g_create_err, sizeof g_create_err, "%s", c->err);
    goto fail;
  }
  if (o.tune_cache) {   // launch shapes recorded by the autotuner for this size
    int route = 0, block = 0;
    if (read_tune_cache(o.tune_cache, c, &route, &block) && mm_set_tuning(c, route, block) != MM_OK) {
      snprintf(g_create_err, sizeof g_create_err, "%s", c->err);
      rc = MM_EINVAL;
      goto fail;
    }
    c->opts.tune_cache = nullptr;   // the path need not outlive mm_create
  }
  {
    // m = (1, 0, 0)
    float* h = (float*)calloc(3 * (size_t)c->d.N, sizeof(float));
    if (!h) { rc = mm_fail(nullptr, MM_ENOMEM, "host allocation failed"); goto fail; }
    for (long long i = 0; i < c->d.N; ++i) h[i] = 1.0f;
    cudaError_t e = cudaMemcpy(c->m0, h, sizeof(float) * 3 * (size_t)c->d.N, cudaMemcpyHostToDevice);
    free(h);
    if (e != cudaSuccess) { rc = mm_fail(nullptr, MM_ECUDA, "initial state upload failed"); goto fail; }
  }
  *out = c;
  return MM_OK;
fail:
  free_ctx(c);
  return rc;
}

extern "C" int mm_set_stream(mm_ctx* c, void* stream) {
  if (!c) return MM_EINVAL;
  c->stream = (cudaStream_t)stream;
  c->opts.stream = stream;
  return MM_OK;
}

extern "C" int mm_padded_dims(const mm_ctx* c, int padded[3]) {
  if (!c || !padded) return MM_EINVAL;
  padded[0] = c->d.px;
  padded[1] = c->d.py;
  padded[2] = c->d.nz;  // z is summed directly, never padded
  return MM_OK;
}

static float* state_ptr(mm_ctx* c) { return c->cur ? c->stA : c->m0; }

extern "C" int mm_set_m(mm_ctx* c, const float* m) {
  if (!c) return MM_EINVAL;
  if (!m) return mm_fail(c, MM_EINVAL, "mm_set_m: m is NULL");
  c->cur = 0;
  c->s_valid = 0;
  // page-locked host memory: the normalising kernel reads it over the bus
  // directly (the SMs keep many more reads in flight than one copy engine);
  // device or pageable memory: one copy, then normalisation in place
  cudaPointerAttributes at;
  const bool pinned = cudaPointerGetAttributes(&at, m) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                      at.devicePointer != nullptr && (c->d.N % 4) == 0 &&
                      ((uintptr_t)at.devicePointer % 16) == 0;
  cudaGetLastError();   // a pointer the runtime does not know (pageable) is not an error here
  if (pinned) {
    if (launch_normalise_from(c->d, (const float*)at.devicePointer, c->m0, c->dflag, c->stream) < 0)
      return mm_fail(c, MM_ECUDA, "normalise launch failed");
  } else {
    MM_CK(c, cudaMemcpyAsync(c->m0, m, sizeof(float) * 3 * (size_t)c->d.N, cudaMemcpyDefault, c->stream));
    if (launch_normalise(c->d, c->m0, c->dflag, c->stream) < 0) return mm_fail(c, MM_ECUDA, "normalise launch failed");
  }
  c->launches++;
  c->steps = 0;
  // the step count (and the observables series) restarts with the new state
  MM_CK(c, cudaMemsetAsync(&c->prog->nstep, 0, sizeof(long long), c->stream));
  if (c->series) MM_CK(c, cudaMemsetAsync(c->series, 0, sizeof(double) * 6 * (size_t)c->series_cap, c->stream));
  return MM_OK;
}

extern "C" int mm_get_m(mm_ctx* c, float* m) {
  if (!c) return MM_EINVAL;
  if (!m) return mm_fail(c, MM_EINVAL, "mm_get_m: m is NULL");
  MM_CK(c, cudaMemcpyAsync(m, state_ptr(c), sizeof(float) * 3 * (size_t)c->d.N, cudaMemcpyDefault, c->stream));
  return MM_OK;
}

extern "C" int mm_set_field(mm_ctx* c, const double b_ext[3], const float* h_map, const float* ku_map) {
  if (!c) return MM_EINVAL;
  if (!b_ext) return mm_fail(c, MM_EINVAL, "mm_set_field: b_ext is NULL");
  for (int i = 0; i < 3; ++i) c->b_ext[i] = b_ext[i];
  const size_t N = (size_t)c->d.N;
  if (h_map) {
    if (!c->hmap && cudaMalloc(&c->hmap, sizeof(float) * 3 * N) != cudaSuccess) {
      cudaGetLastError();
      return mm_fail(c, MM_ENOMEM, "cannot allocate the field map");
    }
    MM_CK(c, cudaMemcpyAsync(c->hmap, h_map, sizeof(float) * 3 * N, cudaMemcpyDefault, c->stream));
  } else if (c->hmap) {
    MM_CK(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->hmap);
    c->hmap = nullptr;
  }
  if (ku_map) {
    if (!c->kumap && cudaMalloc(&c->kumap, sizeof(float) * N) != cudaSuccess) {
      cudaGetLastError();
      return mm_fail(c, MM_ENOMEM, "cannot allocate the Ku map");
    }
    MM_CK(c, cudaMemcpyAsync(c->kumap, ku_map, sizeof(float) * N, cudaMemcpyDefault, c->stream));
  } else if (c->kumap) {
    MM_CK(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->kumap);
    c->kumap = nullptr;
  }
  c->graph_valid = 0;   // kernel parameters changed: re-captured and updated in place by mm_step
  c->param_gen++;
  return mm_prog_push_base(c);
}

extern "C" int mm_set_alpha(mm_ctx* c, double alpha) {
  if (!c) return MM_EINVAL;
  if (!(alpha >= 0)) return mm_fail(c, MM_EINVAL, "alpha must be >= 0");
  c->alpha = alpha;
  c->graph_valid = 0;
  c->param_gen++;
  return mm_prog_push_base(c);
}

// Device address of drive slot s (0..3: RK4 stages of the step under way, 4:
// at the clock) while a field program is installed; otherwise NULL and the
// kernels take the uniform field and damping from their parameters.
static const float* drive_slot(mm_ctx* c, int s) { return c->prog_n > 0 ? &c->prog->drive[s][0] : nullptr; }

static StageArgs base_args(mm_ctx* c) {
  StageArgs a;
  memset(&a, 0, sizeof a);
  a.hmap = c->hmap;
  a.kumap = c->kumap;
  a.drive = drive_slot(c, 4);
  a.xmap = c->xmap;
  return a;
}

// Stage s of a step: its drive slot, and at s = 0 the tick that advances the
// clock (always) and fills the slots.
static void stage_drive(mm_ctx* c, StageArgs& a, int s, double dt) {
  a.drive = drive_slot(c, s);
  a.tick = Tick{};
  if (s == 0) a.tick = Tick{c->prog, dt, c->opts.integrator == MM_EULER};
}

extern "C" int mm_heff(mm_ctx* c, float* H, unsigned mask) {
  NvtxRange nvtx_("mm_heff");
  if (!c) return MM_EINVAL;
  if (!H) return mm_fail(c, MM_EINVAL, "mm_heff: H is NULL");
  if (mask & ~(unsigned)MM_TERM_ALL) return mm_fail(c, MM_EINVAL, "mm_heff: bad term mask 0x%x", mask);
  StageArgs a = base_args(c);
  a.m_in = state_ptr(c);
  a.H_out = H;
  a.mode = 0;
  a.mask = mask;
  const int k = launch_field_eval(c->d, mm_make_phys(c), a, c->tw, c->S, c->Kh, c->dflag, c->stream);
  c->s_valid = 0;
  if (k < 0) return mm_fail(c, MM_ECUDA, "field kernels failed to launch (%d): %s", k, cudaGetErrorString(cudaGetLastError()));
  c->launches += k;
  return MM_OK;
}

// Enqueue one step on stream s; `from` = buffer holding the state (Euler alternates).
// S must hold the x transform of that state on entry; it holds the transform of
// the new state on exit.
static int enqueue_step(mm_ctx* c, cudaStream_t s, double dt, int from, long long* nk) {
  const Phys ph = mm_make_phys(c);
  StageArgs a = base_args(c);
  a.dt = (float)dt;
  *nk = 0;
  if (c->opts.integrator == MM_EULER) {
    a.mode = 2;
    a.m_in = from ? c->stA : c->m0;
    a.m_out = from ? c->m0 : c->stA;
    stage_drive(c, a, 0, dt);
    if (c->series) a.maxdmdt = &c->prog->maxdmdt;
    const int k = launch_stage(c->d, ph, a, c->tw, c->S, c->Kh, c->dflag, s);
    if (k < 0) return k;
    *nk += k;
    if (c->series) {
      if (launch_record(c, a.m_out, s) < 0) return -4;
      *nk += 1;
    }
    return 0;
  }
  a.mode = 1;
  a.m0 = c->m0;
  a.acc = c->acc;
  const float* in[4] = {c->m0, c->stA, c->stB, c->stA};
  float* outp[4] = {c->stA, c->stB, c->stA, c->m0};
  for (int s4 = 0; s4 < 4; ++s4) {
    a.stage = s4;
    a.m_in = in[s4];
    a.m_out = outp[s4];
    stage_drive(c, a, s4, dt);
    a.maxdmdt = (c->series && s4 == 0) ? &c->prog->maxdmdt : nullptr;
    const int k = launch_stage(c->d, ph, a, c->tw, c->S, c->Kh, c->dflag, s);
    if (k < 0) return k;
    *nk += k;
  }
  if (c->series) {
    if (launch_record(c, c->m0, s) < 0) return -4;
    *nk += 1;
  }
  return 0;
}

// Make S the x transform of the current state (after mm_set_m, mm_heff, ...).
static int ensure_spectrum(mm_ctx* c) {
  if (c->s_valid) return MM_OK;
  if (launch_xfwd(c->d, state_ptr(c), c->tw, c->S, c->stream) < 0)
    return mm_fail(c, MM_ECUDA, "x-transform launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  c->launches++;
  c->s_valid = 1;
  return MM_OK;
}

// Steps per graph of the long form: mm_step replays whole graphs of this many
// steps (an even count, so Euler's alternating buffers end where they began)
// and single steps for the rest, so consecutive steps are joined by the graph's
// own edges rather than by a graph launch each.
static constexpr int kStepsPerGraph = 16;

// Capture the step sequence.  An existing executable graph of the same shape
// (only kernel parameters changed: dt, the field, the damping, map pointers)
// is updated in place; otherwise it is instantiated anew.  graph[g] holds one
// step from buffer g, graph[2 + g] kStepsPerGraph steps from it.
static int build_graphs(mm_ctx* c, double dt) {
  if (c->graph_integrator != c->opts.integrator) drop_graphs(c);
  const bool euler = c->opts.integrator == MM_EULER;
  const int ng = euler ? 2 : 1;
  for (int gi = 0; gi < 2 * ng; ++gi) {
    const int g = gi < ng ? gi : 2 + (gi - ng);   // slot: 0, (1,) 2, (3)
    const int from = g & 1;
    const int nsteps = g >= 2 ? kStepsPerGraph : 1;
    cudaGraph_t graph;
    MM_CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    long long nk = 0;
    int r = 0;
    for (int i = 0; i < nsteps && r >= 0; ++i) {
      long long k1 = 0;
      r = enqueue_step(c, c->cap_stream, dt, euler ? (from + i) & 1 : 0, &k1);
      nk += k1;
    }
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (r < 0 || e != cudaSuccess) {
      cudaGetLastError();
      return mm_fail(c, MM_ECUDA, "graph capture failed (%d, %s)", r, cudaGetErrorString(e));
    }
    bool updated = false;
    if (c->graph[g]) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(c->graph[g], graph, &info) == cudaSuccess) {
        updated = true;
      } else {
        cudaGetLastError();
        cudaGraphExecDestroy(c->graph[g]);
        c->graph[g] = nullptr;
      }
    }
    if (!updated) {
      e = cudaGraphInstantiate(&c->graph[g], graph, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        c->graph[g] = nullptr;
        c->graph_valid = 0;
        return mm_fail(c, MM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
      }
    }
    cudaGraphDestroy(graph);
    c->graph_nodes[g] = nk;
    // upload now, so the first replay inside a caller's timed loop does not pay for it
    MM_CK(c, cudaGraphUpload(c->graph[g], c->stream));
  }
  c->graph_valid = 1;
  c->graph_dt = dt;
  c->graph_integrator = c->opts.integrator;
  return MM_OK;
}

extern "C" int mm_step(mm_ctx* c, int n, double dt) {
  NvtxRange nvtx_("mm_step");
  if (!c) return MM_EINVAL;
  if (n < 0) return mm_fail(c, MM_EINVAL, "mm_step: n = %d < 0", n);
  if (!(dt > 0) || dt > 1e-6) return mm_fail(c, MM_EINVAL, "mm_step: dt = %g s out of range (0, 1e-6]", dt);
  if (n == 0) return MM_OK;
  if (!c->graph_valid || c->graph_dt != dt || c->graph_integrator != c->opts.integrator) {
    const int r = build_graphs(c, dt);
    if (r != MM_OK) return r;
  }
  {
    const int r = ensure_spectrum(c);
    if (r != MM_OK) return r;
  }
  const bool euler = c->opts.integrator == MM_EULER;
  int i = 0;
  for (; i + kStepsPerGraph <= n; i += kStepsPerGraph) {   // an even count: Euler's buffer is unchanged
    const int g = 2 + (euler ? c->cur : 0);
    MM_CK(c, cudaGraphLaunch(c->graph[g], c->stream));
    c->launches += c->graph_nodes[g];
  }
  for (; i < n; ++i) {
    const int g = euler ? c->cur : 0;
    MM_CK(c, cudaGraphLaunch(c->graph[g], c->stream));
    c->launches += c->graph_nodes[g];
    if (euler) c->cur ^= 1;
  }
  c->steps += n;
  return MM_OK;
}

extern "C" int mm_step_timed(mm_ctx* c, int n, double dt, double ms_out[3]) {
  NvtxRange nvtx_("mm_step_timed");
  if (!c) return MM_EINVAL;
  if (!ms_out) return mm_fail(c, MM_EINVAL, "mm_step_timed: ms_out is NULL");
  if (n < 0) return mm_fail(c, MM_EINVAL, "mm_step_timed: n = %d < 0", n);
  if (!(dt > 0) || dt > 1e-6) return mm_fail(c, MM_EINVAL, "mm_step_timed: dt = %g s out of range", dt);
  const Phys ph = mm_make_phys(c);
  cudaEvent_t ev[13];
  for (int i = 0; i < 13; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
      return mm_fail(c, MM_ECUDA, "event creation failed");
    }
  int rc = MM_OK;
  if (!c->s_valid) {
    cudaEventRecord(ev[0], c->stream);
    rc = ensure_spectrum(c);
    cudaEventRecord(ev[1], c->stream);
    if (rc == MM_OK && cudaEventSynchronize(ev[1]) == cudaSuccess) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[0], ev[1]);
      ms_out[0] += ms;
    }
  }
  for (int step = 0; step < n && rc == MM_OK; ++step) {
    StageArgs a = base_args(c);
    a.dt = (float)dt;
    int nst = 4;
    const float* in[4] = {c->m0, c->stA, c->stB, c->stA};
    float* outp[4] = {c->stA, c->stB, c->stA, c->m0};
    if (c->opts.integrator == MM_EULER) {
      nst = 1;
      a.mode = 2;
      in[0] = c->cur ? c->stA : c->m0;
      outp[0] = c->cur ? c->m0 : c->stA;
    } else {
      a.mode = 1;
      a.m0 = c->m0;
      a.acc = c->acc;
    }
    int ne = 0;
    int cls[12];
    cudaEventRecord(ev[ne++], c->stream);
    for (int s4 = 0; s4 < nst && rc == MM_OK; ++s4) {
      a.stage = s4;
      a.m_in = in[s4];
      a.m_out = outp[s4];
      stage_drive(c, a, s4, dt);
      for (int part = 1; part < 3; ++part) {
        NvtxRange pass_(part == 1 ? "y/z pass" : "x pass + update");
        const int nl = launch_field_part(c->d, ph, a, c->tw, c->S, c->Kh, c->dflag, c->stream, part);
        if (nl < 0) {
          rc = mm_fail(c, MM_ECUDA, "kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
          break;
        }
        c->launches += nl;
        cls[ne - 1] = part;
        cudaEventRecord(ev[ne++], c->stream);
      }
    }
    if (rc != MM_OK) break;
    if (cudaEventSynchronize(ev[ne - 1]) != cudaSuccess) {
      rc = mm_fail(c, MM_ECUDA, "step failed: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    for (int k = 1; k < ne; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[k - 1], ev[k]);
      ms_out[cls[k - 1]] += ms;
    }
    if (c->opts.integrator == MM_EULER) c->cur ^= 1;
    c->steps++;
  }
  for (int i = 0; i < 13; ++i) cudaEventDestroy(ev[i]);
  return rc;
}

static int check_flag(mm_ctx* c) {
  int h[4];
  MM_CK(c, cudaMemcpyAsync(h, c->dflag, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  MM_CK(c, cudaStreamSynchronize(c->stream));
  if (h[0] || h[1] || h[2]) {
    cudaMemsetAsync(c->dflag, 0, sizeof(int) * 4, c->stream);
    if (h[2]) return mm_fail(c, MM_EBOUNDS, "bounds check: a kernel index was out of range (access skipped)");
    if (h[1]) return mm_fail(c, MM_ETIMEOUT, "a bounded wait inside a kernel gave up (bulk copy did not complete)");
    return mm_fail(c, MM_ENONFINITE, "non-finite or zero magnetisation vector found");
  }
  return MM_OK;
}

static int run_reduce(mm_ctx* c, double* host) {
  StageArgs a = base_args(c);
  a.m_in = state_ptr(c);
  a.H_out = c->Hs;
  a.mode = 0;
  a.mask = MM_TERM_DEMAG;
  const Phys ph = mm_make_phys(c);
  int k = launch_field_eval(c->d, ph, a, c->tw, c->S, c->Kh, c->dflag, c->stream);
  c->s_valid = 0;
  if (k < 0) return mm_fail(c, MM_ECUDA, "field kernels failed to launch");
  c->launches += k;
  k = launch_reduce(c->d, ph, drive_slot(c, 4), state_ptr(c), c->Hs, c->hmap, c->kumap, c->A, c->Ku, c->delta, c->Ms, c->red,
                    c->red_blocks, c->red_out, c->dflag, c->stream);
  if (k < 0) return mm_fail(c, MM_ECUDA, "reduction kernels failed to launch");
  c->launches += k;
  MM_CK(c, cudaMemcpyAsync(host, c->red_out, sizeof(double) * 9, cudaMemcpyDeviceToHost, c->stream));
  return check_flag(c);
}

extern "C" int mm_energy(mm_ctx* c, double E[5]) {
  NvtxRange nvtx_("mm_energy");
  if (!c) return MM_EINVAL;
  if (!E) return mm_fail(c, MM_EINVAL, "mm_energy: E is NULL");
  double r[9];
  const int rc = run_reduce(c, r);
  if (rc != MM_OK) return rc;
  E[0] = r[0]; E[1] = r[1]; E[2] = r[2]; E[3] = r[3];
  E[4] = r[0] + r[1] + r[2] + r[3];
  return MM_OK;
}

extern "C" int mm_observables(mm_ctx* c, double out[5]) {
  NvtxRange nvtx_("mm_observables");
  if (!c) return MM_EINVAL;
  if (!out) return mm_fail(c, MM_EINVAL, "mm_observables: out is NULL");
  double r[9];
  const int rc = run_reduce(c, r);
  if (rc != MM_OK) return rc;
  out[0] = r[4]; out[1] = r[5]; out[2] = r[6]; out[3] = r[7];
  out[4] = (double)c->steps;
  return MM_OK;
}

extern "C" long long mm_launch_count(const mm_ctx* c) { return c ? c->launches : -1; }

extern "C" int mm_build_flags(void) {
#ifdef MM_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

extern "C" int mm_sync(mm_ctx* c) {
  if (!c) return MM_EINVAL;
  MM_CK(c, cudaStreamSynchronize(c->stream));
  return check_flag(c);
}

extern "C" const char* mm_last_error(const mm_ctx* c) { return c ? c->err : g_create_err; }

// ---------------------------------------------------------------------------
// Self-test of the bounded device waits: one CTA waits on an mbarrier phase that
// nothing completes, gives up after `polls` polls, sets the context's timeout
// flag and returns; mm_sync then reports MM_ETIMEOUT.  No fault, no trap, no hang.
// ---------------------------------------------------------------------------
__global__ void k_wait_selftest(int* flag, unsigned polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1) : "memory");
  for (unsigned i = 0; i < polls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(0u)
        : "memory");
    if (ok) return;   // never: no thread arrives on the barrier
  }
  atomicOr(flag + 1, 1);
}

extern "C" int mm_selftest_wait_timeout(mm_ctx* c, unsigned polls) {
  if (polls < 1 || polls > (1u << 20))
    return c ? mm_fail(c, MM_EINVAL, "mm_selftest_wait_timeout: polls out of range") : MM_EINVAL;
  if (!c) {   // the flags of mm_heff_noalloc's scratch on the current device
    unsigned char* base = nullptr;
    if (int rc = mm_noalloc_scratch(&base)) return rc;
    k_wait_selftest<<<1, 32, 0, 0>>>((int*)base, polls);
    return cudaGetLastError() == cudaSuccess ? MM_OK : MM_ECUDA;
  }
  k_wait_selftest<<<1, 32, 0, c->stream>>>(c->dflag, polls);
  if (cudaGetLastError() != cudaSuccess) return mm_fail(c, MM_ECUDA, "self-test launch failed");
  c->launches++;
  return MM_OK;
}

extern "C" int mm_set_tuning(mm_ctx* c, int yz_route, int zt_block) {
  if (!c) return MM_EINVAL;
  if (yz_route < 0 || yz_route > 2) return mm_fail(c, MM_EINVAL, "mm_set_tuning: yz_route %d outside 0..2", yz_route);
  if (zt_block < 0 || (zt_block > 0 && zt_block < 8))
    return mm_fail(c, MM_EINVAL, "mm_set_tuning: zt_block %d (0 or >= 8)", zt_block);
  if (yz_route == 1 && !mm_yz_fits(c->d))
    return mm_fail(c, MM_EUNSUPPORTED, "mm_set_tuning: a kx column does not fit one CTA (no fused route)");
  if (yz_route == 2 && c->d.prec != MM_FP32)
    return mm_fail(c, MM_EUNSUPPORTED, "mm_set_tuning: the split precisions run the fused route only");
  Dims d = c->d;
  d.route = yz_route;
  d.ztkb = zt_block;
  if (!mm_yz_fused(d) && !c->T) {   // the split pass needs its buffer
    if (cudaMalloc(&c->T, sizeof(float2) * (size_t)d.hx * 3 * d.nz * d.py) != cudaSuccess) {
      cudaGetLastError();
      return mm_fail(c, MM_ENOMEM, "mm_set_tuning: cannot allocate the split-pass buffer");
    }
  }
  d.T = c->T;
  c->d = d;
  c->graph_valid = 0;   // the step's launches change
  c->param_gen++;
  return MM_OK;
}

extern "C" int mm_get_tuning(const mm_ctx* c, int* yz_route, int* zt_block) {
  if (!c || !yz_route || !zt_block) return MM_EINVAL;
  *yz_route = mm_yz_fused(c->d) ? 1 : 2;
  *zt_block = mm_zt_kb(c->d);
  return MM_OK;
}

extern "C" int mm_get_series(mm_ctx* c, double* out, int max_records, int* n_records) {
  if (!c) return MM_EINVAL;
  if (!n_records || (max_records > 0 && !out)) return mm_fail(c, MM_EINVAL, "mm_get_series: NULL output");
  *n_records = 0;
  if (!c->series) return mm_fail(c, MM_EINVAL, "mm_get_series: the context was created with obs_every = 0");
  long long nstep = 0;
  MM_CK(c, cudaMemcpyAsync(&nstep, &c->prog->nstep, sizeof nstep, cudaMemcpyDeviceToHost, c->stream));
  MM_CK(c, cudaStreamSynchronize(c->stream));
  const long long total = nstep / c->opts.obs_every;   // records written since mm_set_m
  const long long avail = total < c->series_cap ? total : c->series_cap;
  const long long n = avail < max_records ? avail : (max_records > 0 ? max_records : 0);
  if (n == 0) return MM_OK;
  std::vector<double> ring(6 * (size_t)c->series_cap);
  MM_CK(c, cudaMemcpy(ring.data(), c->series, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost));
  // the n most recent records, oldest first
  for (long long i = 0; i < n; ++i) {
    const long long rec = total - n + i;
    memcpy(out + 6 * i, ring.data() + 6 * (rec % c->series_cap), 6 * sizeof(double));
  }
  *n_records = (int)n;
  return MM_OK;
}
