// Many independent films of uneven size advanced together (a field sweep: one
// film per applied field).  Every film has its own context (its buffers,
// transformed tensor and twiddles); the batch groups the films by padded sizes
// (px, py) and z-product width, and one RK4 step becomes, per group, four
// stages of two batched launches (k_yz, k_x over all films of the group).  The
// groups are independent, so one step is captured as a CUDA graph with one
// parallel branch per group.  A film whose max |dm/dt| (recorded by the first
// stage of every step) falls below a tolerance can be switched off: its CTAs
// return at once.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "common.cuh"

struct BatchGroup {
  int px, py, nzm;
  std::vector<int> films;
  int2 *map_xf = nullptr, *map_yz = nullptr, *map_x = nullptr;
  int n_xf = 0, n_yz = 0, n_x = 0;
  size_t smem_yz = 0;
};

struct mm_batch {
  int nf = 0;
  std::vector<mm_ctx*> film;
  std::vector<BatchFilm> host;
  BatchFilm* dev = nullptr;
  float* maxdmdt = nullptr;   // [nf]
  int* flag = nullptr;        // kernel wait flags
  std::vector<BatchGroup> groups;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> side;   // capture branches (one per group)
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0;
  long long launches = 0;
  long long graph_nodes = 0;
  char err[512] = "";
};

static char g_batch_err[512] = "";

static int bfail(mm_batch* b, int code, const char* fmt, ...) {
  char* dst = b ? b->err : g_batch_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

#define BCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return bfail(b, MM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static void free_batch(mm_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto& g : b->groups) {
    cudaFree(g.map_xf);
    cudaFree(g.map_yz);
    cudaFree(g.map_x);
  }
  cudaFree(b->dev);
  cudaFree(b->maxdmdt);
  cudaFree(b->flag);
  for (auto s : b->side) cudaStreamDestroy(s);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto c : b->film) mm_destroy(c);
  delete b;
}

extern "C" void mm_batch_destroy(mm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

static int pow2_up(int v) {
  int p = 1;
  while (p < v) p *= 2;
  return p;
}

extern "C" int mm_batch_create(mm_batch** out, int nfilms, const int* grids, double delta, double Ms, double A,
                               double Ku, double alpha, double gamma, const mm_opts* opts) {
  if (!out) return bfail(nullptr, MM_EINVAL, "out is NULL");
  *out = nullptr;
  if (nfilms < 1 || !grids) return bfail(nullptr, MM_EINVAL, "need nfilms >= 1 and a grid list");
  mm_opts o;
  mm_default_opts(&o);
  if (opts) o = *opts;
  if (o.integrator != MM_RK4) return bfail(nullptr, MM_EUNSUPPORTED, "batches run RK4 only");
  if (o.precision != MM_FP32) return bfail(nullptr, MM_EUNSUPPORTED, "batches run the FP32 path only");
  for (int f = 0; f < nfilms; ++f)
    if (grids[3 * f + 2] > 16)
      return bfail(nullptr, MM_EUNSUPPORTED, "film %d: nz = %d; batched films have nz <= 16", f, grids[3 * f + 2]);
  mm_batch* b = new mm_batch();
  b->nf = nfilms;
  b->stream = (cudaStream_t)o.stream;
  int rc = MM_OK;
  for (int f = 0; f < nfilms; ++f) {
    mm_ctx* c = nullptr;
    rc = mm_create(&c, grids + 3 * f, delta, Ms, A, Ku, alpha, gamma, &o);
    if (rc != MM_OK) {
      bfail(nullptr, rc, "film %d: %s", f, mm_last_error(nullptr));
      free_batch(b);
      return rc;
    }
    b->film.push_back(c);
    if (!mm_yz_fused(c->d)) {
      free_batch(b);
      return bfail(nullptr, MM_EUNSUPPORTED, "film %d: its kx columns exceed one CTA (batched films need the fused y/z pass)", f);
    }
  }
  if (cudaMalloc(&b->dev, sizeof(BatchFilm) * nfilms) != cudaSuccess ||
      cudaMalloc(&b->maxdmdt, sizeof(float) * nfilms) != cudaSuccess ||
      cudaMalloc(&b->flag, sizeof(int) * 4) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return bfail(nullptr, MM_ENOMEM, "batch descriptors: allocation failed");
  }
  cudaMemset(b->maxdmdt, 0, sizeof(float) * nfilms);
  cudaMemset(b->flag, 0, sizeof(int) * 4);
  // groups by (px, py, z-product width); nz <= 4 share width 4 (planes beyond nz enter as zeros)
  std::map<std::tuple<int, int, int>, int> key;
  for (int f = 0; f < nfilms; ++f) {
    const Dims& d = b->film[f]->d;
    const int nzm = d.nz <= 4 ? 4 : pow2_up(d.nz);
    auto k = std::make_tuple(d.px, d.py, nzm);
    if (!key.count(k)) {
      key[k] = (int)b->groups.size();
      BatchGroup g;
      g.px = d.px; g.py = d.py; g.nzm = nzm;
      b->groups.push_back(g);
    }
    b->groups[key[k]].films.push_back(f);
  }
  for (auto& g : b->groups) {
    std::vector<int2> mxf, myz, mx;
    const int tyf = x_batch_tile(g.px, 0), tyx = x_batch_tile(g.px, 2);
    for (int f : g.films) {
      const Dims& d = b->film[f]->d;
      const int nxf = 3 * d.nz * ((d.ny + tyf - 1) / tyf), nx = d.nz * ((d.ny + tyx - 1) / tyx);
      for (int t = 0; t < nxf; ++t) mxf.push_back(make_int2(f, t));
      for (int t = 0; t < d.hx; ++t) myz.push_back(make_int2(f, t));
      for (int t = 0; t < nx; ++t) mx.push_back(make_int2(f, t));
      g.smem_yz = std::max(g.smem_yz, mm_yz_smem(d));
    }
    g.n_xf = (int)mxf.size(); g.n_yz = (int)myz.size(); g.n_x = (int)mx.size();
    if (cudaMalloc(&g.map_xf, sizeof(int2) * mxf.size()) != cudaSuccess ||
        cudaMalloc(&g.map_yz, sizeof(int2) * myz.size()) != cudaSuccess ||
        cudaMalloc(&g.map_x, sizeof(int2) * mx.size()) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return bfail(nullptr, MM_ENOMEM, "batch maps: allocation failed");
    }
    cudaMemcpy(g.map_xf, mxf.data(), sizeof(int2) * mxf.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(g.map_yz, myz.data(), sizeof(int2) * myz.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(g.map_x, mx.data(), sizeof(int2) * mx.size(), cudaMemcpyHostToDevice);
  }
  b->host.resize(nfilms);
  b->side.resize(b->groups.size());
  b->join.resize(b->groups.size());
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (size_t g = 0; g < b->groups.size() && ok; ++g)
    ok = cudaStreamCreateWithFlags(&b->side[g], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[g], cudaEventDisableTiming) == cudaSuccess;
  if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return bfail(nullptr, MM_ECUDA, "batch set-up failed");
  }
  *out = b;
  return MM_OK;
}

extern "C" mm_ctx* mm_batch_film(mm_batch* b, int f) {
  if (!b || f < 0 || f >= b->nf) return nullptr;
  return b->film[f];
}

extern "C" int mm_batch_group_count(const mm_batch* b) { return b ? (int)b->groups.size() : -1; }
extern "C" long long mm_batch_launch_count(const mm_batch* b) { return b ? b->launches : -1; }
extern "C" const char* mm_batch_last_error(const mm_batch* b) { return b ? b->err : g_batch_err; }

// Refresh the device descriptors from the film contexts (fields, maps, active flags).
static int sync_descriptors(mm_batch* b, const std::vector<int>* active) {  // active: one flag per film
  for (int f = 0; f < b->nf; ++f) {
    mm_ctx* c = b->film[f];
    BatchFilm& h = b->host[f];
    h.d = c->d;
    h.ph = mm_make_phys(c);
    h.m0 = c->m0; h.stA = c->stA; h.stB = c->stB; h.acc = c->acc;
    h.hmap = c->hmap; h.kumap = c->kumap;
    h.S = c->S; h.Kh = c->Kh; h.tw = c->tw;
    h.maxdmdt = b->maxdmdt + f;
    h.active = (*active)[f];
  }
  BCK(cudaMemcpyAsync(b->dev, b->host.data(), sizeof(BatchFilm) * b->nf,
                                          cudaMemcpyHostToDevice, b->stream));
  return MM_OK;
}

// S of every film must hold the x transform of its state before a step.
static int ensure_spectra(mm_batch* b) {
  bool all = true;
  for (auto c : b->film) all = all && c->s_valid;
  if (all) return MM_OK;
  for (auto& g : b->groups) {
    if (launch_batch(b->dev, g.px, g.py, g.nzm, g.map_xf, g.n_xf, g.smem_yz, 0, 0, 0.f, b->flag, b->stream) < 0)
      return bfail(b, MM_ECUDA, "batched x-transform launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    b->launches++;
  }
  for (auto c : b->film) c->s_valid = 1;
  return MM_OK;
}

static int enqueue_group_step(mm_batch* b, const BatchGroup& g, cudaStream_t s, float dt, long long* nk) {
  for (int st = 0; st < 4; ++st) {
    if (launch_batch(b->dev, g.px, g.py, g.nzm, g.map_yz, g.n_yz, g.smem_yz, 1, st, dt, b->flag, s) < 0) return -1;
    if (launch_batch(b->dev, g.px, g.py, g.nzm, g.map_x, g.n_x, g.smem_yz, 2, st, dt, b->flag, s) < 0) return -1;
    *nk += 2;
  }
  return 0;
}

static int build_graph(mm_batch* b, double dt) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaStream_t cap = b->side[0];
  cudaGraph_t graph;
  long long nk = 0;
  BCK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  int r = cudaEventRecord(b->fork, cap) == cudaSuccess ? 0 : -1;
  for (size_t g = 1; g < b->groups.size() && r == 0; ++g)
    r = cudaStreamWaitEvent(b->side[g], b->fork, 0) == cudaSuccess ? 0 : -1;
  for (size_t g = 0; g < b->groups.size() && r == 0; ++g) r = enqueue_group_step(b, b->groups[g], b->side[g], (float)dt, &nk);
  for (size_t g = 1; g < b->groups.size() && r == 0; ++g) {
    r = cudaEventRecord(b->join[g], b->side[g]) == cudaSuccess ? 0 : -1;
    if (r == 0) r = cudaStreamWaitEvent(cap, b->join[g], 0) == cudaSuccess ? 0 : -1;
  }
  cudaError_t e = cudaStreamEndCapture(cap, &graph);
  if (r != 0 || e != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, MM_ECUDA, "batch graph capture failed (%s)", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&b->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(b, MM_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
  b->graph_dt = dt;
  b->graph_nodes = nk;
  return MM_OK;
}

static int run_steps(mm_batch* b, int n, double dt) {
  if (!b->graph || b->graph_dt != dt) {
    const int r = build_graph(b, dt);
    if (r != MM_OK) return r;
  }
  int r = ensure_spectra(b);
  if (r != MM_OK) return r;
  for (int i = 0; i < n; ++i) {
    if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess)
      return bfail(b, MM_ECUDA, "batch graph launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    b->launches += b->graph_nodes;
  }
  for (auto c : b->film) c->steps += n;
  return MM_OK;
}

extern "C" int mm_batch_step(mm_batch* b, int n, double dt) {
  if (!b) return MM_EINVAL;
  if (n < 0) return bfail(b, MM_EINVAL, "mm_batch_step: n < 0");
  if (!(dt > 0) || dt > 1e-6) return bfail(b, MM_EINVAL, "mm_batch_step: dt = %g s out of range", dt);
  if (n == 0) return MM_OK;
  std::vector<int> all(b->nf, 1);
  int r = sync_descriptors(b, &all);
  if (r != MM_OK) return r;
  return run_steps(b, n, dt);
}

extern "C" int mm_batch_run(mm_batch* b, int max_steps, double dt, double tol_dmdt, int check_every,
                            int* steps_out) {
  if (!b) return MM_EINVAL;
  if (max_steps < 0 || check_every < 1) return bfail(b, MM_EINVAL, "mm_batch_run: need max_steps >= 0, check_every >= 1");
  if (!(dt > 0) || dt > 1e-6) return bfail(b, MM_EINVAL, "mm_batch_run: dt = %g s out of range", dt);
  std::vector<int> active(b->nf, 1), steps(b->nf, 0);
  std::vector<float> mx(b->nf);
  int r = MM_OK;
  int done = 0;
  while (done < max_steps) {
    const int chunk = std::min(check_every, max_steps - done);
    if ((r = sync_descriptors(b, &active)) != MM_OK) return r;
    if (chunk > 1 && (r = run_steps(b, chunk - 1, dt)) != MM_OK) return r;
    BCK(cudaMemsetAsync(b->maxdmdt, 0, sizeof(float) * b->nf, b->stream));
    if ((r = run_steps(b, 1, dt)) != MM_OK) return r;   // its first stage records |dm/dt| of the state
    BCK(cudaMemcpyAsync(mx.data(), b->maxdmdt, sizeof(float) * b->nf, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    done += chunk;
    int live = 0;
    for (int f = 0; f < b->nf; ++f) {
      if (!active[f]) continue;
      steps[f] += chunk;
      if (!(mx[f] >= tol_dmdt)) active[f] = 0;   // converged (or non-finite: stop it too)
      live += active[f];
    }
    if (!live) break;
  }
  std::vector<int> all(b->nf, 1);
  if ((r = sync_descriptors(b, &all)) != MM_OK) return r;
  for (int f = 0; f < b->nf; ++f) b->film[f]->steps = steps[f];
  if (steps_out) memcpy(steps_out, steps.data(), sizeof(int) * b->nf);
  return MM_OK;
}

extern "C" int mm_batch_max_dmdt(mm_batch* b, float* out) {
  if (!b || !out) return MM_EINVAL;
  BCK(cudaMemcpyAsync(out, b->maxdmdt, sizeof(float) * b->nf, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return MM_OK;
}
