// Many independent films of uneven size advanced together (a field sweep: one
// film per applied field).  Every film has its own context (its buffers,
// transformed tensor and twiddles).  Two schedules of a step:
//   persistent (the default when every film has a body in it): one launch of
//     kb_persist (field_inst_persist.cu) per RK4 step, whose CTAs take the y/z
//     columns and x tiles of all films from one work queue, each item waiting
//     on its own film's progress counter only;
//   grouped: the films are grouped by padded sizes (px, py) and z-product
//     width, and a step is, per group, four stages of two batched launches
//     (kb_yz, kb_x over the films of the group), one parallel graph branch per
//     group.
// Either way a step is replayed from a captured CUDA graph.  A film whose max
// |dm/dt| (recorded by the first stage of every step) falls below a tolerance
// can be switched off: its work is skipped.
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
  int schedule = 0;               // 1 persistent, 0 grouped
  int persist_ok = 0;             // every film has a body in the persistent kernel
  int* yz_off = nullptr;          // persistent plan: prefix sums of kx columns / x tiles (device)
  int* x_off = nullptr;
  int n_yz = 0, n_x = 0;
  int* next = nullptr;            // work counter, then per-film done counters (device)
  unsigned* done = nullptr;
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
  cudaFree(b->yz_off);
  cudaFree(b->x_off);
  cudaFree(b->next);
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
  // the persistent plan: item offsets of every film (y/z columns, x tiles)
  b->persist_ok = 1;
  for (int f = 0; f < nfilms; ++f) b->persist_ok = b->persist_ok && persist_supported(b->film[f]->d);
  if (b->persist_ok) {
    std::vector<int> yo(nfilms + 1, 0), xo(nfilms + 1, 0);
    for (int f = 0; f < nfilms; ++f) {
      yo[f + 1] = yo[f] + (b->film[f]->d.hx + kPersistGYZ - 1) / kPersistGYZ;
      xo[f + 1] = xo[f] + (persist_x_tiles(b->film[f]->d) + kPersistGX - 1) / kPersistGX;
    }
    b->n_yz = yo[nfilms];
    b->n_x = xo[nfilms];
    if (cudaMalloc(&b->yz_off, sizeof(int) * yo.size()) != cudaSuccess ||
        cudaMalloc(&b->x_off, sizeof(int) * xo.size()) != cudaSuccess ||
        cudaMalloc(&b->next, sizeof(int) * (1 + (size_t)nfilms)) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return bfail(nullptr, MM_ENOMEM, "persistent plan: allocation failed");
    }
    b->done = reinterpret_cast<unsigned*>(b->next + 1);
    cudaMemcpy(b->yz_off, yo.data(), sizeof(int) * yo.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(b->x_off, xo.data(), sizeof(int) * xo.size(), cudaMemcpyHostToDevice);
  }
  b->schedule = b->persist_ok;
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

static PersistPlan persist_plan(mm_batch* b, double dt, int nsteps) {
  PersistPlan p;
  p.F = b->dev;
  p.yz_off = b->yz_off;
  p.x_off = b->x_off;
  p.nf = b->nf;
  p.n_yz = b->n_yz;
  p.n_x = b->n_x;
  p.gyz = kPersistGYZ;
  p.gx = kPersistGX;
  p.nsteps = nsteps;
  p.next = b->next;
  p.done = b->done;
  p.flag = b->flag;
  p.spin_limit = 1u << 26;   // about a second of polls (64 ns naps) before a wait gives up
  p.blocked_film = -1;
  p.dry = 0;
  p.dt = (float)dt;
  return p;
}

// One persistent launch (counters cleared first): 3 graph nodes per step.
static int enqueue_persist(mm_batch* b, const PersistPlan& p, cudaStream_t s) {
  if (cudaMemsetAsync(b->next, 0, sizeof(int) * (1 + (size_t)b->nf), s) != cudaSuccess) return -1;
  return launch_persist(p, s) < 0 ? -1 : 0;
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
  if (b->schedule) {   // persistent: one kernel for every film's step
    const int r = enqueue_persist(b, persist_plan(b, dt, 1), cap);
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    if (r != 0 || e != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, MM_ECUDA, "batch graph capture failed (%s)", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, MM_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
    b->graph_dt = dt;
    b->graph_nodes = 1;
    return MM_OK;
  }
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

extern "C" int mm_batch_set_schedule(mm_batch* b, int persistent) {
  if (!b) return MM_EINVAL;
  if (persistent != 0 && persistent != 1) return bfail(b, MM_EINVAL, "mm_batch_set_schedule: 0 or 1");
  if (persistent && !b->persist_ok)
    return bfail(b, MM_EUNSUPPORTED, "the persistent kernel has no body for some film of this batch "
                                     "(px 32..512, py 16..256, nz <= 4)");
  if (persistent != b->schedule) {
    b->schedule = persistent;
    if (b->graph) {
      cudaStreamSynchronize(b->stream);
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  return MM_OK;
}

extern "C" int mm_batch_get_schedule(const mm_batch* b) { return b ? b->schedule : -1; }

extern "C" int mm_batch_sync(mm_batch* b) {
  if (!b) return MM_EINVAL;
  int h[4];
  BCK(cudaMemcpyAsync(h, b->flag, sizeof h, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (h[0] || h[1]) {
    BCK(cudaMemsetAsync(b->flag, 0, sizeof h, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if (h[1]) return bfail(b, MM_ETIMEOUT, "a bounded wait inside a batched kernel gave up");
    return bfail(b, MM_ENONFINITE, "a batched kernel flagged a non-finite value");
  }
  return MM_OK;
}

extern "C" int mm_batch_selftest_wait_timeout(mm_batch* b, unsigned polls) {
  if (!b) return MM_EINVAL;
  if (!b->persist_ok) return bfail(b, MM_EUNSUPPORTED, "the self-test runs the persistent kernel");
  if (polls < 1 || polls > (1u << 20)) return bfail(b, MM_EINVAL, "mm_batch_selftest_wait_timeout: polls out of range");
  std::vector<int> all(b->nf, 1);
  int r = sync_descriptors(b, &all);
  if (r != MM_OK) return r;
  PersistPlan p = persist_plan(b, 1e-15, 1);
  p.blocked_film = 0;   // film 0's items wait for a count nothing reaches
  p.spin_limit = polls;
  p.dry = 1;            // no item does its work: the films keep their states
  if (enqueue_persist(b, p, b->stream) != 0)
    return bfail(b, MM_ECUDA, "self-test launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  b->launches++;
  return MM_OK;
}
