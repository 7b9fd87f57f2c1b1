// Field program entry points (mm_set_program, mm_set_time, mm_get_time) and
// the stream-ordered writes of the context's base field and damping.  Every
// write is a single-CTA kernel on the context's stream, so it is ordered with
// the captured step graph without invalidating it.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "program.cuh"

namespace {

struct ProgUpload {   // kernel parameter (< 4 KB)
  int nseg;
  ProgSeg seg[MM_PROGRAM_MAX];
};

__device__ void refresh_now(ProgState* p) { prog_eval(p, p->clock, p->drive[4]); }

__global__ void k_prog_init(ProgState* p, Phys ph) {
  if (threadIdx.x != 0) return;
  p->clock = 0.0;
  p->nstep = 0;
  p->maxdmdt = 0.f;
  p->nseg = 0;
  const float b[5] = {ph.bx, ph.by, ph.bz, ph.g1, ph.g2};
  for (int c = 0; c < 8; ++c) p->base[c] = c < 5 ? b[c] : 0.f;
  for (int s = 0; s < 5; ++s)
    for (int c = 0; c < 8; ++c) p->drive[s][c] = c < 5 ? b[c] : 0.f;
}

// New base values; every drive slot is refreshed so that a stage kernel that
// runs before the next tick (mm_heff, the adjoint's recomputation) sees them.
__global__ void k_prog_base(ProgState* p, Phys ph) {
  if (threadIdx.x != 0) return;
  const float b[5] = {ph.bx, ph.by, ph.bz, ph.g1, ph.g2};
  for (int c = 0; c < 5; ++c) p->base[c] = b[c];
  for (int s = 0; s < 4; ++s) prog_eval(p, p->clock, p->drive[s]);
  refresh_now(p);
}

__global__ void k_prog_set(ProgState* p, ProgUpload u) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < u.nseg; ++i) p->seg[i] = u.seg[i];
  p->nseg = u.nseg;
  for (int s = 0; s < 4; ++s) prog_eval(p, p->clock, p->drive[s]);
  refresh_now(p);
}

__global__ void k_prog_clock(ProgState* p, double t) {
  if (threadIdx.x != 0) return;
  p->clock = t;
  for (int s = 0; s < 4; ++s) prog_eval(p, p->clock, p->drive[s]);
  refresh_now(p);
}

void g_of(double gamma, double alpha, float* g1, float* g2) {
  const double g = gamma / (1.0 + alpha * alpha);
  *g1 = (float)(-g);
  *g2 = (float)(-alpha * g);
}

}  // namespace

// Observables record (obs_every > 0), one launch per step after the step's
// kernels: on every obs_every-th step, <m> of the new state (FP64 block sums,
// atomically added into a record the previous record zeroed), the clock, the
// step count and max |dm/dt| at the step's start (recorded by its first stage);
// max |dm/dt| is reset every step.  Off-cadence steps return at once.
__global__ void __launch_bounds__(256) k_record(const float* __restrict__ m, long long N, ProgState* p,
                                                double* series, int cap, int every) {
  const long long n = p->nstep;
  const bool rec_step = n > 0 && n % every == 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && !rec_step) p->maxdmdt = 0.f;
  if (!rec_step) return;
  const long long rec = n / every - 1;
  double* r = series + (rec % cap) * 6;
  double s[3] = {0.0, 0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    s[0] += m[i]; s[1] += m[i + N]; s[2] += m[i + 2 * N];
  }
  __shared__ double red[3][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double v = s[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[c][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[threadIdx.x][k];
    atomicAdd(r + 2 + threadIdx.x, v / (double)N);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    r[0] = p->clock;
    r[1] = (double)n;
    r[5] = (double)p->maxdmdt;
    p->maxdmdt = 0.f;
    double* nx = series + ((rec + 1) % cap) * 6;   // the next record accumulates from zero
    for (int k = 0; k < 6; ++k) nx[k] = 0.0;
  }
}

int launch_record(mm_ctx* c, const float* m, cudaStream_t s) {
  const long long N = c->d.N;
  int nb = (int)((N + 255) / 256);
  if (nb > 296) nb = 296;
  k_record<<<nb, 256, 0, s>>>(m, N, c->prog, c->series, c->series_cap, c->opts.obs_every);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int mm_prog_init(mm_ctx* c) {
  k_prog_init<<<1, 32, 0, c->stream>>>(c->prog, mm_make_phys(c));
  MM_CK(c, cudaGetLastError());
  c->launches++;
  return MM_OK;
}

int mm_prog_push_base(mm_ctx* c) {
  k_prog_base<<<1, 32, 0, c->stream>>>(c->prog, mm_make_phys(c));
  MM_CK(c, cudaGetLastError());
  c->launches++;
  return MM_OK;
}

extern "C" int mm_set_program(mm_ctx* c, int nseg, const mm_segment* seg) {
  if (!c) return MM_EINVAL;
  if (nseg < 0 || nseg > MM_PROGRAM_MAX)
    return mm_fail(c, MM_EINVAL, "mm_set_program: nseg = %d outside 0..%d", nseg, MM_PROGRAM_MAX);
  if (nseg > 0 && !seg) return mm_fail(c, MM_EINVAL, "mm_set_program: seg is NULL");
  ProgUpload u;
  memset(&u, 0, sizeof u);
  u.nseg = nseg;
  for (int i = 0; i < nseg; ++i) {
    const mm_segment& s = seg[i];
    bool ok = isfinite(s.t_begin) && isfinite(s.t_end) && s.t_end > s.t_begin && isfinite(s.alpha);
    for (int k = 0; k < 3; ++k) ok = ok && isfinite(s.b_begin[k]) && isfinite(s.b_end[k]);
    if (!ok) return mm_fail(c, MM_EINVAL, "mm_set_program: segment %d is not finite or has t_end <= t_begin", i);
    ProgSeg& d = u.seg[i];
    d.t0 = s.t_begin;
    d.t1 = s.t_end;
    for (int k = 0; k < 3; ++k) {
      d.b0[k] = (float)s.b_begin[k];
      d.b1[k] = (float)s.b_end[k];
    }
    d.own_g = s.alpha >= 0.0;
    if (d.own_g) g_of(c->gamma, s.alpha, &d.g1, &d.g2);
  }
  k_prog_set<<<1, 32, 0, c->stream>>>(c->prog, u);
  MM_CK(c, cudaGetLastError());
  c->launches++;
  c->prog_n = nseg;
  c->graph_valid = 0;   // the stage kernels switch between parameter and drive-slot inputs
  c->param_gen++;
  return MM_OK;
}

extern "C" int mm_set_time(mm_ctx* c, double t) {
  if (!c) return MM_EINVAL;
  if (!isfinite(t)) return mm_fail(c, MM_EINVAL, "mm_set_time: t is not finite");
  k_prog_clock<<<1, 32, 0, c->stream>>>(c->prog, t);
  MM_CK(c, cudaGetLastError());
  c->launches++;
  return MM_OK;
}

extern "C" int mm_get_time(mm_ctx* c, double* t) {
  if (!c) return MM_EINVAL;
  if (!t) return mm_fail(c, MM_EINVAL, "mm_get_time: t is NULL");
  MM_CK(c, cudaMemcpyAsync(t, &c->prog->clock, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MM_CK(c, cudaStreamSynchronize(c->stream));
  return MM_OK;
}
