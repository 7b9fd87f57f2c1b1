// Device-side evaluation of the field program (ProgState, common.cuh): the
// uniform applied field and the LLG prefactors at a time t, and the per-step
// tick that advances the clock and fills the drive slots the stages read.
#pragma once
#include "common.cuh"

// out[0..2] = mu0 H_ext (T), out[3..4] = g1, g2 at time t: the first segment
// with t0 <= t < t1, linear in t between its end values; the base outside.
static __device__ __forceinline__ void prog_eval(const ProgState* p, double t, float* out) {
  float v[5] = {p->base[0], p->base[1], p->base[2], p->base[3], p->base[4]};
  const int n = p->nseg;
  for (int i = 0; i < n; ++i) {
    const ProgSeg& s = p->seg[i];
    if (t >= s.t0 && t < s.t1) {
      const double f = (t - s.t0) / (s.t1 - s.t0);
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c] = (float)((double)s.b0[c] + f * ((double)s.b1[c] - (double)s.b0[c]));
      if (s.own_g) { v[3] = s.g1; v[4] = s.g2; }
      break;
    }
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) out[c] = v[c];
}

// Called by one full warp: lanes 0..3 fill the stage slots of the step that
// starts at the clock t (RK4 stage times t, t + dt/2, t + dt/2, t + dt; Euler
// uses slot 0 at t), lane 4 the slot of the end of the step; then the clock
// becomes t + dt.
static __device__ __noinline__ void prog_tick(const Tick tk) {
  const int lane = threadIdx.x & 31;
  ProgState* p = tk.p;
  const double t = p->clock;
  if (lane < 5) {
    const double c = lane == 4 ? 1.0 : (tk.euler ? 0.0 : (lane == 0 ? 0.0 : (lane == 3 ? 1.0 : 0.5)));
    prog_eval(p, t + c * tk.dt, p->drive[lane]);
  }
  __syncwarp();
  if (lane == 0) {
    p->clock = t + tk.dt;
    p->nstep += 1;
  }
}
