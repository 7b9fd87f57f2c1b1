// The persistent batched kernel: one launch advances every film of a batch by
// whole RK4 steps.  Each CTA repeatedly takes the next item of a work queue
// (atomic counter) -- a y/z column or an x tile of one film at one stage --
// waits until that film has finished all its earlier items (a per-film
// counter; bounded polls, after which the wait sets the error flag and the
// item and every later one of a failed launch are skipped), runs the item
// with the single-film bodies, and counts it done.  Items are taken in queue
// order (all y/z columns of a stage, then all x tiles of it, film by film), so
// a CTA only ever waits for items that running CTAs have already taken: the
// queue always progresses, with no co-residency assumption.  Films of
// different sizes share the SMs inside the launch: no group waits for another.
//
// Data that another CTA of the launch wrote is read through L2 (the PC
// instances of the bodies), and the bodies keep to plain loads and stores,
// ordered by the counters (release: fence + atomic add; acquire: the polling
// load + fence).
#include "field_kernels.cuh"

static constexpr int kPersistThreads = 256;
static constexpr int kPersistNZM = 4;   // films of 1..4 planes (planes beyond nz enter the z product as zeros)

int persist_supported(const Dims& d) {
  const bool px_ok = d.px == 32 || d.px == 64 || d.px == 128 || d.px == 256 || d.px == 512;
  const bool py_ok = d.py == 16 || d.py == 32 || d.py == 64 || d.py == 128 || d.py == 256;
  return px_ok && py_ok && d.nz <= kPersistNZM && d.prec == 0;
}

int persist_x_tiles(const Dims& d) {
  const int ty = x_tile(d.px / 2);
  return d.nz * ((d.ny + ty - 1) / ty);
}

// the same on the device (rows per tile: XTile, 8 up to px = 512)
__device__ __forceinline__ int persist_x_tiles_dev(const Dims& d) { return d.nz * ((d.ny + 7) / 8); }

static size_t persist_smem() {
  size_t m = x_smem(256);
  Dims d = {};
  d.py = 256;
  d.nz = kPersistNZM;
  const size_t y = yz_smem(d);
  return m > y ? m : y;
}

__device__ __forceinline__ int find_film(const int* __restrict__ off, int nf, int local) {
  int lo = 0, hi = nf - 1;   // the last f with off[f] <= local
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= local) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int HALF>
__device__ __forceinline__ void persist_x(const BatchFilm& f, int tile, int stage, float dt) {
  constexpr int TY = XTile<HALF>::v;
  const int ntyl = (f.d.ny + TY - 1) / TY;
  StageArgs a = {};
  a.mode = 1;
  a.stage = stage;
  a.dt = dt;
  a.m0 = f.m0;
  a.acc = f.acc;
  a.hmap = f.hmap;
  a.kumap = f.kumap;
  a.m_in = stage == 0 ? f.m0 : (stage == 2 ? f.stB : f.stA);
  a.m_out = stage == 0 ? f.stA : (stage == 1 ? f.stB : (stage == 2 ? f.stA : f.m0));
  a.maxdmdt = stage == 0 ? f.maxdmdt : nullptr;
  body_x<HALF, TY, false, true>(a, f.ph, f.S, f.tw + 2 * HALF, f.d, TY, 1, tile / ntyl, (tile % ntyl) * TY);
}

template <int PY>
__device__ __forceinline__ void persist_yz(const BatchFilm& f, int kx, int* flag) {
  body_yz<PY, kPersistNZM, 0, true>(f.S, f.Kh, f.tw + PY, f.d, flag, kx);
}

__global__ void __launch_bounds__(kPersistThreads, 2) kb_persist(PersistPlan P) {
  __shared__ int s_item, s_ok;
  MM_BC_ENTER(P.flag);
  const int per = P.n_yz + P.n_x;   // items of one stage, both passes
  const int total = per * 4 * P.nsteps;
  for (;;) {
    __syncthreads();   // the previous item is done with shared memory and s_item
    if (threadIdx.x == 0) s_item = atomicAdd(P.next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) return;
    const int q = item / per, r = item % per;   // q: stage of the launch
    const int pass = r >= P.n_yz;                // 0: y/z columns, 1: x tiles
    const int local = pass ? r - P.n_yz : r;
    const int* off = pass ? P.x_off : P.yz_off;
    const int fi = find_film(off, P.nf, local);
    const int j = local - __ldg(off + fi);      // the film's j-th item of this pass
    const BatchFilm& f = P.F[fi];
    const int hxf = __ldg(P.yz_off + fi + 1) - __ldg(P.yz_off + fi);
    const int ntf = __ldg(P.x_off + fi + 1) - __ldg(P.x_off + fi);
    const bool active = f.active != 0;
    if (threadIdx.x == 0) {
      // every earlier item of this film: q whole stages, plus this stage's columns for an x tile
      unsigned need = (unsigned)q * (unsigned)(hxf + ntf) + (pass ? (unsigned)hxf : 0u);
      if (fi == P.blocked_film) need += 0x40000000u;
      int ok = 1;
      if (active && need > 0) {
        for (unsigned polls = 0; ld_acquire_u32(P.done + fi) < need; ++polls) {
          if (*(volatile int*)(P.flag + 1)) { ok = 0; break; }   // the launch has failed: skip
          if (polls >= P.spin_limit) {
            atomicOr(P.flag + 1, 1);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    if (!active || !s_ok) continue;
    if (!P.dry) {
      if (pass == 0) {
        const int c1 = min((j + 1) * P.gyz, f.d.hx);
        for (int tile = j * P.gyz; tile < c1; ++tile) {
          if (tile > j * P.gyz) __syncthreads();   // the last column is out of shared memory
          switch (f.d.py) {
            case 16: persist_yz<16>(f, tile, P.flag); break;
            case 32: persist_yz<32>(f, tile, P.flag); break;
            case 64: persist_yz<64>(f, tile, P.flag); break;
            case 128: persist_yz<128>(f, tile, P.flag); break;
            case 256: persist_yz<256>(f, tile, P.flag); break;
          }
        }
      } else {
        const int stage = q & 3;
        const int t1 = min((j + 1) * P.gx, persist_x_tiles_dev(f.d));
        for (int tile = j * P.gx; tile < t1; ++tile) {
          if (tile > j * P.gx) __syncthreads();
          switch (f.d.px) {
            case 32: persist_x<16>(f, tile, stage, P.dt); break;
            case 64: persist_x<32>(f, tile, stage, P.dt); break;
            case 128: persist_x<64>(f, tile, stage, P.dt); break;
            case 256: persist_x<128>(f, tile, stage, P.dt); break;
            case 512: persist_x<256>(f, tile, stage, P.dt); break;
          }
        }
      }
    }
    __syncthreads();   // every thread's writes of the item precede the count
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(P.done + fi, 1u);
    }
  }
}

int launch_persist(const PersistPlan& p, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(kb_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)persist_smem()) !=
        cudaSuccess)
      return -1;
    attr = true;
  }
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_persist, kPersistThreads, persist_smem()) !=
          cudaSuccess)
    return -1;
  if (per_sm < 1) per_sm = 1;
  kb_persist<<<sms * per_sm, kPersistThreads, persist_smem(), s>>>(p);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}
