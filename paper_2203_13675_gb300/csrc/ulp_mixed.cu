// ulp_mixed.cu -- mixed-precision inner solve of Algorithm 1 (reliable-update PCG).
//
// The Krylov recurrence runs on FP32 planes: search direction d, A d, the
// residual r, the preconditioned residual s and the correction x gathered
// since the last refresh, with FP32 copies of the Eq. (UV) weights and the
// diagonal formed on the fly from them.  FP64 is kept where it decides the
// answer:
//   - the inner products behind alpha and beta are accumulated per lane as
//     double-float pairs (exact FP32 products, compensated sums) and summed
//     across lanes and tiles in FP64, so they are FP64-accurate;
//   - alpha, beta, delta and the stop tests are FP64 (the shared finisher);
//   - phi itself stays FP64: every refresh period (Algorithm 1's true-residual
//     step, every 20 iterations here) the FP32 correction is folded into phi
//     and r = b - A phi is recomputed with the FP64 weights and FP64 phi.
// Bytes per pixel per iteration: 24 (phase A) + 32 (phase B) versus 112 in FP64.
#include "ulp_mixed.cuh"
#include "ulp_host.h"

namespace ulp {

// FP32 copies of the weights and the Jacobi inverse; the correction starts at 0.
template <int KIND>
__device__ __forceinline__ void conv_tile(const PcgArgs& a, const MapDesc& M, int t, int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  const size_t P = M.pitch;
  const int j = g.j0 + 2 * lane;
  for (int i = g.i0; i < g.i1; ++i) {
    const size_t off = (size_t)i * P + j;
    const double2 u = ld2(M.f.U, off), v = ld2(M.f.V, off);
    stf2(M.h.U, off, make_float2((float)u.x, (float)u.y));
    stf2(M.h.V, off, make_float2((float)v.x, (float)v.y));
    if (KIND == kJacobi) {
      const double2 di = ld2(M.f.Dinv, off);
      stf2(M.h.Dinv, off, make_float2((float)di.x, (float)di.y));
    }
    stf2(M.h.x, off, make_float2(0.f, 0.f));
  }
}

// True residual in FP64: r = b - A phi (FP64 weights, FP64 phi), rounded to
// FP32 for the recurrence; s = M^-1 r; partials r^T s, r^T r (and b^T b).
template <int KIND>
__device__ __forceinline__ void res64_tile(const PcgArgs& a, const MapDesc& M, MapState* S, int t, bool init,
                                           int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  XPlane x{M.f.phi, (size_t)M.pitch};
  DF rs, rr;
  double bb = 0.0;
  auto epi = [&](size_t off, double2, double2 ax) {
    const double2 bv = ld2(M.f.b, off);
    const float2 r = make_float2((float)(bv.x - ax.x), (float)(bv.y - ax.y));
    stf2(M.h.r, off, r);
    if (KIND == kJacobi) {
      const float2 di = ldf2(M.h.Dinv, off);
      const float2 s = make_float2(di.x * r.x, di.y * r.y);
      stf2(M.h.s, off, s);
      rs.add_prod(r.x, s.x);
      rs.add_prod(r.y, s.y);
    }
    rr.add_prod(r.x, r.x);
    rr.add_prod(r.y, r.y);
    if (init) {
      bb = fma(bv.x, bv.x, bb);
      bb = fma(bv.y, bv.y, bb);
    }
  };
  stencil_tile(M, g.i0, g.i1, g.j0, lane, M.f.U, M.f.V, M.f.D, x, epi);
  const double vrr = rr.value();
  const double vrs = (KIND == kIdentity) ? vrr : rs.value();
  tile_arrive(a, M, S, t, init ? kPhResInit : kPhRes, vrs, vrr, bb, lane);
}

// Phase B's ring slots (kRingB32 per warp, inside the warp's share of phase A's ring).
constexpr int kLeadB32 = 3;
constexpr int kRingB32 = kLeadB32 + 1;  // elementwise: a slot is refilled one row after it was read
struct SlotB32 {
  float2 d[32], x[32], q[32], r[32], di[32];
};
static_assert(kRingB32 * sizeof(SlotB32) <= kRing32 * sizeof(Slot32), "phase B's ring fits phase A's");

// x += alpha d; then either r -= alpha q, s = M^-1 r (partials) or, on a
// refresh iteration, phi += x, x = 0 (the residual is then recomputed in FP64).
// wring: the warp's share of phase A's ring, through which the rows stream kLeadB32
// ahead (or null, and on refresh iterations: loads two rows ahead in registers).
template <int KIND>
__device__ __forceinline__ void b32_tile(const PcgArgs& a, const MapDesc& M, MapState* S, int t, bool refresh,
                                         int lane, unsigned char* wring) {
  const TileGeo g = tile_geo(M, t, a.R);
  const size_t P = M.pitch;
  const long long it = *(volatile long long*)&S->iter;
  const float* d = (it & 1) ? M.h.d0 : M.h.d1;
  const float alpha = (float)*(volatile double*)&S->alpha;
  const int j = g.j0 + 2 * lane;
  const float2 z2 = make_float2(0.f, 0.f);
  struct Row {
    float2 d, x, q, r, di;
  };
  auto load = [&](int i) {
    Row w{z2, z2, z2, z2, z2};
    if (i < g.i1) {
      const size_t off = (size_t)i * P + j;
      w.d = ldf2(d, off);
      w.x = ldf2(M.h.x, off);
      if (!refresh) {
        w.q = ldf2(M.h.q, off);
        w.r = ldf2(M.h.r, off);
        if (KIND == kJacobi) w.di = ldf2(M.h.Dinv, off);
      }
    }
    return w;
  };
  DF rs, rr;
  if (!refresh && wring) {
    // the rows stream through the warp's ring in shared memory (phase A's ring, free in
    // this phase), kLeadB32 rows ahead; the arithmetic is that of the loop below
    SlotB32* ring = reinterpret_cast<SlotB32*>(wring);
    auto issue = [&](SlotB32& sl, int i) {
      const size_t off = (size_t)i * P + j;
      cpa8(&sl.d[lane], d + off, 8);
      cpa8(&sl.x[lane], M.h.x + off, 8);
      cpa8(&sl.q[lane], M.h.q + off, 8);
      cpa8(&sl.r[lane], M.h.r + off, 8);
      if (KIND == kJacobi) cpa8(&sl.di[lane], M.h.Dinv + off, 8);
    };
#pragma unroll
    for (int k = 0; k < kLeadB32; ++k) {
      if (g.i0 + k < g.i1) issue(ring[k], g.i0 + k);
      cpa_commit();
    }
    for (int i = g.i0; i < g.i1; ++i) {
      cpa_wait<kLeadB32 - 1>();
      const SlotB32& sl = ring[(i - g.i0) % kRingB32];
      const float2 dv = sl.d[lane], qv = sl.q[lane];
      float2 xv = sl.x[lane], r = sl.r[lane];
      const float2 di = (KIND == kJacobi) ? sl.di[lane] : z2;
      if (i + kLeadB32 < g.i1) issue(ring[(i + kLeadB32 - g.i0) % kRingB32], i + kLeadB32);
      cpa_commit();
      const size_t off = (size_t)i * P + j;
      xv.x = __fmaf_rn(alpha, dv.x, xv.x);
      xv.y = __fmaf_rn(alpha, dv.y, xv.y);
      stf2(M.h.x, off, xv);
      r.x = __fmaf_rn(-alpha, qv.x, r.x);
      r.y = __fmaf_rn(-alpha, qv.y, r.y);
      stf2(M.h.r, off, r);
      if (KIND == kJacobi) {
        const float2 sv = make_float2(di.x * r.x, di.y * r.y);
        stf2(M.h.s, off, sv);
        rs.add_prod(r.x, sv.x);
        rs.add_prod(r.y, sv.y);
      }
      rr.add_prod(r.x, r.x);
      rr.add_prod(r.y, r.y);
    }
    cpa_wait_all();
    const double vrr = rr.value();
    tile_arrive(a, M, S, t, kPhB, (KIND == kIdentity) ? vrr : rs.value(), vrr, 0.0, lane);
    return;
  }
  Row c0 = load(g.i0), c1 = load(g.i0 + 1);
  for (int i = g.i0; i < g.i1; ++i) {
    const Row c2 = load(i + 2);
    const size_t off = (size_t)i * P + j;
    float2 xv = c0.x;
    xv.x = __fmaf_rn(alpha, c0.d.x, xv.x);
    xv.y = __fmaf_rn(alpha, c0.d.y, xv.y);
    if (refresh) {
      double2 ph = ld2(M.f.phi, off);
      ph.x += (double)xv.x;
      ph.y += (double)xv.y;
      st2(M.f.phi, off, ph);
      stf2(M.h.x, off, z2);
    } else {
      stf2(M.h.x, off, xv);
      float2 r = c0.r;
      r.x = __fmaf_rn(-alpha, c0.q.x, r.x);
      r.y = __fmaf_rn(-alpha, c0.q.y, r.y);
      stf2(M.h.r, off, r);
      if (KIND == kJacobi) {
        const float2 s = make_float2(c0.di.x * r.x, c0.di.y * r.y);
        stf2(M.h.s, off, s);
        rs.add_prod(r.x, s.x);
        rs.add_prod(r.y, s.y);
      }
      rr.add_prod(r.x, r.x);
      rr.add_prod(r.y, r.y);
    }
    c0 = c1;
    c1 = c2;
  }
  if (!refresh) {
    const double vrr = rr.value();
    tile_arrive(a, M, S, t, kPhB, (KIND == kIdentity) ? vrr : rs.value(), vrr, 0.0, lane);
  }
}

// phi += x, x = 0 (end of the solve).
__device__ __forceinline__ void fold_tile(const PcgArgs& a, const MapDesc& M, int t, int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  const size_t P = M.pitch;
  const int j = g.j0 + 2 * lane;
  for (int i = g.i0; i < g.i1; ++i) {
    const size_t off = (size_t)i * P + j;
    const float2 xv = ldf2(M.h.x, off);
    double2 ph = ld2(M.f.phi, off);
    ph.x += (double)xv.x;
    ph.y += (double)xv.y;
    st2(M.f.phi, off, ph);
    stf2(M.h.x, off, make_float2(0.f, 0.f));
  }
}

template <int KIND>
__global__ void __launch_bounds__(kThreads, 2) k_pcg32(PcgArgs a) {
  __shared__ Slot32 ring32[kWarps][kRing32];  // phase A's row rings, phase B's in turn
  __shared__ int s_base[kMaxMaps + 1];
  __shared__ int s_any;
  for (int m = threadIdx.x; m <= a.nmaps; m += blockDim.x)
    s_base[m] = (m < a.nmaps) ? a.maps[m].tile_base : a.ntiles;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int NW = gridDim.x * kWarps;
  auto for_tiles = [&](auto&& body) {
    for (int t = gw; t < a.ntiles; t += NW) {
      const int m = find_map(s_base, a.nmaps, t);
      MapState* S = a.st + m;
      if (*(volatile int*)&S->done) continue;
      body(a.maps[m], S, t);
    }
  };
  // maps active at the start: the final fold must reach them after they stop
  auto for_tiles_started = [&](auto&& body) {
    for (int t = gw; t < a.ntiles; t += NW) {
      const int m = find_map(s_base, a.nmaps, t);
      if (!a.st[m].outer_active) continue;
      body(a.maps[m], t);
    }
  };

  for_tiles([&](const MapDesc& M, MapState*, int t) { conv_tile<KIND>(a, M, t, lane); });
  if (!grid_sync(a.bar, a.timeout_ns)) return;
  for_tiles([&](const MapDesc& M, MapState* S, int t) { res64_tile<KIND>(a, M, S, t, true, lane); });
  if (!grid_sync(a.bar, a.timeout_ns)) return;

  for (int g = 0;; ++g) {
    if (*(volatile int*)a.n_active == 0) break;
    for_tiles([&](const MapDesc& M, MapState* S, int t) { a32_tile<KIND>(a, M, S, t, lane, ring32[threadIdx.x >> 5]); });
    if (!grid_sync(a.bar, a.timeout_ns)) return;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int m = threadIdx.x; m < a.nmaps; m += blockDim.x)
      if (g % a.maps[m].refresh == 0) s_any = 1;
    __syncthreads();
    const bool any_refresh = s_any != 0;
    for_tiles([&](const MapDesc& M, MapState* S, int t) {
      b32_tile<KIND>(a, M, S, t, (g % M.refresh) == 0, lane, reinterpret_cast<unsigned char*>(ring32[threadIdx.x >> 5]));
    });
    if (!grid_sync(a.bar, a.timeout_ns)) return;
    if (any_refresh) {
      for_tiles([&](const MapDesc& M, MapState* S, int t) {
        if ((g % M.refresh) == 0) res64_tile<KIND>(a, M, S, t, false, lane);
      });
      if (!grid_sync(a.bar, a.timeout_ns)) return;
    }
  }
  for_tiles_started([&](const MapDesc& M, int t) { fold_tile(a, M, t, lane); });
}

int pcg32_max_blocks_per_sm(int kind) {
  int nb = 0;
  if (kind == kIdentity) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg32<kIdentity>, kThreads, 0);
  else if (kind == kJacobi) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg32<kJacobi>, kThreads, 0);
  return nb;
}

cudaError_t launch_pcg32(const Plan& pl, int kind, const PcgArgs& a, cudaStream_t st, cudaEvent_t e0,
                         cudaEvent_t e1) {
  pl.kernel_launches += 2;
  pl.solver_launches += 1;
  launch_pcg_reset(pl, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (e0) cudaEventRecord(e0, st);
  const int blocks = pl.nsm * pl.bps;
  void* args[] = {(void*)&a};
  if (kind == kIdentity)
    e = cudaLaunchCooperativeKernel((void*)k_pcg32<kIdentity>, blocks, kThreads, args, 0, st);
  else if (kind == kJacobi)
    e = cudaLaunchCooperativeKernel((void*)k_pcg32<kJacobi>, blocks, kThreads, args, 0, st);
  else
    e = cudaErrorInvalidValue;
  if (e == cudaSuccess && e1) e = cudaEventRecord(e1, st);
  return e;
}

}  // namespace ulp
