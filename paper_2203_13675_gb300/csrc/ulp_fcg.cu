// ulp_fcg.cu -- inner solve with the DCT Poisson preconditioner: flexible CG in
// one CUDA graph.
//
// The DCT preconditioner runs on the tensor cores as four GEMM launches, so
// this solve is not a single persistent kernel: each phase of an iteration is
// its own kernel and the loop is a graph WHILE node whose condition the
// device clears when the map stops (converged, l_max or breakdown), so the
// host never waits inside the solve.  The BF16 GEMMs make M^-1 slightly
// inexact and not exactly symmetric, so beta is the flexible (Polak-Ribiere)
// one, beta = r_{k+1}^T (s_{k+1} - s_k) / r_k^T s_k; the term r_{k+1}^T s_k is
// accumulated in phase B, before the GEMMs overwrite s.  All vectors, alpha,
// beta and the stop tests are FP64, as in the other FP64 solvers.
//
// Per iteration:  A: d = s + beta d, q = A d, d^T q -> alpha
//                 B: phi += alpha d, r -= alpha q (not on refresh iterations), r^T s_k
//                 R: on refresh iterations r = b - A phi, r^T s_k
//                 DCT: s = Pi L^+ r (4 tcgen05 GEMMs on the BF16 copy of r that B and R write)
//                 D: r^T s, r^T r -> beta, stop test, WHILE condition
#include <cuda_bf16.h>

#include "ulp_mixed.cuh"

#include "ulp_host.h"

namespace ulp {

__global__ void k_set_args(PcgArgs a, PcgArgs* dst) { *dst = a; }

// Set-up timing of a flexible-CG solve (plans with options.profile): end = 0 records the
// start of the preconditioner's set-up, end = 1 adds its duration to map 0's statistics.
__global__ void k_setup_stamp(const PcgArgs* pa, int end) {
  MapStats* st = pa->stats;
  if (!st || *(volatile int*)&pa->st->done) return;
  const unsigned long long t = globaltimer();
  if (end) st->setup_ns += t - st->setup_t0;
  else st->setup_t0 = t;
}

// one warp per tile (grid-stride), the single map of the plan
#define FCG_TILE_LOOP(a)                                               \
  const int lane = threadIdx.x & 31;                                   \
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);  \
  const int NW = gridDim.x * (blockDim.x >> 5);                        \
  const MapDesc& M = a.maps[0];                                        \
  MapState* S = a.st;                                                  \
  for (int t = gw; t < a.ntiles; t += NW)

// split BF16 copy of r at (i, j), (i, j+1) for the DCT's first GEMM (high plane bf16(r), low
// plane bf16(r - high)), or the FP32 copy the multigrid cycle starts from (zero beyond column W-1)
__device__ __forceinline__ void put_rbf(const PcgArgs& a, const MapDesc& M, int i, int j, double2 r) {
  if (a.rbf && j < M.W) {
    const float fx = (float)r.x, fy = j + 1 < M.W ? (float)r.y : 0.f;
    const __nv_bfloat162 v = __floats2bfloat162_rn(fx, fy);
    const float2 h = __bfloat1622float2(v);
    const __nv_bfloat162 lo = __floats2bfloat162_rn(fx - h.x, fy - h.y);
    a.rbf[(size_t)i * a.rbf_ld + (j >> 1)] = *reinterpret_cast<const unsigned*>(&v);
    a.rbf_lo[(size_t)i * a.rbf_ld + (j >> 1)] = *reinterpret_cast<const unsigned*>(&lo);
  }
  if (a.rf32 && j < M.W)
    *reinterpret_cast<float2*>(a.rf32 + (size_t)i * M.pitch + j) =
        make_float2((float)r.x, j + 1 < M.W ? (float)r.y : 0.f);
}

// The WHILE loop's own guard (one thread), run after the start phase and at the
// head of every body execution: a map that has stopped -- or was never active in
// this outer pass, so no finisher will run -- clears the condition, and so does
// a loop that has run past l_max (reported as a time-out).  The rest of that body
// execution then finds the map stopped and returns at once.
__global__ void k_f_guard(const PcgArgs* pa, int count) {
  const PcgArgs a = *pa;
  MapState* S = a.st;
  const MapDesc& M = a.maps[0];
  const long long lmax = a.lmax > 0 ? a.lmax : 2LL * M.H * M.W;
  const long long loops = count ? ++S->loops : S->loops;
  if (*(volatile int*)&S->done) {
    cudaGraphSetConditional(a.cond, 0);
  } else if (loops > lmax + 2) {
    S->status = -4;
    S->done = 1;
    atomicSub(a.n_active, 1);
    __threadfence();
    cudaGraphSetConditional(a.cond, 0);
  }
}

// r = b - A phi (start, or refresh iterations only); on refresh iterations also r^T s_k.
__global__ void __launch_bounds__(kThreads, 2) k_f_res(const PcgArgs* pa, int refresh_only) {
  const PcgArgs a = *pa;
  FCG_TILE_LOOP(a) {
    if (*(volatile int*)&S->done) return;
    const long long it = *(volatile long long*)&S->iter;
    if (refresh_only && (it % M.refresh) != 0) return;
    const TileGeo g = tile_geo(M, t, a.R);
    XPlane x{M.f.phi, (size_t)M.pitch};
    double rsp = 0.0;
    const int j = g.j0 + 2 * lane;
    int ir = g.i0;  // the walker calls epi once per row, in order
    auto epi = [&](size_t off, double2, double2 ax) {
      const double2 bv = ld2(M.f.b, off);
      const double2 r = make_double2(bv.x - ax.x, bv.y - ax.y);
      st2(M.f.r, off, r);
      put_rbf(a, M, ir++, j, r);
      if (refresh_only) {
        const double2 sv = ld2(M.f.s, off);
        rsp = fma(r.x, sv.x, rsp);
        rsp = fma(r.y, sv.y, rsp);
      }
    };
    stencil_tile(M, g.i0, g.i1, g.j0, lane, M.f.U, M.f.V, M.f.D, x, epi);
    if (refresh_only) {
      rsp = warp_sum(rsp);
      if (lane == 0) __stcg(a.P2 + t, rsp);
    }
  }
}

// d = s + beta d_old (d = s at l = 0), q = A d, d^T q -> alpha.
__global__ void __launch_bounds__(kThreads) k_f_a(const PcgArgs* pa) {
  const PcgArgs a = *pa;
  FCG_TILE_LOOP(a) {
    if (*(volatile int*)&S->done) return;
    a_tile<kJacobi>(a, M, S, t, lane);
  }
}

// Phase B's row ring of the FP64 flexible CG: kRingF slots per warp of the five FP64
// rows it reads (dynamic shared memory, kRingFSmem per block).
constexpr int kLeadF = 3;
constexpr int kRingF = kLeadF + 1;  // elementwise: a slot is refilled one row after it was read
struct SlotF {
  double2 d[32], ph[32], q[32], s[32], r[32];
};
constexpr size_t kRingFSmem = (size_t)kWarps * kRingF * sizeof(SlotF);  // 81,920 bytes

__device__ __forceinline__ void cpa16f(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}

// phi += alpha d; r -= alpha q and r^T s_k (not on refresh iterations).
__global__ void __launch_bounds__(kThreads) k_f_b(const PcgArgs* pa) {
  extern __shared__ __align__(16) unsigned char fb_dsm[];
  const PcgArgs a = *pa;
  FCG_TILE_LOOP(a) {
    if (*(volatile int*)&S->done) return;
    const long long it = *(volatile long long*)&S->iter;
    const bool refresh = (it % M.refresh) == 0;
    const TileGeo g = tile_geo(M, t, a.R);
    const size_t P = M.pitch;
    const double* __restrict__ d = (it & 1) ? M.f.d0 : M.f.d1;
    double* __restrict__ phi = M.f.phi;
    double* __restrict__ rp = M.f.r;
    const double* __restrict__ qp = M.f.q;
    const double* __restrict__ sp = M.f.s;
    const double alpha = *(volatile double*)&S->alpha;
    const int j = g.j0 + 2 * lane;
    double rsp = 0.0;
    if (!refresh) {
      // the rows stream through the warp's ring in shared memory, kLeadF rows ahead of
      // the arithmetic (that of the loop below)
      SlotF* ring = reinterpret_cast<SlotF*>(fb_dsm) + (threadIdx.x >> 5) * kRingF;
      auto issue = [&](SlotF& sl, int i) {
        const size_t off = (size_t)i * P + j;
        cpa16f(&sl.d[lane], d + off);
        cpa16f(&sl.ph[lane], phi + off);
        cpa16f(&sl.q[lane], qp + off);
        cpa16f(&sl.s[lane], sp + off);
        cpa16f(&sl.r[lane], rp + off);
      };
#pragma unroll
      for (int k = 0; k < kLeadF; ++k) {
        if (g.i0 + k < g.i1) issue(ring[k], g.i0 + k);
        cpa_commit();
      }
      for (int i = g.i0; i < g.i1; ++i) {
        cpa_wait<kLeadF - 1>();
        const SlotF& sl = ring[(i - g.i0) % kRingF];
        const double2 dv = sl.d[lane], qv = sl.q[lane], sv = sl.s[lane];
        double2 ph = sl.ph[lane], r = sl.r[lane];
        if (i + kLeadF < g.i1) issue(ring[(i + kLeadF - g.i0) % kRingF], i + kLeadF);
        cpa_commit();
        const size_t off = (size_t)i * P + j;
        ph.x = fma(alpha, dv.x, ph.x);
        ph.y = fma(alpha, dv.y, ph.y);
        st2(phi, off, ph);
        r.x = fma(-alpha, qv.x, r.x);
        r.y = fma(-alpha, qv.y, r.y);
        st2(rp, off, r);
        put_rbf(a, M, i, j, r);
        rsp = fma(r.x, sv.x, rsp);
        rsp = fma(r.y, sv.y, rsp);
      }
      cpa_wait_all();  // the warp's next tile refills the same slots
      rsp = warp_sum(rsp);
      if (lane == 0) __stcg(a.P2 + t, rsp);
      continue;
    }
    // refresh iterations (phi only): rows in groups of four, all loads of a group first
    for (int i = g.i0; i < g.i1; i += 4) {
      double2 dv[4], ph[4], qv[4], sv[4], rv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (i + k < g.i1) {
          const size_t off = (size_t)(i + k) * P + j;
          dv[k] = ld2(d, off);
          ph[k] = ld2(phi, off);
          if (!refresh) {
            qv[k] = ld2(qp, off);
            sv[k] = ld2(sp, off);
            rv[k] = ld2(rp, off);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (i + k < g.i1) {
          const size_t off = (size_t)(i + k) * P + j;
          ph[k].x = fma(alpha, dv[k].x, ph[k].x);
          ph[k].y = fma(alpha, dv[k].y, ph[k].y);
          st2(phi, off, ph[k]);
          if (!refresh) {
            double2 r = rv[k];
            r.x = fma(-alpha, qv[k].x, r.x);
            r.y = fma(-alpha, qv[k].y, r.y);
            st2(rp, off, r);
            put_rbf(a, M, i + k, j, r);
            rsp = fma(r.x, sv[k].x, rsp);
            rsp = fma(r.y, sv[k].y, rsp);
          }
        }
      }
    }
    if (!refresh) {
      rsp = warp_sum(rsp);
      if (lane == 0) __stcg(a.P2 + t, rsp);
    }
  }
}

// r^T s, r^T r (and b^T b at the start) -> delta, beta, stop test.
__global__ void __launch_bounds__(kThreads, 2) k_f_dots(const PcgArgs* pa, int init) {
  const PcgArgs a = *pa;
  FCG_TILE_LOOP(a) {
    if (*(volatile int*)&S->done) return;
    const TileGeo g = tile_geo(M, t, a.R);
    const size_t P = M.pitch;
    const int j = g.j0 + 2 * lane;
    const double* __restrict__ rp = M.f.r;
    const double* __restrict__ sp = M.f.s;
    const double* __restrict__ bp = M.f.b;
    double rs = 0.0, rr = 0.0, bb = 0.0;
    if (init) {
      for (int i = g.i0; i < g.i1; ++i) {
        const size_t off = (size_t)i * P + j;
        const double2 rv = ld2(rp, off), sv = ld2(sp, off), bv = ld2(bp, off);
        rs = fma(rv.x, sv.x, rs);
        rs = fma(rv.y, sv.y, rs);
        rr = fma(rv.x, rv.x, rr);
        rr = fma(rv.y, rv.y, rr);
        bb = fma(bv.x, bv.x, bb);
        bb = fma(bv.y, bv.y, bb);
      }
    } else {
      // rows in groups of eight, all sixteen loads of a group in flight together
      for (int i = g.i0; i < g.i1; i += 8) {
        double2 rv[8], sv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (i + k < g.i1) {
            const size_t off = (size_t)(i + k) * P + j;
            rv[k] = ld2(rp, off);
            sv[k] = ld2(sp, off);
          }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (i + k < g.i1) {
            rs = fma(rv[k].x, sv[k].x, rs);
            rs = fma(rv[k].y, sv[k].y, rs);
            rr = fma(rv[k].x, rv[k].x, rr);
            rr = fma(rv[k].y, rv[k].y, rr);
          }
        }
      }
    }
    tile_arrive(a, M, S, t, init ? kPhResInit : kPhFcg, rs, rr, bb, lane);
  }
}

// ---------------------------------------------------------------- mixed flexible CG
// The multigrid solve with the precision split of the mixed form: the Krylov
// recurrence (d, q = A d, r, s and the correction x since the last refresh) on
// FP32 planes with FP32 weights, the inner products as double-float sums of exact
// FP32 products, alpha, beta and the stop tests in FP64, and phi in FP64:
// every refresh period the correction is folded into phi and r = b - A phi is
// recomputed with the FP64 weights.  The multigrid cycle
// reads r directly (its FP32 right-hand side is the recurrence's r plane) and
// writes s in FP32.  When the recurrence reports convergence, the next body takes
// no step (A returns at once, B uses alpha = 0): it folds the correction into phi,
// recomputes r = b - A phi in FP64 and s, and the solve stops there if the true
// residual meets the tolerance, with the iteration count of the recurrence's stop
// (the point where Algorithm 1 stops on its recurrence residual); otherwise every
// further iteration is a refresh iteration and the solve stops on a true residual.
//   A: d = s + beta d, q = A d, d^T q  (the mixed engine's phase A)
//   B: x += alpha d; r -= alpha q, r_{k+1}^T s_k and r^T r per tile, or on refresh
//      iterations phi += x, x = 0
//   R: on refresh iterations r = b - A phi (FP64, rounded to FP32), r_{k+1}^T s_k, r^T r
//   M: the V-cycle, whose last kernel sums r^T s and runs the dot phase

// The map state a phase of the mixed flexible CG reads, loaded as one batch of
// independent loads (one round trip to L2, where a chain of tests would wait for each).
// refresh: the iteration recomputes the true residual -- every M.refresh-th after the
// first (the start computed r in FP64 just before iteration 0), the one after ||r|| has
// fallen 100-fold since the last true residual (so the FP32 correction x never holds more
// than about 1 % of the iterate's change since then, and its rounding stays below the
// tolerance's reach), the confirmation body that follows the recurrence's first report of
// convergence, and every iteration within a factor 2 of the tolerance or after a
// confirmation that missed it.
struct XState {
  long long it;
  double alpha;
  int done, confirm, refresh;
};
__device__ __forceinline__ XState x_state(const MapDesc& M, MapState* S) {
  const volatile MapState* v = S;
  XState x;
  x.done = v->done;
  x.it = v->iter;
  const int fr = v->force_refresh;
  x.confirm = v->confirm;
  const int rn = v->refresh_next;
  x.alpha = v->alpha;
  x.refresh = ((x.it > 0 && (x.it % M.refresh) == 0) ? 1 : 0) | fr | x.confirm | rn;
  return x;
}

__global__ void __launch_bounds__(kThreads, 2) k_x_a(const PcgArgs* pa) {
  __shared__ Slot32 ring[kWarps][kRing32];  // the stencil's row rings
  const PcgArgs a = *pa;
  FCG_TILE_LOOP(a) {
    const volatile MapState* v = S;
    const int done = v->done, confirm = v->confirm;
    if (done | confirm) return;  // a confirmation body takes no step
    a32_tile<kJacobi>(a, M, S, t, lane, ring[threadIdx.x >> 5]);
  }
}

// Phase B's row ring: kRingB slots per warp of the five FP32 rows it reads (dynamic
// shared memory, kRingBSmem per block).
constexpr int kLeadB = 6;
constexpr int kRingB = kLeadB + 1;  // elementwise: a slot is refilled one row after it was read
struct SlotB {
  float2 d[32], x[32], q[32], r[32], s[32];
};
constexpr size_t kRingBSmem = (size_t)kWarps * kRingB * sizeof(SlotB);  // 71,680 bytes

__global__ void __launch_bounds__(kThreads, 2) k_x_b(const PcgArgs* pa) {
  extern __shared__ __align__(16) unsigned char xb_dsm[];
  const PcgArgs a = *pa;
  FCG_TILE_LOOP(a) {
    const XState xs = x_state(M, S);
    if (xs.done) return;
    const bool refresh = xs.refresh;
    const long long it = xs.it;
    const TileGeo g = tile_geo(M, t, a.R);
    const size_t P = M.pitch;
    const float* __restrict__ d = (it & 1) ? M.h.d0 : M.h.d1;
    // a confirmation body only folds the correction into phi (no step: alpha = 0)
    const float alpha = xs.confirm ? 0.f : (float)xs.alpha;
    const int j = g.j0 + 2 * lane;
    DF rsp, rrp;
    if (refresh) {
      // phi += x + alpha d, x = 0: rows in groups of four, all loads of a group first
      for (int i = g.i0; i < g.i1; i += 4) {
        float2 dv[4], xv[4];
        double2 pv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (i + k < g.i1) {
            const size_t off = (size_t)(i + k) * P + j;
            dv[k] = ldf2(d, off);
            xv[k] = ldf2(M.h.x, off);
            pv[k] = ld2(M.f.phi, off);
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (i + k < g.i1) {
            const size_t off = (size_t)(i + k) * P + j;
            float2 x = xv[k];
            x.x = __fmaf_rn(alpha, dv[k].x, x.x);
            x.y = __fmaf_rn(alpha, dv[k].y, x.y);
            double2 ph = pv[k];
            ph.x += (double)x.x;
            ph.y += (double)x.y;
            st2(M.f.phi, off, ph);
            stf2(M.h.x, off, make_float2(0.f, 0.f));
          }
        }
      }
    } else {
      // x += alpha d, r -= alpha q and the partials r^T s, r^T r: the five rows of
      // each pixel row stream through the warp's ring in shared memory, kLeadB rows
      // ahead of the arithmetic (the loads in flight cost no registers, and each lane
      // reads back only what it copied)
      SlotB* ring = reinterpret_cast<SlotB*>(xb_dsm) + (threadIdx.x >> 5) * kRingB;
      auto issue = [&](SlotB& sl, int i) {
        const size_t off = (size_t)i * P + j;
        cpa8(&sl.d[lane], d + off, 8);
        cpa8(&sl.x[lane], M.h.x + off, 8);
        cpa8(&sl.q[lane], M.h.q + off, 8);
        cpa8(&sl.r[lane], M.h.r + off, 8);
        cpa8(&sl.s[lane], M.h.s + off, 8);
      };
#pragma unroll
      for (int k = 0; k < kLeadB; ++k) {
        if (g.i0 + k < g.i1) issue(ring[k], g.i0 + k);
        cpa_commit();
      }
      for (int i = g.i0; i < g.i1; ++i) {
        cpa_wait<kLeadB - 1>();  // row i has landed
        const SlotB& sl = ring[(i - g.i0) % kRingB];
        const float2 dv = sl.d[lane], qv = sl.q[lane], sv = sl.s[lane];
        float2 x = sl.x[lane], r = sl.r[lane];
        // the slot of row i - 1 is free: refill it with row i + kLeadB
        if (i + kLeadB < g.i1) issue(ring[(i + kLeadB - g.i0) % kRingB], i + kLeadB);
        cpa_commit();
        const size_t off = (size_t)i * P + j;
        x.x = __fmaf_rn(alpha, dv.x, x.x);
        x.y = __fmaf_rn(alpha, dv.y, x.y);
        stf2(M.h.x, off, x);
        r.x = __fmaf_rn(-alpha, qv.x, r.x);
        r.y = __fmaf_rn(-alpha, qv.y, r.y);
        stf2(M.h.r, off, r);
        rsp.add_prod(r.x, sv.x);
        rsp.add_prod(r.y, sv.y);
        rrp.add_prod(r.x, r.x);
        rrp.add_prod(r.y, r.y);
      }
      cpa_wait_all();  // the warp's next tile refills the same slots
    }
    if (!refresh) {
      // r_{k+1}^T s_k and r_{k+1}^T r_{k+1} per tile for the dot phase
      const double v = warp_sum(rsp.value()), w = warp_sum(rrp.value());
      if (lane == 0) {
        __stcg(a.P2 + t, v);
        __stcg(a.P1 + t, w);
      }
    }
  }
}

// r = b - A phi in FP64, rounded to FP32, and its r^T r per tile (x = 0 with it at the
// start, and the b^T b partials for the start's dot phase); on refresh iterations also
// r_{k+1}^T s_k.
__global__ void __launch_bounds__(kThreads, 2) k_x_res(const PcgArgs* pa, int init) {
  const PcgArgs a = *pa;
  FCG_TILE_LOOP(a) {
    const XState xs = x_state(M, S);
    if (xs.done) return;
    if (!init && !xs.refresh) return;
    // a confirmation body under the relative-residual stop decides here whether the solve ends
    const bool confirm = !init && a.stop_mode == ULP_STOP_RELRES && xs.confirm;
    const TileGeo g = tile_geo(M, t, a.R);
    XPlane x{M.f.phi, (size_t)M.pitch};
    DF rsp, rrp;
    double bb = 0.0;
    auto epi = [&](size_t off, double2, double2 ax) {
      const double2 bv = ld2(M.f.b, off);
      const float2 r = make_float2((float)(bv.x - ax.x), (float)(bv.y - ax.y));
      stf2(M.h.r, off, r);
      rrp.add_prod(r.x, r.x);
      rrp.add_prod(r.y, r.y);
      if (init) {
        stf2(M.h.x, off, make_float2(0.f, 0.f));
        bb = fma(bv.x, bv.x, bb);
        bb = fma(bv.y, bv.y, bb);
      } else {
        const float2 sv = ldf2(M.h.s, off);
        rsp.add_prod(r.x, sv.x);
        rsp.add_prod(r.y, sv.y);
      }
    };
    stencil_tile(M, g.i0, g.i1, g.j0, lane, M.f.U, M.f.V, M.f.D, x, epi);
    const double v = warp_sum(init ? bb : rsp.value());
    if (confirm) {
      // r_{k+1}^T s_k for the dot phase, should the body go on; r^T r through the arrival
      if (lane == 0) __stcg(a.P2 + t, v);
      tile_arrive(a, M, S, t, kPhConfirm, 0.0, rrp.value(), 0.0, lane);
      continue;
    }
    const double w = warp_sum(rrp.value());
    if (lane == 0) {
      __stcg(a.P2 + t, v);
      __stcg(a.P1 + t, w);
    }
  }
}

// r^T s, r^T r (double-float) and, at the start of the solve, b^T b (FP64) -> delta, beta,
// stop test (used where the multigrid cycle cannot carry the dot phase)
__global__ void __launch_bounds__(kThreads, 2) k_x_dots(const PcgArgs* pa, int init) {
  const PcgArgs a = *pa;
  FCG_TILE_LOOP(a) {
    if (*(volatile int*)&S->done) return;
    const TileGeo g = tile_geo(M, t, a.R);
    const size_t P = M.pitch;
    const int j = g.j0 + 2 * lane;
    DF rs, rr;
    double bb = 0.0;
    for (int i = g.i0; i < g.i1; ++i) {
      const size_t off = (size_t)i * P + j;
      const float2 rv = ldf2(M.h.r, off), sv = ldf2(M.h.s, off);
      rs.add_prod(rv.x, sv.x);
      rs.add_prod(rv.y, sv.y);
      rr.add_prod(rv.x, rv.x);
      rr.add_prod(rv.y, rv.y);
      if (init) {
        const double2 bv = ld2(M.f.b, off);
        bb = fma(bv.x, bv.x, bb);
        bb = fma(bv.y, bv.y, bb);
      }
    }
    tile_arrive(a, M, S, t, init ? kPhResInit : kPhFcg, rs.value(), rr.value(), bb, lane);
  }
}

// end of the solve: phi += x; nothing to do after a stop on a refresh iteration (x = 0 then),
// only after l_max or a breakdown
__global__ void __launch_bounds__(kThreads) k_x_fold(const PcgArgs* pa) {
  const PcgArgs a = *pa;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int NW = gridDim.x * (blockDim.x >> 5);
  const MapDesc& M = a.maps[0];
  if (!a.st->outer_active || *(volatile int*)&a.st->x_clean) return;
  for (int t = gw; t < a.ntiles; t += NW) {
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
}

// Learned preconditioner's fallback: s = D^-1 r once the map's fallback flag is
// set (the network kernels skip themselves from then on).
__global__ void __launch_bounds__(kThreads) k_f_jacobi(const PcgArgs* pa) {
  const PcgArgs a = *pa;
  FCG_TILE_LOOP(a) {
    if (*(volatile int*)&S->done || !*(volatile int*)&S->fallback) return;
    const TileGeo g = tile_geo(M, t, a.R);
    const size_t P = M.pitch;
    const int j = g.j0 + 2 * lane;
    const double* __restrict__ rp = M.f.r;
    const double* __restrict__ dp = M.f.Dinv;
    double* __restrict__ sp = M.f.s;
    for (int i = g.i0; i < g.i1; ++i) {
      const size_t off = (size_t)i * P + j;
      const double2 rv = ld2(rp, off), di = ld2(dp, off);
      st2(sp, off, make_double2(di.x * rv.x, di.y * rv.y));
    }
  }
}

static int tile_blocks(const Plan& pl) { return (pl.ntiles + kWarps - 1) / kWarps; }

// s = M^-1 r of the flexible solve: the DCT chain, or the network followed by its
// Jacobi fallback (only one of the two does work in any iteration).
// the mixed flexible CG runs for the multigrid preconditioner on mixed-precision plans
static bool mixed_fcg(const Plan& pl, int kind) {
  return kind == ULP_PRECOND_MG && pl.opt.precision == ULP_PRECISION_MIXED;
}

// With fuse_dots the multigrid cycle's last kernel also runs the dot phase D (at the
// start of a solve, init: its start form, with b^T b).
// part (multigrid): as mg_apply's, so a replay can time the cycle's last kernel alone.
static cudaError_t fcg_precond(Plan& pl, int kind, cudaStream_t st, bool fuse_dots = false, bool init = false,
                               int part = 0) {
  const MapDesc& M = pl.hmaps[0];
  if (kind == ULP_PRECOND_DCT) return dct_apply(*pl.dct, M.f.r, M.pitch, M.f.mask, M.f.s, st, true);
  if (kind == ULP_PRECOND_MG)
    return mg_apply(*pl.mg, M.f.mask, pl.dstate, st, true, fuse_dots ? pl.dargs : nullptr,
                    mixed_fcg(pl, kind) ? M.h.s : nullptr, init, part);
  if (kind == ULP_PRECOND_RBSSOR || kind == ULP_PRECOND_RBILU) return rb_apply(pl, kind, pl.dstate, st);
  const cudaError_t e = unet_apply_plane(*pl.unet, M.f.r, M.f.U, M.f.V, M.f.mask, M.H, M.W, M.pitch, M.f.s,
                                         &pl.dstate[0].fallback, st);
  if (e != cudaSuccess) return e;
  k_f_jacobi<<<tile_blocks(pl), kThreads, 0, st>>>(pl.dargs);
  return cudaGetLastError();
}

// D rides on the multigrid cycle's last kernel where the plan allows it
static bool fused_dots(const Plan& pl, int kind) { return kind == ULP_PRECOND_MG && mg_fuses_dots(*pl.mg); }

// Start of a solve: r = b - A phi (and its BF16 copy), the mask bits, s = M^-1 r, delta_0.
static cudaError_t fcg_start(Plan& pl, int kind, cudaStream_t st) {
  const MapDesc& M = pl.hmaps[0];
  const int nb = tile_blocks(pl);
  const bool stamp = pl.opt.profile != 0;
  if (mixed_fcg(pl, kind)) {
    const bool fd = fused_dots(pl, kind);
    k_x_res<<<nb, kThreads, 0, st>>>(pl.dargs, 1);
    if (stamp) k_setup_stamp<<<1, 1, 0, st>>>(pl.dargs, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = mg_setup(*pl.mg, pl.dstate, st, !pl.system_x);
    if (stamp) k_setup_stamp<<<1, 1, 0, st>>>(pl.dargs, 1);
    if (e == cudaSuccess) e = fcg_precond(pl, kind, st, fd, true);
    if (!fd) k_x_dots<<<nb, kThreads, 0, st>>>(pl.dargs, 1);
    return e == cudaSuccess ? cudaGetLastError() : e;
  }
  k_f_res<<<nb, kThreads, 0, st>>>(pl.dargs, 0);
  if (stamp) k_setup_stamp<<<1, 1, 0, st>>>(pl.dargs, 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && kind == ULP_PRECOND_DCT) e = dct_prepare_mask(*pl.dct, M.f.mask, M.pitch, st);
  if (e == cudaSuccess && kind == ULP_PRECOND_MG) e = mg_setup(*pl.mg, pl.dstate, st);
  if (e == cudaSuccess) e = rb_setup(pl, kind, pl.dstate, st);
  if (stamp) k_setup_stamp<<<1, 1, 0, st>>>(pl.dargs, 1);
  if (e == cudaSuccess) e = fcg_precond(pl, kind, st);
  k_f_dots<<<nb, kThreads, 0, st>>>(pl.dargs, 1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// One iteration: A, B, R, s = M^-1 r, D.
static cudaError_t fcg_iteration(Plan& pl, int kind, cudaStream_t st) {
  const int nb = tile_blocks(pl);
  const bool fd = fused_dots(pl, kind);
  if (mixed_fcg(pl, kind)) {
    k_x_a<<<nb, kThreads, 0, st>>>(pl.dargs);
    k_x_b<<<nb, kThreads, kRingBSmem, st>>>(pl.dargs);
    k_x_res<<<nb, kThreads, 0, st>>>(pl.dargs, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = fcg_precond(pl, kind, st, fd);
    if (!fd) k_x_dots<<<nb, kThreads, 0, st>>>(pl.dargs, 0);
    return e == cudaSuccess ? cudaGetLastError() : e;
  }
  k_f_a<<<nb, kThreads, 0, st>>>(pl.dargs);
  k_f_b<<<nb, kThreads, kRingFSmem, st>>>(pl.dargs);
  k_f_res<<<nb, kThreads, 0, st>>>(pl.dargs, 1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = fcg_precond(pl, kind, st, fd);
  if (!fd) k_f_dots<<<nb, kThreads, 0, st>>>(pl.dargs, 0);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// Dynamic shared memory above 48 KB is an attribute of the function on the current device.
static cudaError_t fcg_attrs() {
  const cudaError_t e = cudaFuncSetAttribute(k_f_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingFSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_x_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBSmem);
}

// Captures the solve graph: start, then WHILE { guard, iteration }.
static cudaError_t fcg_build(Plan& pl, int kind) {
  cudaError_t e = fcg_attrs();
  if (e != cudaSuccess) return e;
  if (!pl.cap_stream) {
    e = cudaStreamCreateWithFlags(&pl.cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  cudaStream_t st = pl.cap_stream;
  cudaGraph_t g = nullptr;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  pl.fcg_cond = h;
  cudaGraphNodeParams cp = {};
  if ((e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  e = fcg_start(pl, kind, st);
  k_f_guard<<<1, 1, 0, st>>>(pl.dargs, 0);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
  cudaGraphNode_t cn = nullptr;
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&cn, g, deps, nullptr, ndeps, &cp);
  }
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(st, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess && mixed_fcg(pl, kind)) {
    k_x_fold<<<tile_blocks(pl), kThreads, 0, st>>>(pl.dargs);
    e = cudaGetLastError();
  }
  cudaGraph_t gout = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &gout);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) ==
      cudaSuccess) {
    k_f_guard<<<1, 1, 0, st>>>(pl.dargs, 1);
    e = fcg_iteration(pl, kind, st);
    cudaGraph_t bout = nullptr;
    const cudaError_t e3 = cudaStreamEndCapture(st, &bout);
    if (e == cudaSuccess) e = e3;
  }
  // kernel counts of the start and of one loop body (every captured node is a kernel,
  // except the conditional node itself)
  size_t n_all = 0, n_body = 0;
  if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &n_all);
  if (e == cudaSuccess) e = cudaGraphGetNodes(body, nullptr, &n_body);
  pl.fcg_start_kernels = (long long)n_all - 1;
  pl.fcg_body_kernels = (long long)n_body;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&pl.fcg_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) pl.fcg_exec = nullptr;
  else {
    pl.fcg_kind = kind;
    if (kind == ULP_PRECOND_LEARNED) pl.fcg_gen = unet_ws_gen(*pl.unet);
  }
  return e;
}

// Host-driven form of the same solve (options.profile = 2): every kernel is a
// host launch, so a profiler sees each one; the host reads the stop flag after
// every iteration.  For measurement only.
static cudaError_t fcg_eager_mixed(Plan& pl, int kind, cudaStream_t st) {
  const int nb = tile_blocks(pl);
  const bool fd = fused_dots(pl, kind);
  cudaError_t e = fcg_attrs();
  if (e != cudaSuccess) return e;
  phase_mark(pl, st, -1);
  k_x_res<<<nb, kThreads, 0, st>>>(pl.dargs, 1);
  phase_mark(pl, st, 2);
  if ((e = mg_setup(*pl.mg, pl.dstate, st, !pl.system_x)) != cudaSuccess) return e;
  if ((e = fcg_precond(pl, kind, st, fd, true)) != cudaSuccess) return e;
  phase_mark(pl, st, 3);
  if (!fd) {
    k_x_dots<<<nb, kThreads, 0, st>>>(pl.dargs, 1);
    phase_mark(pl, st, 4);
  }
  for (long long l = 0;; ++l) {
    int done = 0;
    if ((e = cudaMemcpyAsync(&done, &pl.dstate->done, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (done || l > (1LL << 24)) break;
    phase_mark(pl, st, -1);
    k_x_a<<<nb, kThreads, 0, st>>>(pl.dargs);
    phase_mark(pl, st, 0);
    k_x_b<<<nb, kThreads, kRingBSmem, st>>>(pl.dargs);
    phase_mark(pl, st, 1);
    k_x_res<<<nb, kThreads, 0, st>>>(pl.dargs, 0);
    phase_mark(pl, st, 2);
    if ((e = fcg_precond(pl, kind, st, fd, false, 1)) != cudaSuccess) return e;
    phase_mark(pl, st, 3);
    if ((e = fcg_precond(pl, kind, st, fd, false, 2)) != cudaSuccess) return e;
    phase_mark(pl, st, 5);
    if (!fd) {
      k_x_dots<<<nb, kThreads, 0, st>>>(pl.dargs, 0);
      phase_mark(pl, st, 4);
    }
  }
  k_x_fold<<<nb, kThreads, 0, st>>>(pl.dargs);
  return cudaGetLastError();
}

static cudaError_t fcg_eager(Plan& pl, int kind, cudaStream_t st) {
  if (mixed_fcg(pl, kind)) return fcg_eager_mixed(pl, kind, st);
  const MapDesc& M = pl.hmaps[0];
  const int nb = tile_blocks(pl);
  cudaError_t e = fcg_attrs();
  if (e != cudaSuccess) return e;
  phase_mark(pl, st, -1);
  k_f_res<<<nb, kThreads, 0, st>>>(pl.dargs, 0);
  phase_mark(pl, st, 2);
  if (kind == ULP_PRECOND_DCT) e = dct_prepare_mask(*pl.dct, M.f.mask, M.pitch, st);
  if (e == cudaSuccess && kind == ULP_PRECOND_MG) e = mg_setup(*pl.mg, pl.dstate, st);
  if (e == cudaSuccess) e = rb_setup(pl, kind, pl.dstate, st);
  if (e == cudaSuccess) e = fcg_precond(pl, kind, st);
  if (e != cudaSuccess) return e;
  phase_mark(pl, st, 3);
  k_f_dots<<<nb, kThreads, 0, st>>>(pl.dargs, 1);
  phase_mark(pl, st, 4);
  for (long long l = 0;; ++l) {
    int done = 0;
    if ((e = cudaMemcpyAsync(&done, &pl.dstate->done, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (done || l > (1LL << 24)) break;
    phase_mark(pl, st, -1);
    k_f_a<<<nb, kThreads, 0, st>>>(pl.dargs);
    phase_mark(pl, st, 0);
    k_f_b<<<nb, kThreads, kRingFSmem, st>>>(pl.dargs);
    phase_mark(pl, st, 1);
    k_f_res<<<nb, kThreads, 0, st>>>(pl.dargs, 1);
    phase_mark(pl, st, 2);
    const bool fd = fused_dots(pl, kind);
    if (kind == ULP_PRECOND_MG) {
      if ((e = fcg_precond(pl, kind, st, fd, false, 1)) != cudaSuccess) return e;
      phase_mark(pl, st, 3);
      if ((e = fcg_precond(pl, kind, st, fd, false, 2)) != cudaSuccess) return e;
      phase_mark(pl, st, 5);
    } else {
      if ((e = fcg_precond(pl, kind, st, fd)) != cudaSuccess) return e;
      phase_mark(pl, st, 3);
    }
    if (!fd) {
      k_f_dots<<<nb, kThreads, 0, st>>>(pl.dargs, 0);
      phase_mark(pl, st, 4);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_fcg(Plan& pl, int kind, const PcgArgs& a_in, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  if (pl.nmaps != 1) return cudaErrorNotSupported;
  if (kind == ULP_PRECOND_DCT && !pl.dct) return cudaErrorNotSupported;
  if (kind == ULP_PRECOND_MG && !pl.mg) return cudaErrorNotSupported;
  if (kind == ULP_PRECOND_LEARNED) {
    if (!pl.unet) return cudaErrorNotSupported;
    const MapDesc& M = pl.hmaps[0];
    const int rc = unet_prepare(*pl.unet, 1, (M.H + 127) / 128 * 128, (M.W + 127) / 128 * 128);
    if (rc) return rc == -5 ? cudaErrorMemoryAllocation : cudaErrorUnknown;
  }
  PcgArgs a = a_in;
  a.rbf = nullptr;
  a.rbf_lo = nullptr;
  a.rbf_ld = 0;
  a.rf32 = nullptr;
  if (kind == ULP_PRECOND_DCT) a.rbf = dct_input(*pl.dct, &a.rbf_ld, &a.rbf_lo);
  a.xfcg = mixed_fcg(pl, kind);
  if (kind == ULP_PRECOND_MG && !a.xfcg) a.rf32 = mg_input(*pl.mg);
  a.learned = kind == ULP_PRECOND_LEARNED;
  if (pl.opt.profile == 2) {
    a.cond = 0;
    k_set_args<<<1, 1, 0, st>>>(a, pl.dargs);
    launch_pcg_reset(pl, st);
    if (e0) cudaEventRecord(e0, st);
    const cudaError_t e = fcg_eager(pl, kind, st);
    if (e == cudaSuccess && e1) cudaEventRecord(e1, st);
    return e;
  }
  if (pl.fcg_exec && (pl.fcg_kind != kind || (kind == ULP_PRECOND_LEARNED && pl.fcg_gen != unet_ws_gen(*pl.unet))))
    destroy_fcg(pl);
  if (!pl.fcg_exec) {
    const cudaError_t e = fcg_build(pl, kind);
    if (e != cudaSuccess) return e;
  }
  a.cond = pl.fcg_cond;
  pl.kernel_launches += 2;
  pl.solver_launches += 1;
  k_set_args<<<1, 1, 0, st>>>(a, pl.dargs);
  launch_pcg_reset(pl, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (e0) cudaEventRecord(e0, st);
  e = cudaGraphLaunch(pl.fcg_exec, st);
  if (e == cudaSuccess && e1) e = cudaEventRecord(e1, st);
  return e;
}

void destroy_fcg(Plan& pl) {
  if (pl.fcg_exec) cudaGraphExecDestroy(pl.fcg_exec);
  pl.fcg_exec = nullptr;
  pl.fcg_kind = -1;
}

}  // namespace ulp
