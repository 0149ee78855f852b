// ulp_engine.cuh -- pieces of the persistent PCG engine shared by the FP64 and
// mixed-precision solvers: the FP64 sliding-window stencil walker, tile
// geometry, and the per-map finisher that advances Algorithm 1's scalars
// (alpha, beta, delta, stop tests) from fixed-order sums of per-tile partials.
#pragma once
#include "ulp_internal.cuh"

namespace ulp {

// ------------------------------------------------------------------ stencil walker
// Sliding-window 5-point stencil over one warp tile (64 columns x rows i0..i1-1):
// each lane owns columns j, j+1; north/south neighbours come from the window,
// east/west from the neighbouring lanes, the two tile-edge columns from a halo
// load by lanes 0 and 31.  X supplies the vector being multiplied in two
// stages so that loads run one row ahead of the arithmetic:
//   X::Raw X::load(i, j)   -- the planes behind x at (i, j), (i, j+1)
//   double2 X::make(raw)   -- x itself
//   double X::at(i, c)     -- x at one column (halo lanes)
template <class X, class Epi>
__device__ __forceinline__ void stencil_tile(const MapDesc& M, int i0, int i1, int j0, int lane,
                                             const double* U, const double* V, const double* D,
                                             const X& x, Epi& epi) {
  using Raw = typename X::Raw;
  const int j = j0 + 2 * lane;
  const bool hw = (lane == 0) && (j0 > 0);
  const bool he = (lane == 31) && (j0 + kStrip < M.pitch);
  const bool halo = hw || he;
  const int hc = (lane == 0) ? j0 - 1 : j0 + kStrip;
  const size_t P = (size_t)M.pitch;
  const double2 z2 = make_double2(0.0, 0.0);
  double2 xn = z2, vn = z2;
  if (i0 > 0) {
    xn = x.make(x.load(i0 - 1, j));
    vn = ld2(V, (size_t)(i0 - 1) * P + j);
  }
  double2 xc = x.make(x.load(i0, j));
  Raw rs = (i0 + 1 < M.H) ? x.load(i0 + 1, j) : X::zero();   // row i+1, raw
  size_t off = (size_t)i0 * P + j;
  double2 u = ld2(U, off), v = ld2(V, off), dd = ld2(D, off);
  double h = halo ? x.at(i0, hc) : 0.0;
  double uwh = hw ? ld1(U, (size_t)i0 * P + hc) : 0.0;
  for (int i = i0; i < i1; ++i) {
    // loads for the next row, issued before this row's arithmetic
    const bool more = i + 1 < i1;
    const size_t off2 = off + P;
    Raw rs2 = (more && i + 2 < M.H) ? x.load(i + 2, j) : X::zero();
    double2 u2 = z2, v2 = z2, dd2 = z2;
    double h2 = 0.0, uwh2 = 0.0;
    if (more) {
      u2 = ld2(U, off2);
      v2 = ld2(V, off2);
      dd2 = ld2(D, off2);
      if (halo) h2 = x.at(i + 1, hc);
      if (hw) uwh2 = ld1(U, (size_t)(i + 1) * P + hc);
    }
    const double2 xs = (i + 1 < M.H) ? x.make(rs) : z2;
    double west = __shfl_up_sync(kFull, xc.y, 1);
    double east = __shfl_down_sync(kFull, xc.x, 1);
    double uw = __shfl_up_sync(kFull, u.y, 1);
    if (lane == 0) { west = h; uw = uwh; }
    if (lane == 31) east = h;
    double2 ax;
    ax.x = dd.x * xc.x;
    ax.x = fma(-u.x, xc.y, ax.x);
    ax.x = fma(-uw, west, ax.x);
    ax.x = fma(-v.x, xs.x, ax.x);
    ax.x = fma(-vn.x, xn.x, ax.x);
    ax.y = dd.y * xc.y;
    ax.y = fma(-u.y, east, ax.y);
    ax.y = fma(-u.x, xc.x, ax.y);
    ax.y = fma(-v.y, xs.y, ax.y);
    ax.y = fma(-vn.y, xn.y, ax.y);
    epi(off, xc, ax);
    xn = xc;
    xc = xs;
    vn = v;
    rs = rs2;
    u = u2;
    v = v2;
    dd = dd2;
    h = h2;
    uwh = uwh2;
    off = off2;
  }
}

struct XPlane {  // plain vector
  const double* x;
  size_t P;
  using Raw = double2;
  __device__ __forceinline__ static Raw zero() { return make_double2(0.0, 0.0); }
  __device__ __forceinline__ Raw load(int i, int j) const { return ld2(x, (size_t)i * P + j); }
  __device__ __forceinline__ double2 make(const Raw& r) const { return r; }
  __device__ __forceinline__ double at(int i, int c) const { return ld1(x, (size_t)i * P + c); }
};

struct XDir {  // d = s + beta d_old, or d = s on the first iteration (Algorithm 1)
  const double* s;
  const double* dold;
  double beta;
  bool first;
  size_t P;
  struct Raw {
    double2 s, d;
  };
  __device__ __forceinline__ static Raw zero() { return Raw{make_double2(0.0, 0.0), make_double2(0.0, 0.0)}; }
  __device__ __forceinline__ Raw load(int i, int j) const {
    const size_t off = (size_t)i * P + j;
    Raw r;
    r.s = ld2(s, off);
    r.d = first ? make_double2(0.0, 0.0) : ld2(dold, off);
    return r;
  }
  __device__ __forceinline__ double2 make(const Raw& r) const {
    if (first) return r.s;
    return make_double2(fma(beta, r.d.x, r.s.x), fma(beta, r.d.y, r.s.y));
  }
  __device__ __forceinline__ double at(int i, int c) const {
    const size_t off = (size_t)i * P + c;
    const double sv = ld1(s, off);
    return first ? sv : fma(beta, ld1(dold, off), sv);
  }
};

struct TileGeo {
  int i0, i1, j0;
};
__device__ __forceinline__ TileGeo tile_geo(const MapDesc& M, int t, int R) {
  const int lt = t - M.tile_base;
  const int sy = lt / M.nsx, sx = lt - sy * M.nsx;
  TileGeo g;
  g.i0 = sy * R;
  g.i1 = min(g.i0 + R, M.H);
  g.j0 = sx * kStrip;
  return g;
}

// ------------------------------------------------------------------ PCG engine
// kPhConfirm: the true residual of a mixed flexible-CG confirmation body (its r^T r alone)
enum Phase { kPhResInit = 0, kPhA = 1, kPhB = 2, kPhRes = 3, kPhFcg = 4, kPhConfirm = 5 };

// Runs in the warp whose tile arrival completed phase `ph` for map m: reduces
// the map's tile partials in a fixed order and advances its scalars
// (alpha = delta_new / d^T q; delta_old, delta_new, beta; stop tests).
// ngroups: how many group sums the arrival left (0: as many as the map's tiles make).
// The finisher is the serial tail of its kernel (every other warp has left), so it is
// built as few dependent memory round trips as possible: lane 0 loads every field of
// the map's state it reads in the same round of L2 loads as the group sums (only the
// finisher writes these fields, and every tile of the phase has arrived), works in
// registers, and stores.  No fence closes it: the next phase reads the state after a
// kernel boundary or after the grid barrier that follows every phase of the persistent
// kernels (whose leading __syncthreads and fence cover this warp's stores).
static_assert(kArriveGroups <= 32, "one lane per arrival group");
__device__ __forceinline__ void finish_map(const PcgArgs& a, const MapDesc& M, MapState* Sp, int ph, int lane,
                                           int ngroups = 0) {
  volatile MapState* S = Sp;
  // the per-group sums in group order, then a fixed shuffle tree
  const int n = M.ntiles;
  const int ng = ngroups > 0 ? ngroups : (n < kArriveGroups ? n : kArriveGroups);
  const int cnt = (ph == kPhA) ? 1 : (ph == kPhResInit || ph == kPhFcg) ? 3 : 2;
  const bool own = lane < ng;
  // L2 loads: another warp wrote them, and this SM's L1 may hold an older phase's values
  double v0 = own ? __ldcg(&Sp->gpart[0][lane]) : 0.0;
  double v1 = (own && cnt > 1) ? __ldcg(&Sp->gpart[1][lane]) : 0.0;
  double v2 = (own && cnt > 2) ? __ldcg(&Sp->gpart[2][lane]) : 0.0;
  double delta = 0.0, delta0 = 0.0, bb = 0.0, rr_best = 0.0;
  long long iter = 0;
  int fallback = 0, restart = 0, stall = 0, force_refresh = 0, stop_after = 0, confirm = 0, refresh_next = 0;
  double rr_ref = 0.0;
  if (lane == 0) {
    delta = __ldcg(&Sp->delta);
    delta0 = __ldcg(&Sp->delta0);
    bb = __ldcg(&Sp->bb);
    rr_best = __ldcg(&Sp->rr_best);
    iter = __ldcg(&Sp->iter);
    fallback = __ldcg(&Sp->fallback);
    restart = __ldcg(&Sp->restart);
    stall = __ldcg(&Sp->stall);
    force_refresh = __ldcg(&Sp->force_refresh);
    stop_after = __ldcg(&Sp->stop_after);
    confirm = __ldcg(&Sp->confirm);
    refresh_next = __ldcg(&Sp->refresh_next);
    rr_ref = __ldcg(&Sp->rr_ref);
  }
  v0 = warp_sum(v0);
  v1 = cnt > 1 ? warp_sum(v1) : 0.0;
  v2 = cnt > 2 ? warp_sum(v2) : 0.0;
  bool done = false;
  if (lane == 0) {
    bool refreshed = true;  // r is the true residual (mixed flexible CG: this iteration recomputed it)
    if (ph == kPhConfirm) {
      // the recurrence called the current iterate converged and this body recomputed its
      // residual in FP64: if that meets the tolerance the solve stops here, before the
      // preconditioner runs; otherwise the body goes on (the cycle and the dot phase treat
      // it as a confirmation that missed)
      if (!(v1 > a.tol2 * bb)) {
        done = true;
        S->status = 0;
        S->x_clean = 1;
        S->confirm = 0;
        S->rr = v1;
        S->relres = (bb > 0.0) ? sqrt(v1 / bb) : 0.0;
      }
    } else if (ph == kPhA) {
      S->dq = v0;
      if ((!(v0 > 0.0) || !isfinite(v0)) && a.learned && !fallback) {
        // the network gave a direction that is not a descent direction: no step,
        // Jacobi from now on, and the next direction restarts (beta = 0)
        S->alpha = 0.0;
        S->fallback = 1;
        S->restart = 1;
      } else if (!(v0 > 0.0) || !isfinite(v0)) {  // breakdown: stop after this iteration
        S->status = -3;
        S->alpha = 0.0;
        S->stop_after = 1;
      } else {
        S->alpha = delta / v0;
      }
    } else {
      const double rr = v1;
      if (ph == kPhResInit) {
        delta = v0;
        delta0 = v0;
        bb = v2;
        iter = 0;
        S->delta = v0;
        S->delta0 = v0;
        S->rr = v1;
        S->bb = v2;
        S->iter = 0;
        S->rr_best = v1;
        S->rr_ref = v1;
        S->refresh_next = 0;
        S->stall = 0;
      } else if (ph == kPhFcg) {
        // flexible CG (Polak-Ribiere): beta = r_{k+1}^T (s_{k+1} - s_k) / (r_k^T s_k), v2 = r_{k+1}^T s_k
        refreshed = (a.xfcg ? (iter > 0 && (iter % M.refresh) == 0) : (iter % M.refresh) == 0) || force_refresh ||
                    confirm || refresh_next;
        if (a.xfcg) {
          // mixed: r^T r of the last true residual, and a refresh once ||r|| has fallen 100-fold since
          S->refresh_next = (!refreshed && v1 < 1e-4 * rr_ref) ? 1 : 0;
          if (refreshed) S->rr_ref = v1;
        }
        if (confirm) {
          // mixed flexible CG: this body took no step; it folded the correction into phi and
          // recomputed r and s for the same iterate, so the iteration count and beta (the
          // recurrence's) stay, and delta becomes r^T s of the recomputed pair
          delta = v0;
          S->delta = v0;
          S->rr = v1;
          S->confirm = 0;
        } else {
          const double dold = delta;
          delta = v0;
          iter += 1;
          S->delta = v0;
          S->rr = v1;
          S->beta = restart ? 0.0 : (v0 - v2) / dold;
          S->restart = 0;
          S->iter = iter;
        }
        if (a.learned && !fallback) {
          // progress test: ||r|| must halve (||r||^2 quarter) within every stall_window
          // iterations, measured from the last point where it did
          if (v1 < 0.25 * rr_best) {
            S->rr_best = v1;
            S->stall = 0;
          } else {
            S->stall = stall + 1;
            if (stall + 1 >= a.stall_window || !(v0 > 0.0)) {
              S->fallback = 1;  // the next s is D^-1 r and the direction restarts from it
              S->restart = 1;
            }
          }
        }
      } else {
        const double dold = delta;
        delta = v0;
        iter += 1;
        S->delta = v0;
        S->rr = v1;
        S->beta = v0 / dold;
        S->iter = iter;
      }
      const double tol2 = a.tol2;
      const bool conv = (a.stop_mode == 1) ? !(delta > tol2 * delta0) : !(rr > tol2 * bb);
      S->relres = (bb > 0.0) ? sqrt(rr / bb) : 0.0;
      if (stop_after) {
        done = true;
      } else if (bb == 0.0 || conv) {
        if (ph == kPhFcg && a.xfcg && !refreshed && bb != 0.0) {
          // the FP32 recurrence says converged at this iterate, the point where Algorithm 1
          // stops on its recurrence residual: the next body takes no step, folds the correction
          // into phi and tests the FP64 true residual of this same iterate
          S->confirm = 1;
        } else {
          done = true;
          S->status = 0;
          if (ph == kPhFcg && a.xfcg && refreshed) S->x_clean = 1;  // this iteration folded x into phi
        }
      } else if (ph == kPhFcg && a.xfcg && confirm) {
        // the true residual of the iterate the recurrence called converged misses the
        // tolerance: from here on every iteration recomputes it, and the solve stops on that
        S->force_refresh = 1;
      } else if (ph == kPhFcg && a.xfcg && !force_refresh && bb != 0.0 &&
                 ((a.stop_mode == 1) ? !(delta > 4.0 * tol2 * delta0) : !(rr > 4.0 * tol2 * bb))) {
        // within a factor 2 of the tolerance: the iterates that follow recompute the true
        // residual after their step and stop on it, so the stop falls on the first iterate
        // whose FP64 residual meets the tolerance, where an FP64 recurrence stops, even
        // when the FP32 recurrence lags it by a rounding
        S->force_refresh = 1;
      } else if (iter >= (a.lmax > 0 ? a.lmax : 2LL * M.H * M.W)) {
        done = true;
        S->status = 1;
      }
    }
    S->arrive = 0u;
  }
  // the arrival counters back to zero, one lane per group
  if (lane < kArriveGroups) S->arrive_grp[lane] = 0u;
  __syncwarp();
  if (lane == 0 && done) {
    S->done = 1;
    __threadfence();
    atomicSub(a.n_active, 1);
    if (a.cond) cudaGraphSetConditional(a.cond, 0);  // ends the graph's WHILE loop
  }
  __syncwarp();
}

// Publishes this warp's tile partials and runs the map's finisher if this was
// the last tile of the map in this phase.  Arrival is counted in two levels so
// that no counter takes more than about ntiles / 32 atomics: tile t counts into
// group g = (t - tile_base) mod 32, and the last tile of each group counts into
// the map's counter.  The counts are acquire-release atomics at GPU scope: the
// release orders this warp's partial stores before its count, the acquire of
// the group's last count (and of the map's) makes every earlier count's stores
// visible to it, and __syncwarp passes that on to the finisher's other lanes.
// The reduction is hierarchical for the same reason: the last tile of each
// group sums that group's partials (the groups in parallel), and the finisher
// reads only the 32 group sums; a single warp summing all 2432 tile partials
// in fixed-order rounds of L2 loads took about 20 us per phase on GB300.
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void tile_arrive(const PcgArgs& a, const MapDesc& M, MapState* S, int t,
                                            int ph, double v0, double v1, double v2, int lane) {
  v0 = warp_sum(v0);
  if (ph != kPhA) v1 = warp_sum(v1);
  if (ph == kPhResInit) v2 = warp_sum(v2);
  const int base = M.tile_base, n = M.ntiles;
  const int ng = n < kArriveGroups ? n : kArriveGroups;
  const int g = (t - base) % kArriveGroups;
  const int gsize = (n - g + kArriveGroups - 1) / kArriveGroups;
  int glast = 0;
  if (lane == 0) {
    __stcg(a.P0 + t, v0);
    if (ph != kPhA) __stcg(a.P1 + t, v1);
    if (ph == kPhResInit) __stcg(a.P2 + t, v2);  // kPhFcg: P2 holds r_{k+1}^T s_k from phase B
    glast = atom_add_acq_rel(&S->arrive_grp[g], 1u) == (unsigned)gsize - 1u;
  }
  glast = __shfl_sync(kFull, glast, 0);
  if (!glast) return;
  // the group's last tile sums the group's partials (tiles base + g + 32 m, m in order of
  // lanes then of the stride loop, then a fixed shuffle tree) in parallel with the other groups
  __syncwarp();
  const int cnt = (ph == kPhA) ? 1 : (ph == kPhResInit || ph == kPhFcg) ? 3 : 2;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll 4
  for (int m = lane; m < gsize; m += 32) {
    const int idx = base + g + kArriveGroups * m;
    s0 += __ldcg(a.P0 + idx);
    if (cnt > 1) s1 += __ldcg(a.P1 + idx);
    if (cnt > 2) s2 += __ldcg(a.P2 + idx);
  }
  s0 = warp_sum(s0);
  if (cnt > 1) s1 = warp_sum(s1);
  if (cnt > 2) s2 = warp_sum(s2);
  int last = 0;
  if (lane == 0) {
    volatile double* gp = &S->gpart[0][0];
    gp[0 * kArriveGroups + g] = s0;
    if (cnt > 1) gp[1 * kArriveGroups + g] = s1;
    if (cnt > 2) gp[2 * kArriveGroups + g] = s2;
    last = atom_add_acq_rel(&S->arrive, 1u) == (unsigned)ng - 1u;
  }
  last = __shfl_sync(kFull, last, 0);
  if (last) {
    __syncwarp();
    finish_map(a, M, S, ph, lane);
  }
}

// Arrival of the flexible-CG dot phase from a kernel that covers the map with its
// own decomposition into n warps (32 <= n <= the map's tile count), warp w: its
// r^T s and r^T r go to P0, P1 at tile_base + w and count as above with n in
// place of the tile count; the third sum's partials (r_{k+1}^T s_k left by phase B,
// or b^T b at the start of a solve, ph = kPhResInit) are indexed by the map's
// tiles, so the last warp of group g sums P2 over the map's tiles of group g.
// Same fixed summation order on every run.
// rr_tiles: r^T r comes, like the third sum, as per-tile partials in P1 (left by the
// kernels that wrote r) instead of from this kernel.
__device__ __forceinline__ void warp_arrive_fcg(const PcgArgs& a, const MapDesc& M, MapState* S, int w, int n,
                                                double rs, double rr, int lane, int ph = kPhFcg,
                                                bool rr_tiles = false) {
  rs = warp_sum(rs);
  if (!rr_tiles) rr = warp_sum(rr);
  const int base = M.tile_base;
  const int g = w % kArriveGroups;
  const int gsize = (n - g + kArriveGroups - 1) / kArriveGroups;
  const int gsize2 = g < M.ntiles ? (M.ntiles - g + kArriveGroups - 1) / kArriveGroups : 0;
  int glast = 0;
  if (lane == 0) {
    __stcg(a.P0 + base + w, rs);
    if (!rr_tiles) __stcg(a.P1 + base + w, rr);
    glast = atom_add_acq_rel(&S->arrive_grp[g], 1u) == (unsigned)gsize - 1u;
  }
  glast = __shfl_sync(kFull, glast, 0);
  if (!glast) return;
  __syncwarp();
  // one loop over both index ranges, so that all of a lane's loads are in flight together
  // (each sum still runs over its own range in the same order)
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  const int gmax = gsize > gsize2 ? gsize : gsize2;
#pragma unroll 4
  for (int m = lane; m < gmax; m += 32) {
    const int idx = base + g + kArriveGroups * m;
    if (m < gsize) {
      s0 += __ldcg(a.P0 + idx);
      if (!rr_tiles) s1 += __ldcg(a.P1 + idx);
    }
    if (m < gsize2) {
      s2 += __ldcg(a.P2 + idx);
      if (rr_tiles) s1 += __ldcg(a.P1 + idx);
    }
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  int last = 0;
  if (lane == 0) {
    volatile double* gp = &S->gpart[0][0];
    gp[0 * kArriveGroups + g] = s0;
    gp[1 * kArriveGroups + g] = s1;
    gp[2 * kArriveGroups + g] = s2;
    last = atom_add_acq_rel(&S->arrive, 1u) == (unsigned)kArriveGroups - 1u;
  }
  last = __shfl_sync(kFull, last, 0);
  if (last) {
    __syncwarp();
    finish_map(a, M, S, ph, lane, kArriveGroups);
  }
}

// d = s + beta d_old, q = A d, partial d^T q (Algorithm 1: q <- A d, d^T q).
template <int KIND>
__device__ __forceinline__ void a_tile(const PcgArgs& a, const MapDesc& M, MapState* S, int t, int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  const size_t P = M.pitch;
  const long long it = *(volatile long long*)&S->iter;
  const double* sv = (KIND == kIdentity) ? M.f.r : M.f.s;
  const double* dold = (it & 1) ? M.f.d1 : M.f.d0;
  double* dnew = (it & 1) ? M.f.d0 : M.f.d1;
  XDir x{sv, dold, *(volatile double*)&S->beta, it == 0, P};
  double dq = 0.0;
  auto epi = [&](size_t off, double2 xc, double2 ax) {
    st2(dnew, off, xc);
    st2(M.f.q, off, ax);
    dq = fma(xc.x, ax.x, dq);
    dq = fma(xc.y, ax.y, dq);
  };
  stencil_tile(M, g.i0, g.i1, g.j0, lane, M.f.U, M.f.V, M.f.D, x, epi);
  tile_arrive(a, M, S, t, kPhA, dq, 0.0, 0.0, lane);
}

}  // namespace ulp
