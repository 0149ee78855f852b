// ulp_fp64.cu -- FP64 kernels of Algorithm 1 (arXiv 2203.13675):
//   wrapped differences (Sec. 2.1), weights (Eq. UV), system (Eq. Axb),
//   the persistent PCG engine (Algorithm 1 inner loop) for M = I and
//   M = diag(A), the outer error (Algorithm 1), and single-step kernels.
#include "ulp_internal.cuh"
#include "ulp_host.h"
#include "ulp_sweep.cuh"
#include "ulp_engine.cuh"

#include <math.h>

namespace ulp {

// ------------------------------------------------------------------ pack
// Sec. 2.1: Delta^x = W(psi_{i,j+1} - psi_{i,j}) (j <= W-2), Delta^y likewise
// along i; ghost entries 0.  Also copies the mask and phi^0 into the padded
// planes and checks that psi is finite.
__global__ void k_pack(MapDesc M, MapState* S, const double* __restrict__ psi,
                       const uint8_t* __restrict__ mask, const double* __restrict__ phi0) {
  const size_t n = (size_t)M.H * M.pitch;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((unsigned)t / (unsigned)M.pitch), j = (int)((unsigned)t - (unsigned)i * (unsigned)M.pitch);
    double dx = 0.0, dy = 0.0, ph = 0.0;
    uint8_t mk = 0;
    if (j < M.W) {
      const size_t k = (size_t)i * M.W + j;
      const double c = psi[k];
      if (!isfinite(c)) atomicExch(&S->err_flag, 1);
      if (j + 1 < M.W) dx = wrap_pv(__dsub_rn(psi[k + 1], c));
      if (i + 1 < M.H) dy = wrap_pv(__dsub_rn(psi[k + M.W], c));
      if (mask) mk = mask[k] ? 1 : 0;
      if (phi0) ph = phi0[k];
    }
    M.f.dx[t] = dx;
    M.f.dy[t] = dy;
    M.f.mask[t] = mk;
    M.f.phi[t] = ph;
  }
}

__global__ void k_unpack(MapDesc M, double* __restrict__ phi) {
  const size_t n = (size_t)M.H * M.W;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((unsigned)k / (unsigned)M.W), j = (int)((unsigned)k - (unsigned)i * (unsigned)M.W);
    phi[k] = M.f.phi[(size_t)i * M.pitch + j];
  }
}

// ------------------------------------------------------------------ weights
// Eq. (UV): w(e) = tau / (|e|^(2-p) + tau), with the exponent specialised for
// p in {0, 1, 2}.  Zero on edges leaving the grid or touching a masked pixel.
__device__ __forceinline__ double irls_weight(double e, double p, double tau, int pcase) {
  const double a = fabs(e);
  double t;
  switch (pcase) {
    case 2: t = 1.0; break;                 // p = 2: |e|^0 = 1
    case 1: t = a; break;                   // p = 1
    case 0: t = __dmul_rn(a, a); break;     // p = 0
    default: t = pow(a, 2.0 - p); break;
  }
  return __ddiv_rn(tau, __dadd_rn(t, tau));
}

__device__ __forceinline__ int p_case(double p) {
  return (p == 2.0) ? 2 : (p == 1.0) ? 1 : (p == 0.0) ? 0 : -1;
}

// One outer pass, first half: U, V from phi^k, and phi_prev = phi^k.
__global__ void k_weights(const MapDesc* __restrict__ maps, MapState* S, const double* __restrict__ pv,
                          const double* __restrict__ tauv) {
  const int m = blockIdx.y;
  const MapDesc& M = maps[m];
  if (!S[m].outer_active) return;
  const double p = pv[m], tau = tauv[m];
  const int pc = p_case(p);
  const size_t n = (size_t)M.H * M.pitch;
  const size_t P = M.pitch;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((unsigned)t / (unsigned)P), j = (int)((unsigned)t - (unsigned)i * (unsigned)P);
    const double ph = M.f.phi[t];
    const bool mk = M.f.mask[t] != 0;
    double u = 0.0, v = 0.0;
    if (j + 1 < M.W && !mk && !M.f.mask[t + 1]) {
      const double e = __dsub_rn(__dsub_rn(M.f.phi[t + 1], ph), M.f.dx[t]);
      u = irls_weight(e, p, tau, pc);
    }
    if (j < M.W && i + 1 < M.H && !mk && !M.f.mask[t + P]) {
      const double e = __dsub_rn(__dsub_rn(M.f.phi[t + P], ph), M.f.dy[t]);
      v = irls_weight(e, p, tau, pc);
    }
    M.f.U[t] = u;
    M.f.V[t] = v;
    M.f.phi_prev[t] = ph;
  }
}

// One outer pass, second half: diagonal D, its guarded inverse, and b (Eq. Axb),
// summed in the order the equation writes them.
__global__ void k_system(const MapDesc* __restrict__ maps, MapState* S) {
  const int m = blockIdx.y;
  const MapDesc& M = maps[m];
  if (!S[m].outer_active) return;
  const size_t n = (size_t)M.H * M.pitch;
  const size_t P = M.pitch;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((unsigned)t / (unsigned)P), j = (int)((unsigned)t - (unsigned)i * (unsigned)P);
    const double uw = (j > 0) ? M.f.U[t - 1] : 0.0;
    const double ue = M.f.U[t];
    const double vn = (i > 0) ? M.f.V[t - P] : 0.0;
    const double vs = M.f.V[t];
    const double d = __dadd_rn(__dadd_rn(__dadd_rn(uw, ue), vn), vs);
    double bk = 0.0;
    if (j > 0) bk = __dadd_rn(bk, __dmul_rn(M.f.dx[t - 1], uw));
    bk = __dsub_rn(bk, __dmul_rn(M.f.dx[t], ue));
    if (i > 0) bk = __dadd_rn(bk, __dmul_rn(M.f.dy[t - P], vn));
    bk = __dsub_rn(bk, __dmul_rn(M.f.dy[t], vs));
    M.f.D[t] = d;
    M.f.Dinv[t] = (d > 0.0) ? __drcp_rn(d) : 0.0;
    M.f.b[t] = bk;
  }
}

// ------------------------------------------------------------------ mixed multigrid system
// The mixed-precision multigrid form takes Eq. (UV)'s weights in FP32: the edge
// residual e is formed in FP64 from the FP64 phi, the weight tau / (|e|^(2-p) + tau)
// in FP32.  They are written as the FP32 planes that the FP32 stencil and the
// V-cycle read, and as their exact FP64 promotions, from which D (their FP64 sum,
// exact) and b follow as in k_system for the FP64 true residual; D^-1 is FP32.
// Two pixels per thread.
__device__ __forceinline__ float irls_weight32(double e, float p, float tau, int pcase) {
  const float a = fabsf((float)e);
  float t;
  switch (pcase) {
    case 2: t = 1.f; break;
    case 1: t = a; break;
    case 0: t = __fmul_rn(a, a); break;
    default: t = powf(a, 2.f - p); break;
  }
  return __fdiv_rn(tau, __fadd_rn(t, tau));
}

__global__ void k_weights_x(const MapDesc* __restrict__ maps, MapState* S, const double* __restrict__ pv,
                            const double* __restrict__ tauv) {
  const MapDesc& M = maps[0];
  if (!S[0].outer_active) return;
  const float p = (float)pv[0], tau = (float)tauv[0];
  const int pc = p_case(pv[0]);
  const unsigned half = (unsigned)M.pitch / 2u;
  const size_t n = (size_t)M.H * half;
  const size_t P = M.pitch;
  for (size_t t2 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t2 < n; t2 += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((unsigned)t2 / half), j = 2 * (int)((unsigned)t2 - (unsigned)i * half);
    const size_t o = (size_t)i * P + j;
    const double2 ph = ld2(M.f.phi, o);
    float2 u = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f);
    if (j < M.W) {
      const double2 dxv = ld2(M.f.dx, o);
      const bool m0 = M.f.mask[o] != 0, m1 = M.f.mask[o + 1] != 0;
      // east edges of (i, j) and (i, j+1)
      if (j + 1 < M.W && !m0 && !m1) u.x = irls_weight32(__dsub_rn(__dsub_rn(ph.y, ph.x), dxv.x), p, tau, pc);
      if (j + 2 < M.W && !m1 && !M.f.mask[o + 2])
        u.y = irls_weight32(__dsub_rn(__dsub_rn(M.f.phi[o + 2], ph.y), dxv.y), p, tau, pc);
      // south edges
      if (i + 1 < M.H) {
        const double2 dyv = ld2(M.f.dy, o), ps = ld2(M.f.phi, o + P);
        if (!m0 && !M.f.mask[o + P]) v.x = irls_weight32(__dsub_rn(__dsub_rn(ps.x, ph.x), dyv.x), p, tau, pc);
        if (j + 1 < M.W && !m1 && !M.f.mask[o + P + 1])
          v.y = irls_weight32(__dsub_rn(__dsub_rn(ps.y, ph.y), dyv.y), p, tau, pc);
      }
    }
    *reinterpret_cast<float2*>(M.h.U + o) = u;
    *reinterpret_cast<float2*>(M.h.V + o) = v;
    st2(M.f.U, o, make_double2((double)u.x, (double)u.y));
    st2(M.f.V, o, make_double2((double)v.x, (double)v.y));
    st2(M.f.phi_prev, o, ph);
  }
}

__global__ void k_system_x(const MapDesc* __restrict__ maps, MapState* S) {
  const MapDesc& M = maps[0];
  if (!S[0].outer_active) return;
  const unsigned half = (unsigned)M.pitch / 2u;
  const size_t n = (size_t)M.H * half;
  const size_t P = M.pitch;
  for (size_t t2 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t2 < n; t2 += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((unsigned)t2 / half), j = 2 * (int)((unsigned)t2 - (unsigned)i * half);
    const size_t o = (size_t)i * P + j;
    const double2 ue = ld2(M.f.U, o), vs = ld2(M.f.V, o), dxv = ld2(M.f.dx, o), dyv = ld2(M.f.dy, o);
    const double uw0 = (j > 0) ? M.f.U[o - 1] : 0.0;
    const double dxw = (j > 0) ? M.f.dx[o - 1] : 0.0;
    double2 vn = make_double2(0.0, 0.0), dyn = make_double2(0.0, 0.0);
    if (i > 0) {
      vn = ld2(M.f.V, o - P);
      dyn = ld2(M.f.dy, o - P);
    }
    const double uw[2] = {uw0, ue.x}, uev[2] = {ue.x, ue.y}, vnv[2] = {vn.x, vn.y}, vsv[2] = {vs.x, vs.y};
    const double dxwv[2] = {dxw, dxv.x}, dxv2[2] = {dxv.x, dxv.y}, dynv[2] = {dyn.x, dyn.y},
                 dyv2[2] = {dyv.x, dyv.y};
    double d2[2], b2[2];
    float di[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double d = __dadd_rn(__dadd_rn(__dadd_rn(uw[k], uev[k]), vnv[k]), vsv[k]);
      // b as in k_system, with fused multiply-adds (this form's system is not compared bit
      // for bit with the FP64 one: its weights are FP32); FP64 issue is what bounds the kernel
      double bk = 0.0;
      if (j + k > 0) bk = __dmul_rn(dxwv[k], uw[k]);
      bk = __fma_rn(-dxv2[k], uev[k], bk);
      if (i > 0) bk = __fma_rn(dynv[k], vnv[k], bk);
      bk = __fma_rn(-dyv2[k], vsv[k], bk);
      d2[k] = d;
      b2[k] = bk;
      di[k] = (d > 0.0) ? __fdiv_rn(1.f, (float)d) : 0.f;
    }
    st2(M.f.D, o, make_double2(d2[0], d2[1]));
    st2(M.f.b, o, make_double2(b2[0], b2[1]));
    *reinterpret_cast<float2*>(M.h.Dinv + o) = make_float2(di[0], di[1]);
  }
}

// r = b - A phi, s = M^{-1} r, partials r^T s, r^T r (and b^T b at the start).
template <int KIND>
__device__ __forceinline__ void res_tile(const PcgArgs& a, const MapDesc& M, MapState* S, int t,
                                         bool init, int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  const size_t P = M.pitch;
  XPlane x{M.f.phi, P};
  double rs = 0.0, rr = 0.0, bb = 0.0;
  auto epi = [&](size_t off, double2 xc, double2 ax) {
    const double2 bv = ld2(M.f.b, off);
    double2 r = make_double2(bv.x - ax.x, bv.y - ax.y);
    st2(M.f.r, off, r);
    if (KIND == kJacobi) {
      const double2 di = ld2(M.f.Dinv, off);
      const double2 s = make_double2(di.x * r.x, di.y * r.y);
      st2(M.f.s, off, s);
      rs = fma(r.x, s.x, rs);
      rs = fma(r.y, s.y, rs);
    }
    rr = fma(r.x, r.x, rr);
    rr = fma(r.y, r.y, rr);
    if (init) {
      bb = fma(bv.x, bv.x, bb);
      bb = fma(bv.y, bv.y, bb);
    }
  };
  stencil_tile(M, g.i0, g.i1, g.j0, lane, M.f.U, M.f.V, M.f.D, x, epi);
  if (KIND == kIdentity) rs = rr;
  tile_arrive(a, M, S, t, init ? kPhResInit : kPhRes, rs, rr, bb, lane);
}

// phi += alpha d; r -= alpha q; s = M^{-1} r; partials r^T s, r^T r.
// On a refresh iteration only phi is updated (the residual is recomputed).
template <int KIND>
__device__ __forceinline__ void b_tile(const PcgArgs& a, const MapDesc& M, MapState* S, int t,
                                       bool refresh, int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  const size_t P = M.pitch;
  const long long it = *(volatile long long*)&S->iter;
  const double* d = (it & 1) ? M.f.d0 : M.f.d1;
  const double alpha = *(volatile double*)&S->alpha;
  const int j = g.j0 + 2 * lane;
  const double2 z2 = make_double2(0.0, 0.0);
  double rs = 0.0, rr = 0.0;
  size_t off = (size_t)g.i0 * P + j;
  double2 dv = ld2(d, off), ph = ld2(M.f.phi, off);
  double2 qv = z2, rv = z2, di = z2;
  if (!refresh) {
    qv = ld2(M.f.q, off);
    rv = ld2(M.f.r, off);
    if (KIND == kJacobi) di = ld2(M.f.Dinv, off);
  }
  for (int i = g.i0; i < g.i1; ++i) {
    const size_t off2 = off + P;
    const bool more = i + 1 < g.i1;
    double2 dv2 = z2, ph2 = z2, qv2 = z2, rv2 = z2, di2 = z2;
    if (more) {
      dv2 = ld2(d, off2);
      ph2 = ld2(M.f.phi, off2);
      if (!refresh) {
        qv2 = ld2(M.f.q, off2);
        rv2 = ld2(M.f.r, off2);
        if (KIND == kJacobi) di2 = ld2(M.f.Dinv, off2);
      }
    }
    ph.x = fma(alpha, dv.x, ph.x);
    ph.y = fma(alpha, dv.y, ph.y);
    st2(M.f.phi, off, ph);
    if (!refresh) {
      rv.x = fma(-alpha, qv.x, rv.x);
      rv.y = fma(-alpha, qv.y, rv.y);
      st2(M.f.r, off, rv);
      if (KIND == kJacobi) {
        const double2 sv = make_double2(di.x * rv.x, di.y * rv.y);
        st2(M.f.s, off, sv);
        rs = fma(rv.x, sv.x, rs);
        rs = fma(rv.y, sv.y, rs);
      }
      rr = fma(rv.x, rv.x, rr);
      rr = fma(rv.y, rv.y, rr);
    }
    dv = dv2;
    ph = ph2;
    qv = qv2;
    rv = rv2;
    di = di2;
    off = off2;
  }
  if (!refresh) {
    if (KIND == kIdentity) rs = rr;
    tile_arrive(a, M, S, t, kPhB, rs, rr, 0.0, lane);
  }
}

// The inner PCG of Algorithm 1 for every map of the call, as one persistent
// cooperative kernel: phases separated by grid barriers, per-map scalars
// advanced by the last warp of each phase.  Maps that converge drop out.
template <int KIND>
__global__ void __launch_bounds__(kThreads, 2) k_pcg64(PcgArgs a) {
  __shared__ int s_base[kMaxMaps + 1];
  __shared__ int s_any;
  for (int m = threadIdx.x; m <= a.nmaps; m += blockDim.x)
    s_base[m] = (m < a.nmaps) ? a.maps[m].tile_base : a.ntiles;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int NW = gridDim.x * kWarps;

  for (int t = gw; t < a.ntiles; t += NW) {
    const int m = find_map(s_base, a.nmaps, t);
    MapState* S = a.st + m;
    if (*(volatile int*)&S->done) continue;
    res_tile<KIND>(a, a.maps[m], S, t, true, lane);
  }
  if (!grid_sync(a.bar, a.timeout_ns)) return;

  for (int g = 0;; ++g) {
    if (*(volatile int*)a.n_active == 0) break;
    for (int t = gw; t < a.ntiles; t += NW) {
      const int m = find_map(s_base, a.nmaps, t);
      MapState* S = a.st + m;
      if (*(volatile int*)&S->done) continue;
      a_tile<KIND>(a, a.maps[m], S, t, lane);
    }
    if (!grid_sync(a.bar, a.timeout_ns)) return;
    // refresh iterations (l mod period = 0) are a static function of g
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int m = threadIdx.x; m < a.nmaps; m += blockDim.x)
      if (g % a.maps[m].refresh == 0) s_any = 1;
    __syncthreads();
    const bool any_refresh = s_any != 0;
    for (int t = gw; t < a.ntiles; t += NW) {
      const int m = find_map(s_base, a.nmaps, t);
      MapState* S = a.st + m;
      if (*(volatile int*)&S->done) continue;
      const MapDesc& M = a.maps[m];
      b_tile<KIND>(a, M, S, t, (g % M.refresh) == 0, lane);
    }
    if (!grid_sync(a.bar, a.timeout_ns)) return;
    if (any_refresh) {
      for (int t = gw; t < a.ntiles; t += NW) {
        const int m = find_map(s_base, a.nmaps, t);
        MapState* S = a.st + m;
        const MapDesc& M = a.maps[m];
        if (*(volatile int*)&S->done || (g % M.refresh) != 0) continue;
        res_tile<KIND>(a, M, S, t, false, lane);
      }
      if (!grid_sync(a.bar, a.timeout_ns)) return;
    }
  }
}

// ------------------------------------------------------------------ ILU(0) / IC(0) / SSOR engine
// Factor applied to r before the forward sweep: 1 for ILU/IC, (2 - omega)/omega
// for SSOR (the omega/(2 - omega) of M moved onto the right-hand side).
template <int KIND>
__device__ __forceinline__ double sweep_rscale(const PcgArgs& a) {
  return (KIND == kSsor) ? (2.0 - a.omega) / a.omega : 1.0;
}

// r = b - A phi and the forward sweep's right-hand side r pinv c (stored in s).
template <int KIND>
__device__ __forceinline__ void res_tile_sweep(const PcgArgs& a, const MapDesc& M, int t, int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  XPlane x{M.f.phi, (size_t)M.pitch};
  const double c = sweep_rscale<KIND>(a);
  auto epi = [&](size_t off, double2, double2 ax) {
    const double2 bv = ld2(M.f.b, off);
    const double2 r = make_double2(bv.x - ax.x, bv.y - ax.y);
    st2(M.f.r, off, r);
    const double2 pv = ld2(M.f.piv, off);
    st2(M.f.s, off, make_double2(r.x * pv.x * c, r.y * pv.y * c));
  };
  stencil_tile(M, g.i0, g.i1, g.j0, lane, M.f.U, M.f.V, M.f.D, x, epi);
}

// phi += alpha d; r -= alpha q (not on refresh iterations); s = r pinv c.
template <int KIND>
__device__ __forceinline__ void b_tile_sweep(const PcgArgs& a, const MapDesc& M, MapState* S, int t,
                                             bool refresh, int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  const size_t P = M.pitch;
  const long long it = *(volatile long long*)&S->iter;
  const double* d = (it & 1) ? M.f.d0 : M.f.d1;
  const double alpha = *(volatile double*)&S->alpha;
  const double c = sweep_rscale<KIND>(a);
  const int j = g.j0 + 2 * lane;
  for (int i = g.i0; i < g.i1; ++i) {
    const size_t off = (size_t)i * P + j;
    const double2 dv = ld2(d, off);
    double2 ph = ld2(M.f.phi, off);
    double2 qv, rv, pv;
    if (!refresh) {
      qv = ld2(M.f.q, off);
      rv = ld2(M.f.r, off);
      pv = ld2(M.f.piv, off);
    }
    ph.x = fma(alpha, dv.x, ph.x);
    ph.y = fma(alpha, dv.y, ph.y);
    st2(M.f.phi, off, ph);
    if (!refresh) {
      rv.x = fma(-alpha, qv.x, rv.x);
      rv.y = fma(-alpha, qv.y, rv.y);
      st2(M.f.r, off, rv);
      st2(M.f.s, off, make_double2(rv.x * pv.x * c, rv.y * pv.y * c));
    }
  }
}

// Partials r^T s, r^T r (and b^T b on the first pass) after the backward sweep.
__device__ __forceinline__ void dots_tile(const PcgArgs& a, const MapDesc& M, MapState* S, int t, bool init,
                                          int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  const size_t P = M.pitch;
  const int j = g.j0 + 2 * lane;
  double rs = 0.0, rr = 0.0, bb = 0.0;
  for (int i = g.i0; i < g.i1; ++i) {
    const size_t off = (size_t)i * P + j;
    const double2 rv = ld2(M.f.r, off), sv = ld2(M.f.s, off);
    rs = fma(rv.x, sv.x, rs);
    rs = fma(rv.y, sv.y, rs);
    rr = fma(rv.x, rv.x, rr);
    rr = fma(rv.y, rv.y, rr);
    if (init) {
      const double2 bv = ld2(M.f.b, off);
      bb = fma(bv.x, bv.x, bb);
      bb = fma(bv.y, bv.y, bb);
    }
  }
  tile_arrive(a, M, S, t, init ? kPhResInit : kPhB, rs, rr, bb, lane);
}

// Sweep coefficients from U, V and 1/P (SSOR: 1/P = omega/D, D = 0 read as 1).
template <int KIND>
__device__ __forceinline__ void coef_tile(const PcgArgs& a, const MapDesc& M, int t, int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  const size_t P = M.pitch;
  const int j = g.j0 + 2 * lane;
  for (int i = g.i0; i < g.i1; ++i) {
    const size_t off = (size_t)i * P + j;
    double2 pv;
    if (KIND == kSsor) {
      const double2 dd = ld2(M.f.D, off);
      pv.x = a.omega / (dd.x > 0.0 ? dd.x : 1.0);
      pv.y = a.omega / (dd.y > 0.0 ? dd.y : 1.0);
      st2(M.f.piv, off, pv);
    } else {
      pv = ld2(M.f.piv, off);
    }
    const double2 u = ld2(M.f.U, off), v = ld2(M.f.V, off);
    const double uw = (j > 0) ? ld1(M.f.U, off - 1) : 0.0;
    const double2 vn = (i > 0) ? ld2(M.f.V, off - P) : make_double2(0.0, 0.0);
    st2(M.f.cw, off, make_double2(uw * pv.x, u.x * pv.y));
    st2(M.f.cn, off, make_double2(vn.x * pv.x, vn.y * pv.y));
    st2(M.f.ce, off, make_double2(u.x * pv.x, u.y * pv.y));
    st2(M.f.cs, off, make_double2(v.x * pv.x, v.y * pv.y));
  }
}

// Runs one sweep over every band of every map still iterating: consecutive
// slots sit on different SMs; forward sweeps take bands in increasing order,
// backward sweeps in decreasing order, so every wait is on a band that an
// earlier-ordered slot step has already been given (no cycle).
template <int MODE>
__device__ bool sweep_phase(const PcgArgs& a, const int* s_bbase, bool (*want)(const MapState*)) {
  const int lane = threadIdx.x & 31;
  const int slot = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const int NS = gridDim.x * kWarps;
  for (int k = slot; k < a.nbands; k += NS) {
    const int gb = (MODE == kSweepBwd) ? a.nbands - 1 - k : k;
    const int m = find_map(s_bbase, a.nmaps, gb);
    MapState* S = a.st + m;
    if (!want(S)) continue;
    const MapDesc& M = a.maps[m];
    const int band = gb - M.band_base, nb = M.nbands;
    const size_t P = M.pitch;
    SweepIO io;
    if (MODE == kSweepBwd) {
      io = SweepIO{M.f.y, M.f.ce, M.f.cs, M.f.s, nullptr, nullptr};
      if (band + 1 < nb) io.xin = M.xb + (size_t)(band + 1) * P;
      if (band > 0) io.xout = M.xb + (size_t)band * P;
    } else {
      if (MODE == kSweepPiv) io = SweepIO{M.f.D, M.f.U, M.f.V, M.f.piv, nullptr, nullptr};
      else io = SweepIO{M.f.s, M.f.cw, M.f.cn, M.f.y, nullptr, nullptr};
      if (band > 0) io.xin = M.xf + (size_t)(band - 1) * P;
      if (band + 1 < nb) io.xout = M.xf + (size_t)band * P;
    }
    if (!band_sweep<MODE>(M, band, lane, io, a.timeout_ns, &a.bar->err))
      return false;  // the error flag is set: the next grid barrier ends every block
  }
  return true;
}

// Fills every exchange row with the sentinel (start of a launch).
__device__ void reset_exchange(const PcgArgs& a, const int* s_bbase) {
  const int lane = threadIdx.x & 31;
  const int slot = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const int NS = gridDim.x * kWarps;
  for (int gb = slot; gb < a.nbands; gb += NS) {
    const int m = find_map(s_bbase, a.nmaps, gb);
    const MapDesc& M = a.maps[m];
    const size_t off = (size_t)(gb - M.band_base) * M.pitch;
    for (int j = lane; j < M.pitch; j += 32) {
      st_relaxed(M.xf + off + j, sentinel());
      st_relaxed(M.xb + off + j, sentinel());
    }
  }
}

__device__ bool map_active(const MapState* S) { return *(volatile const int*)&S->done == 0; }

template <int KIND>
__global__ void __launch_bounds__(kThreads, 1) k_pcg64_sweep(PcgArgs a) {
  __shared__ int s_base[kMaxMaps + 1];
  __shared__ int s_bbase[kMaxMaps + 1];
  __shared__ int s_any;
  for (int m = threadIdx.x; m <= a.nmaps; m += blockDim.x) {
    s_base[m] = (m < a.nmaps) ? a.maps[m].tile_base : a.ntiles;
    s_bbase[m] = (m < a.nmaps) ? a.maps[m].band_base : a.nbands;
  }
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

  reset_exchange(a, s_bbase);
  if (!grid_sync(a.bar, a.timeout_ns)) return;
  // preconditioner set-up (Algorithm 1: estimate M from A), timed by block 0 between the
  // grid barriers that bracket it
  const unsigned long long t_setup = (blockIdx.x == 0 && threadIdx.x == 0) ? globaltimer() : 0ull;
  if (KIND == kIlu) {
    sweep_phase<kSweepPiv>(a, s_bbase, map_active);
    if (!grid_sync(a.bar, a.timeout_ns)) return;
  }
  for_tiles([&](const MapDesc& M, MapState*, int t) { coef_tile<KIND>(a, M, t, lane); });
  if (!grid_sync(a.bar, a.timeout_ns)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats && !a.apply_only)
    atomicAdd(&a.stats->setup_ns, globaltimer() - t_setup);
  // r = b - A phi, d = M^-1 r, delta_new = r^T d
  for_tiles([&](const MapDesc& M, MapState*, int t) { res_tile_sweep<KIND>(a, M, t, lane); });
  if (!grid_sync(a.bar, a.timeout_ns)) return;
  sweep_phase<kSweepFwd>(a, s_bbase, map_active);
  if (!grid_sync(a.bar, a.timeout_ns)) return;
  sweep_phase<kSweepBwd>(a, s_bbase, map_active);
  if (!grid_sync(a.bar, a.timeout_ns)) return;
  for_tiles([&](const MapDesc& M, MapState* S, int t) { dots_tile(a, M, S, t, true, lane); });
  if (!grid_sync(a.bar, a.timeout_ns)) return;
  if (a.apply_only) return;

  for (int g = 0;; ++g) {
    if (*(volatile int*)a.n_active == 0) break;
    for_tiles([&](const MapDesc& M, MapState* S, int t) { a_tile<kIlu>(a, M, S, t, lane); });
    if (!grid_sync(a.bar, a.timeout_ns)) return;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int m = threadIdx.x; m < a.nmaps; m += blockDim.x)
      if (g % a.maps[m].refresh == 0) s_any = 1;
    __syncthreads();
    const bool any_refresh = s_any != 0;
    for_tiles([&](const MapDesc& M, MapState* S, int t) {
      b_tile_sweep<KIND>(a, M, S, t, (g % M.refresh) == 0, lane);
    });
    if (!grid_sync(a.bar, a.timeout_ns)) return;
    if (any_refresh) {
      for_tiles([&](const MapDesc& M, MapState*, int t) {
        if ((g % M.refresh) == 0) res_tile_sweep<KIND>(a, M, t, lane);
      });
      if (!grid_sync(a.bar, a.timeout_ns)) return;
    }
    sweep_phase<kSweepFwd>(a, s_bbase, map_active);
    if (!grid_sync(a.bar, a.timeout_ns)) return;
    sweep_phase<kSweepBwd>(a, s_bbase, map_active);
    if (!grid_sync(a.bar, a.timeout_ns)) return;
    for_tiles([&](const MapDesc& M, MapState* S, int t) { dots_tile(a, M, S, t, false, lane); });
    if (!grid_sync(a.bar, a.timeout_ns)) return;
  }
}

// Resets the per-map solver state before a PCG launch.
__global__ void k_pcg_reset(MapState* S, int nmaps, int* n_active, Barrier* bar) {
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  for (int m = threadIdx.x; m < nmaps; m += blockDim.x) {
    MapState* s = S + m;
    const int act = s->outer_active;
    s->delta = s->delta0 = s->rr = s->bb = s->dq = s->alpha = s->beta = s->relres = 0.0;
    s->iter = 0;
    s->status = 0;
    s->done = act ? 0 : 1;
    s->stop_after = 0;
    s->arrive = 0u;
    for (int g = 0; g < kArriveGroups; ++g) s->arrive_grp[g] = 0u;
    s->loops = 0;
    s->fallback = 0;
    s->restart = 0;
    s->stall = 0;
    s->force_refresh = 0;
    s->x_clean = 0;
    s->confirm = 0;
    s->refresh_next = 0;
    s->rr_ref = 0.0;
    s->rr_best = 0.0;
    if (act) atomicAdd(&s_cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *n_active = s_cnt;
    bar->count = 0u;
    bar->err = 0;
    __threadfence();
  }
}

// ------------------------------------------------------------------ outer error
// Algorithm 1: error = ||phi^{k+1} - phi^k|| / ||phi^k|| (infinite when
// ||phi^k|| = 0); records the pass in the map's statistics and decides
// whether the next pass runs.
__global__ void k_outer_error(const MapDesc* __restrict__ maps, MapState* S, MapStats* stats,
                              double* part, int nbx, double outer_tol, int max_outer, int* bar_err) {
  const int m = blockIdx.y;
  const MapDesc& M = maps[m];
  MapState* s = S + m;
  if (!s->outer_active) return;
  // two elements per thread (the planes' pitch is even; padding columns are 0 in both)
  const size_t n2 = (size_t)M.H * M.pitch / 2;
  double num = 0.0, den = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n2; t += (size_t)gridDim.x * blockDim.x) {
    const double2 ph = ld2(M.f.phi, 2 * t), pp = ld2(M.f.phi_prev, 2 * t);
    const double ex = ph.x - pp.x, ey = ph.y - pp.y;
    num = fma(ex, ex, num);
    num = fma(ey, ey, num);
    den = fma(pp.x, pp.x, den);
    den = fma(pp.y, pp.y, den);
  }
  __shared__ double sn[kWarps], sd[kWarps];
  num = warp_sum(num);
  den = warp_sum(den);
  if ((threadIdx.x & 31) == 0) {
    sn[threadIdx.x >> 5] = num;
    sd[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  __shared__ unsigned s_old;
  double* pn = part + (size_t)m * nbx * 2;   // nbx numerators, then nbx denominators
  double* pd = pn + nbx;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sn[w]; b += sd[w]; }
    pn[blockIdx.x] = a;
    pd[blockIdx.x] = b;
    __threadfence();
    s_old = atomicAdd(&s->arrive_outer, 1u);
  }
  __syncthreads();
  if (s_old != (unsigned)gridDim.x - 1u || threadIdx.x >= 32) return;
  __threadfence();
  const double a = warp_sum_partials(pn, gridDim.x, threadIdx.x);
  const double b = warp_sum_partials(pd, gridDim.x, threadIdx.x);
  if (threadIdx.x != 0) return;
  const double err = (b > 0.0) ? sqrt(a) / sqrt(b) : INFINITY;
  MapStats* st = stats + m;
  const int k = s->outer_k;
  if (k < 64) {
    st->inner[k] = s->iter;
    st->relres[k] = s->relres;
    st->outer_err[k] = err;
  }
  st->inner_total += s->iter;
  st->fallbacks += s->fallback;
  int status = s->status;
  if (*(volatile int*)bar_err) status = -4;
  if (status < 0) st->status = status;
  else if (status == 1 && st->status == 0) st->status = 1;
  st->outer = k + 1;
  s->outer_err = err;
  s->outer_k = k + 1;
  s->arrive_outer = 0u;
  s->outer_active = (status >= 0 && err > outer_tol && k + 1 < max_outer) ? 1 : 0;
  __threadfence();
}

// Starts a call: statistics cleared, every map active unless its input failed the checks.
__global__ void k_begin(MapState* S, MapStats* stats, int nmaps) {
  for (int m = threadIdx.x; m < nmaps; m += blockDim.x) {
    MapState* s = S + m;
    MapStats* st = stats + m;
    st->status = 0;
    st->outer = 0;
    st->inner_total = 0;
    st->fallbacks = 0;
    st->setup_ns = 0;
    for (int k = 0; k < 64; ++k) { st->inner[k] = 0; st->relres[k] = 0.0; st->outer_err[k] = 0.0; }
    s->outer_k = 0;
    s->arrive_outer = 0u;
    s->err_flag = 0;
    s->outer_active = 1;
  }
}

__global__ void k_check_input(MapState* S, MapStats* stats, int nmaps) {
  for (int m = threadIdx.x; m < nmaps; m += blockDim.x) {
    if (S[m].err_flag) {
      S[m].outer_active = 0;
      stats[m].status = -1;
    }
  }
}

// ------------------------------------------------------------------ single steps
// y = A x on one map, with the solver's stencil walker.
__global__ void __launch_bounds__(kThreads) k_matvec(MapDesc M, const double* __restrict__ xin, double* y, int R) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int NW = gridDim.x * kWarps;
  for (int t = gw; t < M.ntiles; t += NW) {
    const TileGeo g = tile_geo(M, t + M.tile_base, R);
    XPlane x{xin, (size_t)M.pitch};
    auto epi = [&](size_t off, double2, double2 ax) { st2(y, off, ax); };
    stencil_tile(M, g.i0, g.i1, g.j0, lane, M.f.U, M.f.V, M.f.D, x, epi);
  }
}

__global__ void k_jacobi_apply(MapDesc M, const double* __restrict__ r, double* s, int kind) {
  const size_t n = (size_t)M.H * M.pitch;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    s[t] = (kind == kJacobi) ? M.f.Dinv[t] * r[t] : r[t];
}

// Copies a user-layout H x W array into a padded plane (zero padding) and back.
__global__ void k_to_plane(MapDesc M, const double* __restrict__ src, double* dst) {
  const size_t n = (size_t)M.H * M.pitch;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((unsigned)t / (unsigned)M.pitch), j = (int)((unsigned)t - (unsigned)i * (unsigned)M.pitch);
    dst[t] = (j < M.W) ? src[(size_t)i * M.W + j] : 0.0;
  }
}
__global__ void k_from_plane(MapDesc M, const double* __restrict__ src, double* dst) {
  const size_t n = (size_t)M.H * M.W;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((unsigned)k / (unsigned)M.W), j = (int)((unsigned)k - (unsigned)i * (unsigned)M.W);
    dst[k] = src[(size_t)i * M.pitch + j];
  }
}
__global__ void k_mask_to_plane(MapDesc M, const uint8_t* __restrict__ src) {
  const size_t n = (size_t)M.H * M.pitch;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((unsigned)t / (unsigned)M.pitch), j = (int)((unsigned)t - (unsigned)i * (unsigned)M.pitch);
    M.f.mask[t] = (j < M.W && src) ? (src[(size_t)i * M.W + j] ? 1 : 0) : 0;
  }
}

// ------------------------------------------------------------------ host side
static int grid_for(size_t n, int nsm) {
  size_t b = (n + kThreads - 1) / kThreads;
  size_t cap = (size_t)nsm * 8;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

cudaError_t launch_pack(const Plan& pl, int m, const double* psi, const uint8_t* mask, const double* phi0,
                        cudaStream_t st) {
  const MapDesc& M = pl.hmaps[m];
  pl.kernel_launches += 1;
  k_pack<<<grid_for((size_t)M.H * M.pitch, pl.nsm), kThreads, 0, st>>>(M, pl.dstate + m, psi, mask, phi0);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const Plan& pl, int m, double* phi, cudaStream_t st) {
  const MapDesc& M = pl.hmaps[m];
  pl.kernel_launches += 1;
  k_unpack<<<grid_for((size_t)M.H * M.W, pl.nsm), kThreads, 0, st>>>(M, phi);
  return cudaGetLastError();
}

cudaError_t launch_begin(const Plan& pl, cudaStream_t st) {
  pl.kernel_launches += 1;
  k_begin<<<1, kThreads, 0, st>>>(pl.dstate, pl.dstats, pl.nmaps);
  return cudaGetLastError();
}

cudaError_t launch_check(const Plan& pl, cudaStream_t st) {
  pl.kernel_launches += 1;
  k_check_input<<<1, kThreads, 0, st>>>(pl.dstate, pl.dstats, pl.nmaps);
  return cudaGetLastError();
}

cudaError_t launch_diag(const Plan& pl, cudaStream_t st) {
  dim3 grid(pl.bx_elem, pl.nmaps);
  pl.kernel_launches += 1;
  k_system<<<grid, kThreads, 0, st>>>(pl.dmaps, pl.dstate);
  return cudaGetLastError();
}

cudaError_t launch_system(const Plan& pl, const double* d_p, const double* d_tau, cudaStream_t st) {
  dim3 grid(pl.bx_elem, pl.nmaps);
  pl.kernel_launches += 2;
  k_weights<<<grid, kThreads, 0, st>>>(pl.dmaps, pl.dstate, d_p, d_tau);
  k_system<<<grid, kThreads, 0, st>>>(pl.dmaps, pl.dstate);
  return cudaGetLastError();
}

cudaError_t launch_system_x(const Plan& pl, const double* d_p, const double* d_tau, cudaStream_t st) {
  if (pl.nmaps != 1) return cudaErrorNotSupported;
  pl.kernel_launches += 2;
  k_weights_x<<<pl.bx_elem, kThreads, 0, st>>>(pl.dmaps, pl.dstate, d_p, d_tau);
  k_system_x<<<pl.bx_elem, kThreads, 0, st>>>(pl.dmaps, pl.dstate);
  return cudaGetLastError();
}

cudaError_t launch_outer_error(const Plan& pl, double outer_tol, int max_outer, cudaStream_t st) {
  dim3 grid(pl.bx_elem, pl.nmaps);
  pl.kernel_launches += 1;
  k_outer_error<<<grid, kThreads, 0, st>>>(pl.dmaps, pl.dstate, pl.dstats, pl.outer_part, pl.bx_elem,
                                           outer_tol, max_outer, &pl.bar->err);
  return cudaGetLastError();
}

template <int KIND>
static cudaError_t launch_pcg64_kind(const Plan& pl, const PcgArgs& a, int blocks, cudaStream_t st) {
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((void*)k_pcg64<KIND>, blocks, kThreads, args, 0, st);
}

int pcg64_max_blocks_per_sm(int kind) {
  int nb = 0;
  switch (kind) {
    case kIdentity: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg64<kIdentity>, kThreads, 0); break;
    case kJacobi: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg64<kJacobi>, kThreads, 0); break;
    case kIlu:
    case kIc: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg64_sweep<kIlu>, kThreads, 0); break;
    case kSsor: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg64_sweep<kSsor>, kThreads, 0); break;
    default: nb = 0;
  }
  return nb;
}

void launch_pcg_reset(const Plan& pl, cudaStream_t st) {
  k_pcg_reset<<<1, kThreads, 0, st>>>(pl.dstate, pl.nmaps, pl.n_active, pl.bar);
}

cudaError_t launch_pcg64(const Plan& pl, int kind, const PcgArgs& a, cudaStream_t st, cudaEvent_t e0,
                         cudaEvent_t e1) {
  pl.kernel_launches += 2;
  pl.solver_launches += 1;
  k_pcg_reset<<<1, kThreads, 0, st>>>(pl.dstate, pl.nmaps, pl.n_active, pl.bar);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (e0) cudaEventRecord(e0, st);
  const int blocks = pl.nsm * pl.bps;
  switch (kind) {
    case kIdentity: e = launch_pcg64_kind<kIdentity>(pl, a, blocks, st); break;
    case kJacobi: e = launch_pcg64_kind<kJacobi>(pl, a, blocks, st); break;
    case kIlu:
    case kIc: {
      void* args[] = {(void*)&a};
      e = cudaLaunchCooperativeKernel((void*)k_pcg64_sweep<kIlu>, pl.nsm * pl.bps_sweep, kThreads, args, 0, st);
      break;
    }
    case kSsor: {
      void* args[] = {(void*)&a};
      e = cudaLaunchCooperativeKernel((void*)k_pcg64_sweep<kSsor>, pl.nsm * pl.bps_sweep, kThreads, args, 0, st);
      break;
    }
    default: e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess && e1) e = cudaEventRecord(e1, st);
  return e;
}

cudaError_t launch_matvec(const Plan& pl, const double* x, double* y, cudaStream_t st) {
  const MapDesc& M = pl.hmaps[0];
  const int blocks = (M.ntiles + kWarps - 1) / kWarps;
  pl.kernel_launches += 1;
  k_matvec<<<blocks, kThreads, 0, st>>>(M, x, y, pl.R);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_apply(const Plan& pl, int kind, const double* r, double* s, cudaStream_t st) {
  const MapDesc& M = pl.hmaps[0];
  pl.kernel_launches += 1;
  k_jacobi_apply<<<grid_for((size_t)M.H * M.pitch, pl.nsm), kThreads, 0, st>>>(M, r, s, kind);
  return cudaGetLastError();
}

cudaError_t launch_to_plane(const Plan& pl, const double* src, double* dst, cudaStream_t st) {
  const MapDesc& M = pl.hmaps[0];
  pl.kernel_launches += 1;
  k_to_plane<<<grid_for((size_t)M.H * M.pitch, pl.nsm), kThreads, 0, st>>>(M, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_from_plane(const Plan& pl, const double* src, double* dst, cudaStream_t st) {
  const MapDesc& M = pl.hmaps[0];
  pl.kernel_launches += 1;
  k_from_plane<<<grid_for((size_t)M.H * M.W, pl.nsm), kThreads, 0, st>>>(M, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_mask_to_plane(const Plan& pl, const uint8_t* mask, cudaStream_t st) {
  const MapDesc& M = pl.hmaps[0];
  pl.kernel_launches += 1;
  k_mask_to_plane<<<grid_for((size_t)M.H * M.pitch, pl.nsm), kThreads, 0, st>>>(M, mask);
  return cudaGetLastError();
}

}  // namespace ulp
