// ulp_mixed.cuh -- FP32 pieces of the mixed-precision solvers shared by the
// persistent reliable-update PCG (ulp_mixed.cu) and the mixed flexible CG
// (ulp_fcg.cu): double-float accumulation of FP32 products, the FP32
// sliding-window stencil, and phase A (d = s + beta d, q = A d, d^T q).
#pragma once
#include "ulp_engine.cuh"

namespace ulp {

// Double-float accumulator of FP32 products: a*b = p + e exactly (FMA), and
// the running sum is carried as hi + lo with Knuth's two-sum.
struct DF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ float2 ldf2(const float* base, size_t off) {
  return __ldcg(reinterpret_cast<const float2*>(base + off));
}
__device__ __forceinline__ void stf2(float* base, size_t off, float2 v) {
  __stcg(reinterpret_cast<float2*>(base + off), v);
}

struct XDir32 {  // d = s + beta d_old (FP32), d = s on the first iteration
  const float* s;
  const float* dold;
  float beta;
  bool first;
  size_t P;
  struct Raw {
    float2 s, d;
  };
  __device__ __forceinline__ static Raw zero() { return Raw{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
  __device__ __forceinline__ Raw load(int i, int j) const {
    const size_t off = (size_t)i * P + j;
    Raw r;
    r.s = ldf2(s, off);
    r.d = first ? make_float2(0.f, 0.f) : ldf2(dold, off);
    return r;
  }
  __device__ __forceinline__ float2 make(const Raw& r) const {
    if (first) return r.s;
    return make_float2(__fmaf_rn(beta, r.d.x, r.s.x), __fmaf_rn(beta, r.d.y, r.s.y));
  }
  __device__ __forceinline__ float at(int i, int c) const {
    const size_t off = (size_t)i * P + c;
    const float sv = __ldcg(s + off);
    return first ? sv : __fmaf_rn(beta, __ldcg(dold + off), sv);
  }
};

// FP32 sliding-window stencil (same tiling as the FP64 walker), summed over the
// edges as w (x_i - x_j) from the FP32 weights: the FP32 operator keeps A 1 = 0
// exactly, and for the smooth directions of a well-preconditioned solve its error
// stays relative to |A x| rather than to |A| |x|.  FP32 rows move half the bytes of
// FP64 ones, so loads run LA rows ahead of the arithmetic (a ring of raw rows in
// registers) to keep more bytes in flight with two blocks per SM.
template <class X, class Epi, int LA = 3>
__device__ __forceinline__ void stencil_tile32(const MapDesc& M, int i0, int i1, int j0, int lane,
                                               const float* U, const float* V, const X& x, Epi& epi) {
  using Raw = typename X::Raw;
  const int j = j0 + 2 * lane;
  const bool hw = (lane == 0) && (j0 > 0);
  const bool he = (lane == 31) && (j0 + kStrip < M.pitch);
  const bool halo = hw || he;
  const int hc = (lane == 0) ? j0 - 1 : j0 + kStrip;
  const size_t P = (size_t)M.pitch;
  const float2 z2 = make_float2(0.f, 0.f);
  float2 xn = z2, vn = z2;
  if (i0 > 0) {
    xn = x.make(x.load(i0 - 1, j));
    vn = ldf2(V, (size_t)(i0 - 1) * P + j);
  }
  float2 xc = x.make(x.load(i0, j));
  // rings: raw x of rows i+1 .. i+LA (row r is needed while row r-1 is in the tile);
  // weights and halo of rows i .. i+LA-1
  Raw rx[LA];
  float2 uu[LA], vv[LA];
  float hh[LA], ww[LA];
#pragma unroll
  for (int k = 0; k < LA; ++k) {
    const int ri = i0 + 1 + k, wi = i0 + k;
    rx[k] = (ri < M.H && ri - 1 < i1) ? x.load(ri, j) : X::zero();
    uu[k] = vv[k] = z2;
    hh[k] = ww[k] = 0.f;
    if (wi < i1) {
      const size_t o = (size_t)wi * P + j;
      uu[k] = ldf2(U, o);
      vv[k] = ldf2(V, o);
      if (halo) hh[k] = x.at(wi, hc);
      if (hw) ww[k] = __ldcg(U + o - j + hc);
    }
  }
  size_t off = (size_t)i0 * P + j;
  // unrolled by LA so the ring shifts become register renames (measured: mixed Jacobi
  // PCG 6.0 -> 6.2 Mpx/s at 2048^2 with LA = 3; LA = 4 unrolled spills)
#pragma unroll LA
  for (int i = i0; i < i1; ++i) {
    // issue the loads LA rows ahead
    const int rn = i + 1 + LA, wn = i + LA;
    const Raw rnew = (rn < M.H && rn - 1 < i1) ? x.load(rn, j) : X::zero();
    float2 unew = z2, vnew = z2;
    float hnew = 0.f, wnew = 0.f;
    if (wn < i1) {
      const size_t o = off + (size_t)LA * P;
      unew = ldf2(U, o);
      vnew = ldf2(V, o);
      if (halo) hnew = x.at(wn, hc);
      if (hw) wnew = __ldcg(U + o - j + hc);
    }
    const float2 u0 = uu[0], v0 = vv[0];
    const float2 xs = (i + 1 < M.H) ? x.make(rx[0]) : z2;
    float west = __shfl_up_sync(kFull, xc.y, 1);
    float east = __shfl_down_sync(kFull, xc.x, 1);
    float uw = __shfl_up_sync(kFull, u0.y, 1);
    if (lane == 0) { west = hh[0]; uw = ww[0]; }
    if (lane == 31) east = hh[0];
    // sum over the four edges of w (x_i - x_j): the neighbour differences are nearly
    // exact for a smooth x, where D x_i - sum w x_j would cancel to a few bits
    float2 ax;
    ax.x = __fmul_rn(u0.x, __fsub_rn(xc.x, xc.y));
    ax.x = __fmaf_rn(uw, __fsub_rn(xc.x, west), ax.x);
    ax.x = __fmaf_rn(vn.x, __fsub_rn(xc.x, xn.x), ax.x);
    ax.x = __fmaf_rn(v0.x, __fsub_rn(xc.x, xs.x), ax.x);
    ax.y = __fmul_rn(u0.y, __fsub_rn(xc.y, east));
    ax.y = __fmaf_rn(u0.x, __fsub_rn(xc.y, xc.x), ax.y);
    ax.y = __fmaf_rn(vn.y, __fsub_rn(xc.y, xn.y), ax.y);
    ax.y = __fmaf_rn(v0.y, __fsub_rn(xc.y, xs.y), ax.y);
    epi(off, xc, ax);
    xn = xc;
    xc = xs;
    vn = v0;
#pragma unroll
    for (int k = 0; k + 1 < LA; ++k) {
      rx[k] = rx[k + 1];
      uu[k] = uu[k + 1];
      vv[k] = vv[k + 1];
      hh[k] = hh[k + 1];
      ww[k] = ww[k + 1];
    }
    rx[LA - 1] = rnew;
    uu[LA - 1] = unew;
    vv[LA - 1] = vnew;
    hh[LA - 1] = hnew;
    ww[LA - 1] = wnew;
    off += P;
  }
}

// d = s + beta d_old, q = A d in FP32, d^T q FP64-accurate.
template <int KIND>
__device__ __forceinline__ void a32_tile(const PcgArgs& a, const MapDesc& M, MapState* S, int t, int lane) {
  const TileGeo g = tile_geo(M, t, a.R);
  const long long it = *(volatile long long*)&S->iter;
  const float* sv = (KIND == kIdentity) ? M.h.r : M.h.s;
  const float* dold = (it & 1) ? M.h.d1 : M.h.d0;
  float* dnew = (it & 1) ? M.h.d0 : M.h.d1;
  XDir32 x{sv, dold, (float)*(volatile double*)&S->beta, it == 0, (size_t)M.pitch};
  DF dq;
  auto epi = [&](size_t off, float2 xc, float2 ax) {
    stf2(dnew, off, xc);
    stf2(M.h.q, off, ax);
    dq.add_prod(xc.x, ax.x);
    dq.add_prod(xc.y, ax.y);
  };
  stencil_tile32(M, g.i0, g.i1, g.j0, lane, M.h.U, M.h.V, x, epi);
  tile_arrive(a, M, S, t, kPhA, dq.value(), 0.0, 0.0, lane);
}

}  // namespace ulp
