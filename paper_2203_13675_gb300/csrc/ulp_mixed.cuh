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

// cp.async helpers: each lane copies its own pieces into shared memory (zero-filled
// where the source size is 0) and waits on its own copies only.
__device__ __forceinline__ void cpa8(void* sdst, const void* gsrc, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sa), "l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cpa4(void* sdst, const void* gsrc, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// FP32 sliding-window stencil (same tiling as the FP64 walker), summed over the
// edges as w (x_i - x_j) from the FP32 weights: the FP32 operator keeps A 1 = 0
// exactly, and for the smooth directions of a well-preconditioned solve its error
// stays relative to |A x| rather than to |A| |x|.  The rows stream through a ring of
// kRing32 slots per warp in shared memory, filled by cp.async kLead32 rows ahead of
// the arithmetic (rows outside the grid zero-filled): the loads in flight cost no
// registers, and a row's wait is the hardware wait on the lane's own copies.
constexpr int kLead32 = 3;
// a slot is refilled only after the arithmetic that consumed the row it held: the row
// two behind the one just read, so the ring holds kLead32 + 2 rows
constexpr int kRing32 = kLead32 + 2;
struct Slot32 {
  float2 S[32], D[32], U[32], V[32];  // s, d_old, U, V at the lane's two columns
  float hs[2], hd[2], hu, pad_[3];    // halo columns: s, d_old for lanes 0 and 31, U for lane 0
};

__device__ __forceinline__ void slot32_issue(Slot32& sl, const MapDesc& M, const XDir32& x, const float* U,
                                             const float* V, int r, int j, int lane, bool hw, bool halo, int hc) {
  const bool in = r >= 0 && r < M.H;
  const size_t o = in ? (size_t)r * M.pitch + j : 0;
  const int nb = in ? 8 : 0;
  cpa8(&sl.S[lane], x.s + o, nb);
  cpa8(&sl.D[lane], x.dold + o, x.first ? 0 : nb);
  cpa8(&sl.U[lane], U + o, nb);
  cpa8(&sl.V[lane], V + o, nb);
  if (halo) {
    const size_t oh = in ? (size_t)r * M.pitch + hc : 0;
    const int k = lane == 0 ? 0 : 1;
    cpa4(&sl.hs[k], x.s + oh, in ? 4 : 0);
    cpa4(&sl.hd[k], x.dold + oh, (in && !x.first) ? 4 : 0);
    if (hw) cpa4(&sl.hu, U + oh, in ? 4 : 0);
  }
}

// ring: the warp's kRing32 slots in shared memory
template <class Epi>
__device__ __forceinline__ void stencil_tile32(const MapDesc& M, int i0, int i1, int j0, int lane,
                                               const float* U, const float* V, const XDir32& x, Epi& epi,
                                               Slot32* ring) {
  const int j = j0 + 2 * lane;
  const bool hw = (lane == 0) && (j0 > 0);
  const bool he = (lane == 31) && (j0 + kStrip < M.pitch);
  const bool halo = hw || he;
  const int hc = (lane == 0) ? j0 - 1 : j0 + kStrip;
  const int hk = lane == 0 ? 0 : 1;
  // rows rb = i0-1 .. re = i1 stream through the ring, row r in slot (r - rb) % kRing32
  const int rb = i0 - 1, re = i1;
#pragma unroll
  for (int k = 0; k < kLead32; ++k) {
    if (rb + k <= re) slot32_issue(ring[k], M, x, U, V, rb + k, j, lane, hw, halo, hc);
    cpa_commit();
  }
  auto make = [&](const float2 sv, const float2 dv) {
    return x.first ? sv : make_float2(__fmaf_rn(x.beta, dv.x, sv.x), __fmaf_rn(x.beta, dv.y, sv.y));
  };
  auto make1 = [&](float sv, float dv) { return x.first ? sv : __fmaf_rn(x.beta, dv, sv); };
  const float2 z2 = make_float2(0.f, 0.f);
  float2 xn = z2, vn = z2, xc = z2, u0 = z2, v0 = z2;
  float h0 = 0.f, w0 = 0.f;
  size_t off = (size_t)i0 * M.pitch + j;
  for (int r = rb; r <= re; ++r) {
    // every row r + kLead32 and later is still in flight: row r has landed
    cpa_wait<kLead32 - 1>();
    const Slot32& sl = ring[(r - rb) % kRing32];
    const float2 xs = make(sl.S[lane], sl.D[lane]);
    const float2 u1 = sl.U[lane], v1 = sl.V[lane];
    const float h1 = halo ? make1(sl.hs[hk], sl.hd[hk]) : 0.f;
    const float w1 = hw ? sl.hu : 0.f;
    if (r >= i0 + 1) {
      // row i = r - 1, with x below it from row r
      float west = __shfl_up_sync(kFull, xc.y, 1);
      float east = __shfl_down_sync(kFull, xc.x, 1);
      float uw = __shfl_up_sync(kFull, u0.y, 1);
      if (lane == 0) { west = h0; uw = w0; }
      if (lane == 31) east = h0;
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
      off += M.pitch;
    }
    // shift: rows r-1 and r become the rows above and at the next output row
    xn = xc;
    vn = v0;
    xc = xs;
    u0 = u1;
    v0 = v1;
    h0 = h1;
    w0 = w1;
    // refill the slot of row r - 2, whose values the arithmetic above has consumed
    // (rows rb-2 and rb-1 are the ring's two unused slots)
    if (r + kLead32 <= re) slot32_issue(ring[(r + kLead32 - rb) % kRing32], M, x, U, V, r + kLead32, j, lane, hw, halo, hc);
    cpa_commit();
  }
  cpa_wait_all();  // the next tile of this warp refills the same slots
}

// d = s + beta d_old, q = A d in FP32, d^T q FP64-accurate.
// ring: the warp's kRing32 ring slots in shared memory
template <int KIND>
__device__ __forceinline__ void a32_tile(const PcgArgs& a, const MapDesc& M, MapState* S, int t, int lane,
                                         Slot32* ring) {
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
  stencil_tile32(M, g.i0, g.i1, g.j0, lane, M.h.U, M.h.V, x, epi, ring);
  tile_arrive(a, M, S, t, kPhA, dq.value(), 0.0, 0.0, lane);
}

}  // namespace ulp
