// ulp_sweep.cuh -- wavefront triangular sweeps for the no-fill preconditioners
// (Sec. 2 list items 3-5: ILU(0), IC(0), SOR read as SSOR) in natural
// row-major order.
//
// For the symmetric 5-point A with strict lower part L (entries -U_{i,j-1},
// -V_{i-1,j}) all three have the form M = c (P + L) P^-1 (P + L^T):
//   ILU(0) = IC(0): P = pivots p_k = a_kk - U_{i,j-1}^2/p_{k-1} - V_{i-1,j}^2/p_{k-W}, c = 1
//   SSOR(omega):     P = D / omega,                                      c = omega/(2-omega)
// so s = M^-1 r is a forward sweep z_k = (r_k/c + U_{i,j-1} z_{k-1} + V_{i-1,j} z_{k-W}) / P_k
// and a backward sweep s_k = z_k + (U_{i,j} s_{k+1} + V_{i,j} s_{k+W}) / P_k.
// With pinv = 1/P and the coefficient planes cw = U_{i,j-1} pinv, cn = V_{i-1,j} pinv,
// ce = U_{i,j} pinv, cs = V_{i,j} pinv precomputed, each sweep step is two
// dependent FMAs: out = fma(c2, v_nb, fma(c1, v_prev, a)).
//
// Work decomposition: a warp owns a band of 32 rows (one row per lane); lane i
// runs one column behind lane i-1 (forward) or lane i+1 (backward), so the
// neighbour row's value for the same column arrives by a shuffle of the
// previous step.  Band b needs the last row of band b-1 (forward) or the first
// row of band b+1 (backward).  The producing band writes that row a second
// time into an exchange row that holds a signalling-NaN sentinel until the
// value lands, so the value itself is the flag: the consuming band reads the
// values it will need one block of steps ahead with relaxed loads, re-reads
// any that still hold the sentinel (with a time limit), and puts the sentinel
// back after use.  Inputs are loaded PF steps ahead through a register ring.
#pragma once
#include <type_traits>

#include "ulp_internal.cuh"

namespace ulp {

constexpr unsigned long long kSentinelBits = 0x7ff4dead5eed0001ull;  // a NaN no arithmetic produces

__device__ __forceinline__ double sentinel() { return __longlong_as_double((long long)kSentinelBits); }
__device__ __forceinline__ bool is_sentinel(double v) {
  return (unsigned long long)__double_as_longlong(v) == kSentinelBits;
}
__device__ __forceinline__ double ld_relaxed(const double* p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

enum SweepMode { kSweepFwd = 0, kSweepBwd = 1, kSweepPiv = 2 };

struct SweepIO {
  const double* a;   // FWD: r pinv / c    BWD: z      PIV: D
  const double* b;   // FWD: cw            BWD: ce     PIV: U (read at j-1)
  const double* c;   // FWD: cn            BWD: cs     PIV: V (read at i-1)
  double* out;       // FWD: z             BWD: s      PIV: pinv
  double* xin;       // exchange row of the neighbour band (read, then reset), or null
  double* xout;      // this band's exchange row for its neighbour (written), or null
};

// Sweeps one band of one map.  Returns false if a wait ran out (error flag set).
template <int MODE>
__device__ bool band_sweep(const MapDesc& M, int band, int lane, const SweepIO& io,
                           unsigned long long timeout_ns, int* err) {
  constexpr bool FWD = (MODE != kSweepBwd);
  constexpr int PF = 16;  // input prefetch distance in steps
  constexpr int PB = 8;   // boundary block: steps served by one set of exchange reads
  const int H = M.H, W = M.W;
  const size_t P = (size_t)M.pitch;
  const int row0 = band * 32;
  const int nrows = min(32, H - row0);
  const bool act = lane < nrows;
  const int row = act ? row0 + lane : row0;
  const bool has_nb = io.xin != nullptr;
  const int edge = FWD ? 0 : nrows - 1;               // lane that consumes the neighbour's row
  const int pub = FWD ? nrows - 1 : 0;                // lane whose row the neighbour consumes
  const bool publish = io.xout != nullptr;
  const int skew = FWD ? lane : (nrows - 1 - lane);  // steps behind the leading lane
  const int nsteps = W + nrows - 1;

  auto col = [&](int t) -> int {  // column processed at step t, or -1
    const int c = t - skew;
    if (!act || c < 0 || c >= W) return -1;
    return FWD ? c : W - 1 - c;
  };
  auto load = [&](int t, double& va, double& vb, double& vc) {
    const int j = col(t);
    va = vb = vc = 0.0;
    if (j < 0) return;
    const size_t off = (size_t)row * P + j;
    va = __ldcg(io.a + off);
    if (MODE == kSweepPiv) {
      if (j > 0) vb = __ldcg(io.b + off - 1);
      if (row > 0) vc = __ldcg(io.c + off - P);
    } else {
      vb = __ldcg(io.b + off);
      vc = __ldcg(io.c + off);
    }
  };
  // exchange column read by lane l (< PB) for the block starting at step t0 (edge lane: column t0 + l)
  auto xcol = [&](int t0) -> int {
    const int je = t0 + lane;
    if (lane >= PB || je >= W) return -1;
    return FWD ? je : W - 1 - je;
  };

  double ra[PF], rb[PF], rc[PF];
#pragma unroll
  for (int k = 0; k < PF; ++k) load(k, ra[k], rb[k], rc[k]);
  double bcur = 0.0, bnxt = 0.0;
  if (has_nb) {
    const int c0 = xcol(0), c1 = xcol(PB);
    if (c0 >= 0) bcur = ld_relaxed(io.xin + c0);
    if (c1 >= 0) bnxt = ld_relaxed(io.xin + c1);
  }
  double prev = 0.0, carry = 0.0;

  auto block = [&](int t0, auto slot0) -> bool {
    constexpr int S0 = decltype(slot0)::value;
    if (has_nb) {
      // wait for the exchange values of this block, then hand the slots back
      const int c = xcol(t0);
      bool ok = true;
      if (c >= 0 && is_sentinel(bcur)) {
        const unsigned long long t_start = globaltimer();
        do {
          if (*(volatile int*)err) { ok = false; break; }
          if (globaltimer() - t_start > timeout_ns) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          bcur = ld_relaxed(io.xin + c);
        } while (is_sentinel(bcur));
      }
      if (!__all_sync(kFull, ok)) return false;
      if (c >= 0) st_relaxed(io.xin + c, sentinel());
    }
    const double bblk = bcur;
    // exchange reads for the block after next are issued now, a block ahead of use
    bcur = bnxt;
    if (has_nb) {
      const int c2 = xcol(t0 + 2 * PB);
      bnxt = (c2 >= 0) ? ld_relaxed(io.xin + c2) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < PB; ++k) {
      const int t = t0 + k;
      const double va = ra[S0 + k], vb = rb[S0 + k], vc = rc[S0 + k];
      load(t + PF, ra[S0 + k], rb[S0 + k], rc[S0 + k]);
      double nbv = FWD ? __shfl_up_sync(kFull, carry, 1) : __shfl_down_sync(kFull, carry, 1);
      const double bv = __shfl_sync(kFull, bblk, k);
      if (lane == edge) nbv = has_nb ? bv : 0.0;
      const int j = col(t);
      double v = 0.0;
      if (j >= 0) {
        if (MODE == kSweepPiv) {
          // p = a_kk - U_{i,j-1}^2 pinv_{k-1} - V_{i-1,j}^2 pinv_{k-W}, guarded, then 1/p
          double p = fma(-(vc * vc), nbv, fma(-(vb * vb), prev, va));
          if (!(p > 1e-12 * va && p > 0.0)) p = (va > 0.0) ? va : 1.0;
          v = 1.0 / p;
        } else {
          v = fma(vc, nbv, fma(vb, prev, va));
        }
        __stcg(io.out + (size_t)row * P + j, v);
        if (publish && lane == pub) st_relaxed(io.xout + j, v);
        prev = v;
      }
      carry = v;
    }
    return true;
  };

  for (int t0 = 0; t0 < nsteps; t0 += 2 * PB) {
    if (!block(t0, std::integral_constant<int, 0>{})) return false;
    if (t0 + PB < nsteps && !block(t0 + PB, std::integral_constant<int, PB>{})) return false;
  }
  return true;
}

}  // namespace ulp
