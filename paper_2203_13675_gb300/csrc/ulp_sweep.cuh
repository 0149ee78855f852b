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
// row of band b+1 (backward): the producing band publishes how many columns of
// that row it has finished (64-bit flag: epoch << 32 | columns, release order)
// and the consuming band waits on it with an acquire load and a time limit.
// Inputs are loaded PF steps ahead through a register ring.
#pragma once
#include "ulp_internal.cuh"

namespace ulp {

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

enum SweepMode { kSweepFwd = 0, kSweepBwd = 1, kSweepPiv = 2 };

struct SweepIO {
  const double* a;   // FWD: r pinv / c    BWD: z      PIV: D
  const double* b;   // FWD: cw            BWD: ce     PIV: U (read at j-1)
  const double* c;   // FWD: cn            BWD: cs     PIV: V (read at i-1)
  double* out;       // FWD: z             BWD: s      PIV: pinv
};

// Sweeps one band of one map.  Returns false if a wait ran out (error flag set).
template <int MODE>
__device__ bool band_sweep(const MapDesc& M, int band, int lane, unsigned long long* prog,
                           unsigned long long epoch, const SweepIO& io,
                           unsigned long long timeout_ns, int* err) {
  constexpr bool FWD = (MODE != kSweepBwd);
  constexpr int PF = 4;  // prefetch distance in steps (one boundary fetch covers PF columns)
  const int H = M.H, W = M.W, nb = M.nbands;
  const size_t P = (size_t)M.pitch;
  const int row0 = band * 32;
  const int nrows = min(32, H - row0);
  const bool act = lane < nrows;
  const int row = act ? row0 + lane : row0;
  const bool has_nb = FWD ? (band > 0) : (band + 1 < nb);
  const int nbrow = FWD ? row0 - 1 : row0 + 32;
  const int edge = FWD ? 0 : nrows - 1;               // lane that reads the neighbour band
  const int pub = FWD ? nrows - 1 : 0;                // lane whose row the neighbour band needs
  const bool publish = FWD ? (band + 1 < nb) : (band > 0);
  const int skew = FWD ? lane : (nrows - 1 - lane);  // steps behind the leading lane
  const int nsteps = W + nrows - 1;
  unsigned long long* my_flag = prog + band;
  const unsigned long long* nb_flag = prog + (FWD ? band - 1 : band + 1);

  // column processed at step t, or -1
  auto col = [&](int t) -> int {
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

  double ra[PF], rb[PF], rc[PF];
#pragma unroll
  for (int k = 0; k < PF; ++k) load(k, ra[k], rb[k], rc[k]);
  double prev = 0.0, carry = 0.0, buf = 0.0;
  for (int t0 = 0; t0 < nsteps; t0 += PF) {
    // neighbour band's boundary row for the edge lane's next PF columns
    if (has_nb) {
      bool ok = true;
      if (lane < PF && t0 < W) {
        const unsigned long long need = (epoch << 32) | (unsigned long long)min(t0 + PF, W);
        const unsigned long long t_start = globaltimer();
        while (ld_acquire64(nb_flag) < need) {
          if (*(volatile int*)err) { ok = false; break; }
          if (globaltimer() - t_start > timeout_ns) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
        }
        const int je = t0 + lane;  // edge lane's step -> column
        buf = 0.0;
        if (ok && je < W) buf = __ldcg(io.out + (size_t)nbrow * P + (FWD ? je : W - 1 - je));
      }
      if (!__all_sync(kFull, ok)) return false;
    }
#pragma unroll
    for (int k = 0; k < PF; ++k) {
      const int t = t0 + k;
      const double va = ra[k], vb = rb[k], vc = rc[k];
      load(t + PF, ra[k], rb[k], rc[k]);
      double nbv = FWD ? __shfl_up_sync(kFull, carry, 1) : __shfl_down_sync(kFull, carry, 1);
      const double bv = __shfl_sync(kFull, buf, k);
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
        prev = v;
      }
      carry = v;
      if (publish && lane == pub && j >= 0) {
        const int cnt = t - skew + 1;
        if ((cnt & 7) == 0 || cnt == W) st_release64(my_flag, (epoch << 32) | (unsigned long long)cnt);
      }
    }
  }
  return true;
}

}  // namespace ulp
