// ulp_internal.cuh -- internal types and device helpers of the GB300 L^p
// phase-unwrapping library (not part of the C ABI).
//
// Data layout in HBM: every internal plane of a map is an H x pitch row-major
// array, pitch = W rounded up to a multiple of 64 elements, so each row starts
// on a 512-byte boundary and a warp moving one double2 per lane covers one
// 64-column strip.  Columns W..pitch-1 are zero padding with zero weights, so
// every kernel may treat them as part of the grid.
//
// Work unit: a warp tile = 64 columns x R rows of one map.  Tiles of all maps
// of a call are numbered consecutively (map by map, row band by row band);
// per-tile partial sums make every reduction independent of which warp or
// block processed which tile.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace ulp {

constexpr int kStrip = 64;            // columns per warp tile (32 lanes x double2 / float2)
constexpr int kThreads = 256;         // threads per block of the persistent solver
constexpr int kWarps = kThreads / 32;
constexpr int kMaxMaps = 256;
constexpr unsigned kFull = 0xffffffffu;

enum Kind { kIdentity = 0, kJacobi = 1, kIlu = 2, kIc = 3, kSsor = 4, kDct = 5 };

// FP64 planes of one map (all H x pitch).
struct Planes64 {
  double *dx, *dy;          // wrapped differences (Sec. 2.1)
  double *U, *V;            // Eq. (UV) weights
  double *D, *Dinv;         // diagonal of A and its guarded inverse
  double *b;                // Eq. (Axb) right-hand side
  double *phi, *phi_prev;   // current iterate, previous outer iterate
  double *r, *s, *q;        // PCG residual, preconditioned residual, A d
  double *d0, *d1;          // search direction (ping-pong)
  double *piv;              // 1/P: inverse ILU(0)/IC(0) pivots, or omega/D for SSOR
  double *y;                // forward-sweep result z
  double *cw, *cn, *ce, *cs; // sweep coefficients U_{i,j-1}/P, V_{i-1,j}/P, U_{i,j}/P, V_{i,j}/P
  uint8_t* mask;            // 1 = excluded pixel
};

// FP32 planes of one map for the mixed-precision solver.
struct Planes32 {
  float *U, *V, *Dinv;      // weights (FP32) and Jacobi inverse
  float *x, *r, *s, *q, *d0, *d1;
  float *cw, *cn, *pinv, *y; // sweep coefficients (mixed ILU/SSOR)
};

struct MapDesc {
  int H, W, pitch;
  int nsx, nsy;             // strips (pitch/64) and row bands
  int tile_base, ntiles;    // first tile index, number of tiles
  int refresh;              // true-residual period
  int nbands, band_base;    // 32-row bands of the triangular sweeps
  Planes64 f;
  Planes32 h;
  double *xf, *xb;          // sweep exchange rows: last row of each band (forward), first row (backward)
};

// Mutable per-map solver state (device).
constexpr int kArriveGroups = 32;

struct MapState {
  double delta, delta0, rr, bb, dq, alpha, beta, relres;
  long long iter;
  int status, done, stop_after, outer_active;
  int outer_k, err_flag;
  unsigned arrive, arrive_outer;
  double outer_err;
  long long loops;          // body executions of the graph-driven solve since its start
  unsigned arrive_grp[kArriveGroups];  // two-level tile arrival: tile t counts into group (t - tile_base) % 32
  double gpart[3][kArriveGroups];      // per-group sums of the tile partials, written by each group's last tile
  // learned preconditioner: switch to Jacobi after a stall or a breakdown
  int fallback;             // 1: s = D^-1 r from now on in this solve
  int restart;              // 1: the next beta is 0
  int stall;                // iterations since rr last fell below 0.99 rr_best
  int force_refresh;        // mixed flexible CG: every further iteration recomputes the true residual
  double rr_best;
  int x_clean;              // mixed flexible CG: stopped right after a refresh, so the correction is 0
  int confirm;              // mixed flexible CG: the next body re-evaluates the current iterate on the FP64
                            // true residual without taking a step
  int refresh_next;         // mixed flexible CG: ||r|| fell 100-fold since the last true residual
  int pad3_;
  double rr_ref;            // mixed flexible CG: r^T r of the last true residual
};

// Device-side record of one call (per map), copied to the host at the end.
struct MapStats {
  int status, outer;
  long long inner_total;
  long long inner[64];
  double relres[64];
  double outer_err[64];
  int fallbacks;
  unsigned long long setup_ns;   // device time spent building the preconditioner in this call
  unsigned long long setup_t0;   // %globaltimer at the start of the current set-up (flexible CG)
};

struct Barrier {
  unsigned count;
  unsigned gen;
  int err;
  int pad;
};

// Arguments of the persistent PCG kernels.
struct PcgArgs {
  const MapDesc* maps;
  MapState* st;
  int nmaps, ntiles, R, nbands;
  double *P0, *P1, *P2;     // per-tile partial sums
  Barrier* bar;
  int* n_active;
  int stop_mode;
  double tol2;
  long long lmax;
  unsigned long long timeout_ns;
  double omega;
  int apply_only;           // sweep solvers: stop after the first s = M^-1 r (single-step entry point)
  unsigned long long cond;  // flexible-CG graph: WHILE-node handle cleared when the map stops (0 = none)
  unsigned* rbf;            // flexible-CG graph: BF16 copy of r as column pairs (the DCT input), or null
  unsigned* rbf_lo;         // its low plane (r - bf16(r), BF16 pairs): the DCT's operands are split BF16
  int rbf_ld;               // its row stride in pairs
  float* rf32;              // flexible-CG graph: FP32 copy of r (the multigrid's right-hand side), or null
  int learned;              // flexible CG with the learned preconditioner: stall / breakdown fall back to Jacobi
  int stall_window;
  MapStats* stats;          // per-map statistics (the set-up time is added to map 0's), or null
  int xfcg;                 // mixed flexible CG: convergence of the FP32 recurrence is confirmed on the
                            // FP64 true residual before the solve stops
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_i(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_i(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative (co-resident) grid with a bounded wait.
// Returns false if any block gave up; every caller then leaves the kernel.
__device__ __forceinline__ bool grid_sync(Barrier* b, unsigned long long timeout_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned g = ld_acquire(&b->gen);
    __threadfence();
    unsigned arrived = atomicAdd(&b->count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      st_release(&b->gen, g + 1u);
    } else {
      unsigned long long t0 = globaltimer();
      while (ld_acquire(&b->gen) == g) {
        if (*(volatile int*)&b->err) break;
        if (globaltimer() - t0 > timeout_ns) {
          atomicExch(&b->err, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)&b->err == 0;
}

__device__ __forceinline__ double2 ld2(const double* base, size_t off) {
  return __ldcg(reinterpret_cast<const double2*>(base + off));
}
__device__ __forceinline__ void st2(double* base, size_t off, double2 v) {
  __stcg(reinterpret_cast<double2*>(base + off), v);
}
__device__ __forceinline__ double ld1(const double* base, size_t off) { return __ldcg(base + off); }

// Deterministic warp sum: fixed shfl_down tree, result broadcast from lane 0.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return __shfl_sync(kFull, v, 0);
}

// Fixed-order sum of n partials (stride-32 lanes, 4 accumulators, fixed tree).
__device__ __forceinline__ double warp_sum_partials(const double* P, int n, int lane) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int k = lane;
  for (; k + 96 < n; k += 128) {
    a0 += __ldcg(P + k);
    a1 += __ldcg(P + k + 32);
    a2 += __ldcg(P + k + 64);
    a3 += __ldcg(P + k + 96);
  }
  if (k < n) a0 += __ldcg(P + k);
  if (k + 32 < n) a1 += __ldcg(P + k + 32);
  if (k + 64 < n) a2 += __ldcg(P + k + 64);
  return warp_sum((a0 + a1) + (a2 + a3));
}

// Fixed-order sums of n partials of up to three arrays at once (cnt = 1, 2, 3):
// lane l adds P[l + 32 (8 j + u)] into accumulator u, the 8 cnt loads of a round
// issued together, then a fixed tree over u and over the lanes.  Latency: one
// L2 round trip per 256 partials instead of one per 128 partials and array.
__device__ __forceinline__ void warp_sum_partials3(const double* P0, const double* P1, const double* P2, int cnt,
                                                   int n, int lane, double& v0, double& v1, double& v2) {
  double a0[8], a1[8], a2[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a0[u] = a1[u] = a2[u] = 0.0;
  int k = lane;
  for (; k + 32 * 7 < n; k += 256) {
    double t0[8], t1[8], t2[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      t0[u] = __ldcg(P0 + k + 32 * u);
      t1[u] = cnt > 1 ? __ldcg(P1 + k + 32 * u) : 0.0;
      t2[u] = cnt > 2 ? __ldcg(P2 + k + 32 * u) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      a0[u] += t0[u];
      a1[u] += t1[u];
      a2[u] += t2[u];
    }
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (k + 32 * u < n) {
      a0[u] += __ldcg(P0 + k + 32 * u);
      if (cnt > 1) a1[u] += __ldcg(P1 + k + 32 * u);
      if (cnt > 2) a2[u] += __ldcg(P2 + k + 32 * u);
    }
  }
  v0 = warp_sum(((a0[0] + a0[1]) + (a0[2] + a0[3])) + ((a0[4] + a0[5]) + (a0[6] + a0[7])));
  v1 = cnt > 1 ? warp_sum(((a1[0] + a1[1]) + (a1[2] + a1[3])) + ((a1[4] + a1[5]) + (a1[6] + a1[7]))) : 0.0;
  v2 = cnt > 2 ? warp_sum(((a2[0] + a2[1]) + (a2[2] + a2[3])) + ((a2[4] + a2[5]) + (a2[6] + a2[7]))) : 0.0;
}

__device__ __forceinline__ int find_map(const int* base, int nmaps, int t) {
  int lo = 0, hi = nmaps - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Principal value onto (-pi, pi] (Eq. wrapped): x - 2 pi ceil((x - pi) / (2 pi)).
__device__ __forceinline__ double wrap_pv(double x) {
  const double pi = 3.14159265358979323846;
  const double two_pi = 2.0 * pi;
  double k = ceil(__ddiv_rn(__dsub_rn(x, pi), two_pi));
  return __dsub_rn(x, __dmul_rn(two_pi, k));
}

}  // namespace ulp
