// ulp_mg.cu -- aggregation-multigrid preconditioner: s = one symmetric V-cycle
// applied to r (the paper names multigrid next to the Fourier methods as the
// fast solvers of this system, Sec. 1).
//
// Grids: level 0 is the map (the plan's U, V, D^-1 planes with their pitch);
// level l+1 aggregates 2x2 cells of level l (clipped at the border), and its
// operator is the Galerkin product P^T A_l P, which for piecewise-constant P is
// again a 5-point weighted Laplacian whose edge weights are the sums of the
// fine edges crossing between aggregates.  Grids stop at 16 unknowns.
// Cycle, per level: two damped-Jacobi sweeps (omega = 2/3) from zero, the
// residual restricted by summing over each aggregate, the coarse cycle, the
// correction prolonged and scaled by 1.5, two more sweeps; thirty sweeps from
// zero on the coarsest grid.  The same number of sweeps before and after keeps
// the cycle symmetric.  Fusions (the values each thread needs at its
// neighbours are recomputed there, not read back):
//   K_pre    both pre-sweeps: x1 = w D^-1 b is elementwise, so x2 needs no pass of its own
//   K_res    residual b - A x and the restriction, one thread per aggregate
//   K_post1  prolongation + correction + the first post-sweep
//   K_post2  the second post-sweep (and, on level 0, the mask)
// The cycle runs in FP32: on GB300 FP64 issues at 1/64 of the FP32 rate, and
// these fused sweeps spend about 22 arithmetic instructions per pixel, which in
// FP64 made the cycle issue-bound at several times its memory time.  Level 0
// keeps FP32 copies of the map's U, V, D^-1 (made once per solve) and of r;
// the result s is written in FP64.  The flexible CG around it, its vectors and
// its scalars stay FP64; one application matches the FP64 oracle's cycle to
// FP32 rounding.
#include <vector>

#include "ulp_mixed.cuh"
#include "ulp_host.h"

namespace ulp {

namespace mg {

constexpr int kCoarseSweeps = 30;
constexpr long long kCoarseMax = 16;

// One grid: edge weights, D^-1 and vectors (FP32), row stride ld.
struct Grid {
  int H, W, ld;
  const float *U, *V, *Dinv;
  float *x, *b, *t;
};

constexpr float kOmegaF = (float)(2.0 / 3.0);
constexpr float kCCF = 1.5f;

#define MG_LOOP(t, n) for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (n); t += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ bool skip_map(const MapState* S) { return S && *(volatile const int*)&S->done; }

// (A x)_{ij} with x given by a functor xv(i, j)
template <class XV>
__device__ __forceinline__ float ax_at(const Grid& g, int i, int j, const XV& xv) {
  const size_t o = (size_t)i * g.ld + j;
  float acc = 0.f;
  float d = g.U[o] + g.V[o];
  if (j + 1 < g.W) acc -= g.U[o] * xv(i, j + 1);
  if (j > 0) {
    d += g.U[o - 1];
    acc -= g.U[o - 1] * xv(i, j - 1);
  }
  if (i + 1 < g.H) acc -= g.V[o] * xv(i + 1, j);
  if (i > 0) {
    d += g.V[o - g.ld];
    acc -= g.V[o - g.ld] * xv(i - 1, j);
  }
  return d * xv(i, j) + acc;
}

// Coarse weights and D^-1 of level l+1 from level l (one thread per aggregate).
__global__ void k_mg_coarsen(Grid f, Grid c, const MapState* S) {
  if (skip_map(S)) return;
  MG_LOOP(t, (long long)c.H * c.W) {
    const int I = (int)(t / c.W), J = (int)(t % c.W);
    // U_c(I, J') for J' = J - 1, J and V_c(I', J) for I' = I - 1, I
    auto uc = [&](int Jp) {
      float u = 0.f;
      if (Jp >= 0 && 2 * Jp + 2 < f.W)
        for (int i = 2 * I; i <= 2 * I + 1 && i < f.H; ++i) u += f.U[(size_t)i * f.ld + 2 * Jp + 1];
      return u;
    };
    auto vc = [&](int Ip) {
      float v = 0.f;
      if (Ip >= 0 && 2 * Ip + 2 < f.H)
        for (int j = 2 * J; j <= 2 * J + 1 && j < f.W; ++j) v += f.V[(size_t)(2 * Ip + 1) * f.ld + j];
      return v;
    };
    const float u = uc(J), v = vc(I);
    const float d = u + v + uc(J - 1) + vc(I - 1);
    const size_t o = (size_t)I * c.ld + J;
    const_cast<float*>(c.U)[o] = u;
    const_cast<float*>(c.V)[o] = v;
    const_cast<float*>(c.Dinv)[o] = d > 0.f ? 1.f / d : 0.f;
  }
}

// The coarse grids from index l0 on, made one after the other by one block (the
// small grids of the hierarchy: one launch instead of one per grid).
struct CoarsenList {
  int n;          // grids g[0..n-1]: g[k+1] is made from g[k]
  Grid g[16];
};

__global__ void __launch_bounds__(1024) k_mg_coarsen_small(CoarsenList cl, const MapState* S) {
  if (skip_map(S)) return;
  for (int k = 0; k + 1 < cl.n; ++k) {
    const Grid& f = cl.g[k];
    const Grid& c = cl.g[k + 1];
    for (int t = threadIdx.x; t < c.H * c.W; t += blockDim.x) {
      const int I = t / c.W, J = t - (t / c.W) * c.W;
      auto uc = [&](int Jp) {
        float u = 0.f;
        if (Jp >= 0 && 2 * Jp + 2 < f.W)
          for (int i = 2 * I; i <= 2 * I + 1 && i < f.H; ++i) u += f.U[(size_t)i * f.ld + 2 * Jp + 1];
        return u;
      };
      auto vc = [&](int Ip) {
        float v = 0.f;
        if (Ip >= 0 && 2 * Ip + 2 < f.H)
          for (int j = 2 * J; j <= 2 * J + 1 && j < f.W; ++j) v += f.V[(size_t)(2 * Ip + 1) * f.ld + j];
        return v;
      };
      const float u = uc(J), v = vc(I);
      const float d = u + v + uc(J - 1) + vc(I - 1);
      const size_t o = (size_t)I * c.ld + J;
      const_cast<float*>(c.U)[o] = u;
      const_cast<float*>(c.V)[o] = v;
      const_cast<float*>(c.Dinv)[o] = d > 0.f ? 1.f / d : 0.f;
    }
    __syncthreads();
  }
}

// x = two damped-Jacobi sweeps from zero
__global__ void k_mg_pre(Grid g, const MapState* S) {
  if (skip_map(S)) return;
  MG_LOOP(t, (long long)g.H * g.W) {
    const int i = (int)(t / g.W), j = (int)(t % g.W);
    const size_t o = (size_t)i * g.ld + j;
    auto x1 = [&](int a, int c) {
      const size_t p = (size_t)a * g.ld + c;
      return kOmegaF * g.Dinv[p] * g.b[p];
    };
    const float ax = ax_at(g, i, j, x1);
    g.x[o] = x1(i, j) + kOmegaF * g.Dinv[o] * (g.b[o] - ax);
  }
}

// b_c = P^T (b - A x): one thread per aggregate
__global__ void k_mg_res(Grid f, Grid c, const MapState* S) {
  if (skip_map(S)) return;
  MG_LOOP(t, (long long)c.H * c.W) {
    const int I = (int)(t / c.W), J = (int)(t % c.W);
    auto xv = [&](int a, int cc) { return f.x[(size_t)a * f.ld + cc]; };
    float acc = 0.f;
    for (int i = 2 * I; i <= 2 * I + 1 && i < f.H; ++i)
      for (int j = 2 * J; j <= 2 * J + 1 && j < f.W; ++j)
        acc += f.b[(size_t)i * f.ld + j] - ax_at(f, i, j, xv);
    c.b[(size_t)I * c.ld + J] = acc;
  }
}

// t = x' + w D^-1 (b - A x'), x' = x + cc P x_c
__global__ void k_mg_post1(Grid f, Grid c, const MapState* S) {
  if (skip_map(S)) return;
  MG_LOOP(t, (long long)f.H * f.W) {
    const int i = (int)(t / f.W), j = (int)(t % f.W);
    const size_t o = (size_t)i * f.ld + j;
    auto xp = [&](int a, int cc) {
      return f.x[(size_t)a * f.ld + cc] + kCCF * c.x[(size_t)(a >> 1) * c.ld + (cc >> 1)];
    };
    const float ax = ax_at(f, i, j, xp);
    f.t[o] = xp(i, j) + kOmegaF * f.Dinv[o] * (f.b[o] - ax);
  }
}

// x = t + w D^-1 (b - A t); on level 0 written in FP64 into s (zero on masked pixels)
__global__ void k_mg_post2(Grid g, const uint8_t* mask, double* s, const MapState* S) {
  if (skip_map(S)) return;
  MG_LOOP(t, (long long)g.H * g.W) {
    const int i = (int)(t / g.W), j = (int)(t % g.W);
    const size_t o = (size_t)i * g.ld + j;
    auto tv = [&](int a, int cc) { return g.t[(size_t)a * g.ld + cc]; };
    const float ax = ax_at(g, i, j, tv);
    const float v = g.t[o] + kOmegaF * g.Dinv[o] * (g.b[o] - ax);
    if (s) s[o] = (mask && mask[o]) ? 0.0 : (double)v;
    else g.x[o] = v;
  }
}

// level 0: FP32 copies of the map's U, V, D^-1 (once per solve)
__global__ void k_mg_level0(const double* __restrict__ U, const double* __restrict__ V,
                            const double* __restrict__ Dinv, Grid g, const MapState* S) {
  if (skip_map(S)) return;
  MG_LOOP(t, (long long)g.H * g.W) {
    const size_t o = (size_t)(t / g.W) * g.ld + (t % g.W);
    const_cast<float*>(g.U)[o] = (float)U[o];
    const_cast<float*>(g.V)[o] = (float)V[o];
    const_cast<float*>(g.Dinv)[o] = (float)Dinv[o];
  }
}

// level 0: b = (float) r
__global__ void k_mg_rhs(const double* __restrict__ r, Grid g, const MapState* S) {
  if (skip_map(S)) return;
  MG_LOOP(t, (long long)g.H * g.W) {
    const size_t o = (size_t)(t / g.W) * g.ld + (t % g.W);
    g.b[o] = (float)r[o];
  }
}

// coarsest grid: thirty sweeps from zero in one block (x and t ping-pong)
__global__ void k_mg_coarsest(Grid g, const MapState* S) {
  if (skip_map(S)) return;
  const int n = g.H * g.W;
  for (int k = threadIdx.x; k < n; k += blockDim.x) g.x[(size_t)(k / g.W) * g.ld + k % g.W] = 0.f;
  __syncthreads();
  float* src = g.x;
  float* dst = g.t;
  for (int s = 0; s < kCoarseSweeps; ++s) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const int i = k / g.W, j = k % g.W;
      const size_t o = (size_t)i * g.ld + j;
      auto xv = [&](int a, int c) { return src[(size_t)a * g.ld + c]; };
      dst[o] = src[o] + kOmegaF * g.Dinv[o] * (g.b[o] - ax_at(g, i, j, xv));
    }
    __syncthreads();
    float* tmp = src;
    src = dst;
    dst = tmp;
  }
  if (src != g.x) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const size_t o = (size_t)(k / g.W) * g.ld + k % g.W;
      g.x[o] = src[o];
    }
  }
}


// ---------------------------------------------------------------- vector kernels (wide grids)
// A thread owns 4 consecutive pixels of a row (float4 accesses: on GB300 one
// float per thread per load leaves too few bytes in flight to keep HBM busy), a
// warp 128 columns of one row.  The column neighbours of a thread's pixels come
// from the neighbouring lanes by shuffles (two scalar loads at the warp's ends),
// the rows above and below as float4 loads.  Rows are padded to a multiple of 4
// floats; values at columns >= W are taken as 0.  Same arithmetic per pixel as
// the per-pixel kernels.
enum { kSrcX1 = 0, kSrcXP = 1, kSrcT = 2, kSrcX = 3 };

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float f4(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

// the source vector at (i, j..j+3) of grid f (0 outside the grid)
template <int SRC>
__device__ __forceinline__ float4 src4(const Grid& f, const Grid& c, int i, int j) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i < 0 || i >= f.H || j >= f.W) return v;
  const size_t o = (size_t)i * f.ld + j;
  if (SRC == kSrcX1) {
    const float4 d = ld4(f.Dinv + o), b = ld4(f.b + o);
    v = make_float4(kOmegaF * d.x * b.x, kOmegaF * d.y * b.y, kOmegaF * d.z * b.z, kOmegaF * d.w * b.w);
  } else if (SRC == kSrcXP) {
    const float4 x = ld4(f.x + o);
    const float2 xc = *reinterpret_cast<const float2*>(c.x + (size_t)(i >> 1) * c.ld + (j >> 1));
    v = make_float4(x.x + kCCF * xc.x, x.y + kCCF * xc.x, x.z + kCCF * xc.y, x.w + kCCF * xc.y);
  } else if (SRC == kSrcT) {
    v = ld4(f.t + o);
  } else {
    v = ld4(f.x + o);
  }
  if (j + 1 >= f.W) v.y = 0.f;
  if (j + 2 >= f.W) v.z = 0.f;
  if (j + 3 >= f.W) v.w = 0.f;
  return v;
}
// one pixel of the source (halo of a warp's segment)
template <int SRC>
__device__ __forceinline__ float src1(const Grid& f, const Grid& c, int i, int j) {
  if (i < 0 || i >= f.H || j < 0 || j >= f.W) return 0.f;
  const size_t o = (size_t)i * f.ld + j;
  if (SRC == kSrcX1) return kOmegaF * f.Dinv[o] * f.b[o];
  if (SRC == kSrcXP) return f.x[o] + kCCF * c.x[(size_t)(i >> 1) * c.ld + (j >> 1)];
  if (SRC == kSrcT) return f.t[o];
  return f.x[o];
}
__device__ __forceinline__ float4 w4(const float* p, int i, int j, const Grid& f) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i < 0 || i >= f.H || j >= f.W) return v;
  v = ld4(p + (size_t)i * f.ld + j);
  if (j + 1 >= f.W) v.y = 0.f;
  if (j + 2 >= f.W) v.z = 0.f;
  if (j + 3 >= f.W) v.w = 0.f;
  return v;
}

// (A x) at the 4 pixels (i, j..j+3); xc, xn, xs the source at rows i, i-1, i+1
template <int SRC>
__device__ __forceinline__ float4 ax4(const Grid& f, const Grid& c, int i, int j, int lane, float4 xc, float4 xn,
                                      float4 xs) {
  const float4 U = w4(f.U, i, j, f), V = w4(f.V, i, j, f), Vn = w4(f.V, i - 1, j, f);
  float ul = __shfl_up_sync(0xffffffffu, U.w, 1);
  float xl = __shfl_up_sync(0xffffffffu, xc.w, 1);
  float xr = __shfl_down_sync(0xffffffffu, xc.x, 1);
  if (lane == 0) {
    ul = (j > 0 && i < f.H && j - 1 < f.W) ? f.U[(size_t)i * f.ld + j - 1] : 0.f;
    xl = src1<SRC>(f, c, i, j - 1);
  }
  if (lane == 31) xr = src1<SRC>(f, c, i, j + 4);
  const float uw[4] = {ul, U.x, U.y, U.z};
  const float ue[4] = {U.x, U.y, U.z, U.w};
  const float xw[4] = {xl, xc.x, xc.y, xc.z};
  const float xe[4] = {xc.y, xc.z, xc.w, xr};
  float out[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float d = ue[k] + f4(V, k) + uw[k] + f4(Vn, k);
    out[k] = d * f4(xc, k) - ue[k] * xe[k] - uw[k] * xw[k] - f4(V, k) * f4(xs, k) - f4(Vn, k) * f4(xn, k);
  }
  return make_float4(out[0], out[1], out[2], out[3]);
}

__device__ __forceinline__ bool warp_row(const Grid& f, int rows, int& i, int& j, int& lane) {
  const int nseg = (f.W + 127) / 128;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  lane = threadIdx.x & 31;
  if (w >= rows * nseg) return false;
  i = w / nseg;
  j = (w % nseg) * 128 + 4 * lane;
  return true;
}

// out = src + w D^-1 (b - A src) on row i (SRC x1: pre-smoothing, xp: first post-sweep, t: second)
template <int SRC>
__global__ void __launch_bounds__(256) k_mg_sweep_v(Grid f, Grid c, float* out, const uint8_t* mask, double* s,
                                                    const MapState* S) {
  if (skip_map(S)) return;
  int i, j, lane;
  if (!warp_row(f, f.H, i, j, lane)) return;
  const float4 xc = src4<SRC>(f, c, i, j), xn = src4<SRC>(f, c, i - 1, j), xs = src4<SRC>(f, c, i + 1, j);
  const float4 ax = ax4<SRC>(f, c, i, j, lane, xc, xn, xs);
  if (j >= f.W) return;
  const size_t o = (size_t)i * f.ld + j;
  const float4 D = ld4(f.Dinv + o), b = ld4(f.b + o);
  const float4 v = make_float4(xc.x + kOmegaF * D.x * (b.x - ax.x), xc.y + kOmegaF * D.y * (b.y - ax.y),
                               xc.z + kOmegaF * D.z * (b.z - ax.z), xc.w + kOmegaF * D.w * (b.w - ax.w));
  if (s) {
    // the map's grid: s in FP64, 0 on masked pixels and nothing beyond column W - 1
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (j + k < f.W) s[o + k] = (mask && mask[o + k]) ? 0.0 : (double)f4(v, k);
  } else {
    *reinterpret_cast<float4*>(out + o) = v;
  }
}

// residual and restriction: rows 2I, 2I+1 of a thread's 4 columns -> b_c(I, j/2), b_c(I, j/2 + 1)
__global__ void __launch_bounds__(256) k_mg_res_v(Grid f, Grid c, const MapState* S) {
  if (skip_map(S)) return;
  int I, j, lane;
  if (!warp_row(f, c.H, I, j, lane)) return;
  const int i = 2 * I;
  const float4 x0 = src4<kSrcX>(f, c, i - 1, j), x1 = src4<kSrcX>(f, c, i, j), x2 = src4<kSrcX>(f, c, i + 1, j),
               x3 = src4<kSrcX>(f, c, i + 2, j);
  const float4 a1 = ax4<kSrcX>(f, c, i, j, lane, x1, x0, x2);
  const float4 a2 = ax4<kSrcX>(f, c, i + 1, j, lane, x2, x1, x3);
  if (j >= f.W) return;
  const float4 b1 = w4(f.b, i, j, f), b2 = w4(f.b, i + 1, j, f);
  const bool r2 = i + 1 < f.H;
  float lo = (b1.x - a1.x) + (b1.y - a1.y), hi = (b1.z - a1.z) + (b1.w - a1.w);
  if (r2) {
    lo += (b2.x - a2.x) + (b2.y - a2.y);
    hi += (b2.z - a2.z) + (b2.w - a2.w);
  }
  // columns beyond W - 1 contribute 0: their b is 0 and A x there is 0 (zero weights, zero x)
  *reinterpret_cast<float2*>(c.b + (size_t)I * c.ld + (j >> 1)) = make_float2(lo, hi);
}

// level 0: b = (float) r, four pixels per thread
__global__ void k_mg_rhs_v(const double* __restrict__ r, Grid g, const MapState* S) {
  if (skip_map(S)) return;
  const int nq = (g.W + 3) / 4;
  MG_LOOP(t, (long long)g.H * nq) {
    const int i = (int)(t / nq), j = (int)(t % nq) * 4;
    const size_t o = (size_t)i * g.ld + j;
    float4 v;
    v.x = (float)r[o];
    v.y = j + 1 < g.W ? (float)r[o + 1] : 0.f;
    v.z = j + 2 < g.W ? (float)r[o + 2] : 0.f;
    v.w = j + 3 < g.W ? (float)r[o + 3] : 0.f;
    *reinterpret_cast<float4*>(g.b + o) = v;
  }
}

// ---------------------------------------------------------------- tiled fused kernels
// One launch per grid and direction.  A block of 256 threads owns a tile: a
// window of 128 columns starting at j0 = 120 k - 4 (four pixels per lane, float4
// accesses; lanes 1..30 produce the window's inner 120 columns, lanes 0 and 31
// only supply column neighbours, exact two sweeps deep because the window extends
// four columns past the output on each side) and TR rows, plus the two rows above
// and below that two sweeps reach.  The block issues every load of its tile at
// once into shared memory (one memory round trip), then runs each sweep over the
// tile from shared memory with a block barrier in between; the halo rows and
// columns are recomputed, so no value crosses between blocks within a launch.
//   k_mg_down: x1 = w D^-1 b, x2 = x1 + w D^-1 (b - A x1) (both pre-sweeps), x = x2
//              written, and b_c = P^T (b - A x2) (residual + restriction)
//   k_mg_up:   x' = x + cc P x_c, t = x' + w D^-1 (b - A x'), s = t + w D^-1 (b - A t);
//              s goes to the grid's t plane (x is still being read by the
//              neighbouring tiles), or on the map's grid to the FP64 s (0 on
//              masked pixels) or to the FP32 s of the mixed solve, where the block
//              also sums r^T s and r^T r for the flexible CG's dot phase.
// Per pixel the arithmetic is that of the per-step kernels above.
constexpr int kSegOut = 120;
constexpr int kWin = 128;
constexpr int kTileThreads = 256;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kTileMaxRows = 16;                                   // TR <= 16
constexpr int kTilePlane = (kTileMaxRows + 4) * kWin;              // floats per shared plane
constexpr size_t kTileSmem = 6 * kTilePlane * sizeof(float);        // six planes: 61,440 bytes

// row i of a plane at the lane's 4 columns from j: 0 outside the grid
__device__ __forceinline__ float4 lrow(const float* p, const Grid& f, int i, int j) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i >= 0 && i < f.H && j >= 0 && j < f.W) v = ld4(p + (size_t)i * f.ld + j);
  v.y = j + 1 < f.W ? v.y : 0.f;
  v.z = j + 2 < f.W ? v.z : 0.f;
  v.w = j + 3 < f.W ? v.w : 0.f;
  return v;
}

// (A y) at the lane's 4 pixels of row i: y at rows i-1, i, i+1, U and V of row i, V of
// row i-1; column neighbours from the adjacent lanes (lanes 0 and 31 take 0 outside)
__device__ __forceinline__ float4 arow(const float4& yn, const float4& yc, const float4& ys, const float4& U,
                                       const float4& V, const float4& Vn, int lane) {
  float ul = __shfl_up_sync(0xffffffffu, U.w, 1);
  float yl = __shfl_up_sync(0xffffffffu, yc.w, 1);
  float yr = __shfl_down_sync(0xffffffffu, yc.x, 1);
  if (lane == 0) ul = yl = 0.f;
  if (lane == 31) yr = 0.f;
  const float uw[4] = {ul, U.x, U.y, U.z};
  const float ue[4] = {U.x, U.y, U.z, U.w};
  const float yw[4] = {yl, yc.x, yc.y, yc.z};
  const float ye[4] = {yc.y, yc.z, yc.w, yr};
  float out[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float d = ue[k] + f4(V, k) + uw[k] + f4(Vn, k);
    out[k] = d * f4(yc, k) - ue[k] * ye[k] - uw[k] * yw[k] - f4(V, k) * f4(ys, k) - f4(Vn, k) * f4(yn, k);
  }
  return make_float4(out[0], out[1], out[2], out[3]);
}

// y + w D^-1 (b - a)
__device__ __forceinline__ float4 jac4(const float4& y, const float4& D, const float4& b, const float4& a) {
  return make_float4(y.x + kOmegaF * D.x * (b.x - a.x), y.y + kOmegaF * D.y * (b.y - a.y),
                     y.z + kOmegaF * D.z * (b.z - a.z), y.w + kOmegaF * D.w * (b.w - a.w));
}

__device__ __forceinline__ float4 lds4(const float* p, int rr, int lane) {
  return *reinterpret_cast<const float4*>(p + rr * kWin + 4 * lane);
}
__device__ __forceinline__ void sts4(float* p, int rr, int lane, const float4& v) {
  *reinterpret_cast<float4*>(p + rr * kWin + 4 * lane) = v;
}

// pre-smoothing + residual + restriction for the fine rows [TR band, TR band + TR), TR even
__global__ void __launch_bounds__(kTileThreads) k_mg_down_t(Grid f, Grid c, int TR, const MapState* S) {
  if (skip_map(S)) return;
  extern __shared__ float4 tsm4[];
  float* sU = reinterpret_cast<float*>(tsm4);
  float* sV = sU + kTilePlane;
  float* sD = sV + kTilePlane;
  float* sB = sD + kTilePlane;
  float* sX1 = sB + kTilePlane;
  float* sX2 = sX1 + kTilePlane;
  const int nseg = (f.W + kSegOut - 1) / kSegOut;
  const int seg = blockIdx.x % nseg, band = blockIdx.x / nseg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = seg * kSegOut - 4 + 4 * lane;
  const bool out = lane >= 1 && lane <= 30 && j < f.W;
  const int r0 = band * TR, r1 = min(f.H, r0 + TR);
  const int nrow = r1 - r0 + 4;  // rows r0-2 .. r1+1, shared row rr = r - r0 + 2
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int rr = warp; rr < nrow; rr += kTileWarps) {
    const int r = r0 - 2 + rr;
    const float4 U = lrow(f.U, f, r, j), V = lrow(f.V, f, r, j), D = lrow(f.Dinv, f, r, j), B = lrow(f.b, f, r, j);
    sts4(sU, rr, lane, U);
    sts4(sV, rr, lane, V);
    sts4(sD, rr, lane, D);
    sts4(sB, rr, lane, B);
    sts4(sX1, rr, lane,
         make_float4(kOmegaF * D.x * B.x, kOmegaF * D.y * B.y, kOmegaF * D.z * B.z, kOmegaF * D.w * B.w));
  }
  __syncthreads();
  // x2 at rows r0-1 .. r1 (0 outside the grid)
  for (int rr = 1 + warp; rr <= nrow - 2; rr += kTileWarps) {
    const int r = r0 - 2 + rr;
    float4 X2 = z;
    if (r >= 0 && r < f.H) {
      const float4 xc = lds4(sX1, rr, lane);
      X2 = jac4(xc, lds4(sD, rr, lane), lds4(sB, rr, lane),
                arow(lds4(sX1, rr - 1, lane), xc, lds4(sX1, rr + 1, lane), lds4(sU, rr, lane), lds4(sV, rr, lane),
                     lds4(sV, rr - 1, lane), lane));
      if (out && r >= r0 && r < r1) *reinterpret_cast<float4*>(f.x + (size_t)r * f.ld + j) = X2;
    }
    sts4(sX2, rr, lane, X2);
  }
  __syncthreads();
  // residual at the fine rows 2I, 2I+1, summed over the aggregate's two columns and two rows
  for (int I = r0 / 2 + warp; 2 * I < r1; I += kTileWarps) {
    const int p = 2 * I, rr = p - r0 + 2;
    const float4 x0 = lds4(sX2, rr - 1, lane), x1 = lds4(sX2, rr, lane), x2 = lds4(sX2, rr + 1, lane);
    const float4 a1 = arow(x0, x1, x2, lds4(sU, rr, lane), lds4(sV, rr, lane), lds4(sV, rr - 1, lane), lane);
    const float4 b1 = lds4(sB, rr, lane);
    float lo = (b1.x - a1.x) + (b1.y - a1.y), hi = (b1.z - a1.z) + (b1.w - a1.w);
    if (p + 1 < f.H) {
      const float4 a2 = arow(x1, x2, lds4(sX2, rr + 2, lane), lds4(sU, rr + 1, lane), lds4(sV, rr + 1, lane),
                             lds4(sV, rr, lane), lane);
      const float4 b2 = lds4(sB, rr + 1, lane);
      lo += (b2.x - a2.x) + (b2.y - a2.y);
      hi += (b2.z - a2.z) + (b2.w - a2.w);
    }
    if (out) *reinterpret_cast<float2*>(c.b + (size_t)I * c.ld + (j >> 1)) = make_float2(lo, hi);
  }
}

// prolongation + correction + both post-sweeps for the rows [TR band, TR band + TR).
// xc: the coarse grid's corrected solution.  MODE kUpCoarse: s to the grid's t plane.
// kUp64 (the map's grid): s in FP64; with pa, r^T s and r^T r (r: the map's FP64
// residual) over the block's pixels arrive in the flexible CG's dot phase.  kUp32 (the
// map's grid, mixed flexible CG): s in FP32 into s32; with pa, the same dot phase in
// double-float sums of exact FP32 products, r being the cycle's right-hand side.
enum { kUpCoarse = 0, kUp64 = 1, kUp32 = 2 };
template <int MODE>
__global__ void __launch_bounds__(kTileThreads) k_mg_up_t(Grid f, Grid c, const float* __restrict__ xc, int TR,
                                                        const uint8_t* mask, double* s, const double* __restrict__ rv,
                                                        float* s32, const PcgArgs* pa, const MapState* S, int ph) {
  constexpr bool MAP = MODE != kUpCoarse;
  constexpr int kOut = kTileMaxRows / kTileWarps;  // output rows per warp at most
  if (skip_map(S)) return;
  extern __shared__ float4 tsm4[];
  __shared__ double red[2][kTileWarps];
  float* sU = reinterpret_cast<float*>(tsm4);
  float* sV = sU + kTilePlane;
  float* sD = sV + kTilePlane;
  float* sB = sD + kTilePlane;
  float* sXP = sB + kTilePlane;
  float* sT = sXP + kTilePlane;
  const int nseg = (f.W + kSegOut - 1) / kSegOut;
  const int seg = blockIdx.x % nseg, band = blockIdx.x / nseg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = seg * kSegOut - 4 + 4 * lane;
  const bool out = lane >= 1 && lane <= 30 && j < f.W;
  const int r0 = band * TR, r1 = min(f.H, r0 + TR);
  const int nrow = r1 - r0 + 4;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  // the map's grid: mask and FP64 r of this warp's output rows, loaded with the tile
  uchar4 mk[kOut];
  double2 ra[kOut], rb[kOut];
#pragma unroll
  for (int k = 0; k < kOut; ++k) {
    mk[k] = make_uchar4(0, 0, 0, 0);
    ra[k] = rb[k] = make_double2(0.0, 0.0);
    const int r = r0 + warp + kTileWarps * k;
    if (MAP && r < r1 && j >= 0 && j < f.W) {
      const size_t o = (size_t)r * f.ld + j;
      if (mask) mk[k] = *reinterpret_cast<const uchar4*>(mask + o);
      if (MODE == kUp64 && rv) {
        ra[k] = *reinterpret_cast<const double2*>(rv + o);
        rb[k] = *reinterpret_cast<const double2*>(rv + o + 2);
      }
    }
  }
  for (int rr = warp; rr < nrow; rr += kTileWarps) {
    const int r = r0 - 2 + rr;
    sts4(sU, rr, lane, lrow(f.U, f, r, j));
    sts4(sV, rr, lane, lrow(f.V, f, r, j));
    sts4(sD, rr, lane, lrow(f.Dinv, f, r, j));
    sts4(sB, rr, lane, lrow(f.b, f, r, j));
    float4 XP = lrow(f.x, f, r, j);
    if (r >= 0 && r < f.H && j >= 0 && j < f.W) {
      const float2 e = *reinterpret_cast<const float2*>(xc + (size_t)(r >> 1) * c.ld + (j >> 1));
      XP = make_float4(XP.x + kCCF * e.x, XP.y + kCCF * e.x, XP.z + kCCF * e.y, XP.w + kCCF * e.y);
      if (j + 1 >= f.W) XP.y = 0.f;
      if (j + 2 >= f.W) XP.z = 0.f;
      if (j + 3 >= f.W) XP.w = 0.f;
    }
    sts4(sXP, rr, lane, XP);
  }
  __syncthreads();
  // t at rows r0-1 .. r1 (0 outside the grid)
  for (int rr = 1 + warp; rr <= nrow - 2; rr += kTileWarps) {
    const int r = r0 - 2 + rr;
    float4 T = z;
    if (r >= 0 && r < f.H) {
      const float4 xp = lds4(sXP, rr, lane);
      T = jac4(xp, lds4(sD, rr, lane), lds4(sB, rr, lane),
               arow(lds4(sXP, rr - 1, lane), xp, lds4(sXP, rr + 1, lane), lds4(sU, rr, lane), lds4(sV, rr, lane),
                    lds4(sV, rr - 1, lane), lane));
    }
    sts4(sT, rr, lane, T);
  }
  __syncthreads();
  // s at rows r0 .. r1-1
  double rs = 0.0, rr2 = 0.0;
  DF rs32;
#pragma unroll
  for (int k = 0; k < kOut; ++k) {
    const int r = r0 + warp + kTileWarps * k;
    if (r >= r1) continue;
    const int rr = r - r0 + 2;
    const float4 tc = lds4(sT, rr, lane), B = lds4(sB, rr, lane);
    const float4 v = jac4(tc, lds4(sD, rr, lane), B,
                          arow(lds4(sT, rr - 1, lane), tc, lds4(sT, rr + 1, lane), lds4(sU, rr, lane),
                               lds4(sV, rr, lane), lds4(sV, rr - 1, lane), lane));
    if (!out) continue;
    const size_t o = (size_t)r * f.ld + j;
    if (MODE == kUpCoarse) {
      *reinterpret_cast<float4*>(f.t + o) = v;
    } else if (MODE == kUp32) {
      const float4 sv = make_float4(mk[k].x ? 0.f : v.x, mk[k].y ? 0.f : v.y, mk[k].z ? 0.f : v.z,
                                    mk[k].w ? 0.f : v.w);
      *reinterpret_cast<float4*>(s32 + o) = sv;
      if (pa) {
        // r is the cycle's right-hand side (zero beyond column W - 1, as is s there);
        // r^T r comes per tile from the kernels that wrote r
        rs32.add_prod(B.x, sv.x);
        rs32.add_prod(B.y, sv.y);
        rs32.add_prod(B.z, sv.z);
        rs32.add_prod(B.w, sv.w);
      }
    } else {
      // FP64 s, 0 on masked pixels and nothing beyond column W - 1
      const double sv[4] = {mk[k].x ? 0.0 : (double)v.x, mk[k].y ? 0.0 : (double)v.y,
                            mk[k].z ? 0.0 : (double)v.z, mk[k].w ? 0.0 : (double)v.w};
      if (j + 4 <= f.W) {
        *reinterpret_cast<double2*>(s + o) = make_double2(sv[0], sv[1]);
        *reinterpret_cast<double2*>(s + o + 2) = make_double2(sv[2], sv[3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (j + q < f.W) s[o + q] = sv[q];
      }
      if (pa && rv) {
        const double rk[4] = {ra[k].x, ra[k].y, rb[k].x, rb[k].y};
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (j + q < f.W) {
            rs = fma(rk[q], sv[q], rs);
            rr2 = fma(rk[q], rk[q], rr2);
          }
      }
    }
  }
  if (MAP && pa) {
    if (MODE == kUp32) rs = rs32.value();
    // block sums in warp order, then the arrival of the block as one unit
    rs = warp_sum(rs);
    rr2 = warp_sum(rr2);
    if (lane == 0) {
      red[0][warp] = rs;
      red[1][warp] = rr2;
    }
    __syncthreads();
    if (warp == 0) {
      const PcgArgs a = *pa;
      const double v0 = lane < kTileWarps ? red[0][lane] : 0.0, v1 = lane < kTileWarps ? red[1][lane] : 0.0;
      warp_arrive_fcg(a, a.maps[0], a.st, (int)blockIdx.x, (int)gridDim.x, v0, v1, lane, ph, MODE == kUp32);
    }
  }
}

// ---------------------------------------------------------------- row walkers (wide grids)
// On grids wide and tall enough to give every SM a full wave of warps, the same two
// fused steps run as row walkers: a warp owns one 128-column window (as in a tile)
// and a band of rows, and walks down the band keeping the last rows of every
// quantity in registers, the next row's loads issued one row ahead.  There the
// walkers keep more bytes in flight than shared-memory tiles, whose 61 KB per
// block leave little of the SM's L1 for the tile loads (measured at 2048^2:
// map-grid up step 45 us as a walker, 70 us as tiles; the 512^2 and smaller grids
// go the other way, 4.6-7.3 us as tiles against 8-9 us).
__device__ __forceinline__ bool walk_warp(int W, int bands, int& seg, int& band, int& j, int& lane) {
  const int nseg = (W + kSegOut - 1) / kSegOut;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  lane = threadIdx.x & 31;
  if (w >= nseg * bands) return false;
  seg = w % nseg;
  band = w / nseg;
  j = seg * kSegOut - 4 + 4 * lane;
  return true;
}

// The raw loads of one row, issued one row ahead of the arithmetic that uses them
// (a warp's walk is otherwise one memory round trip per row).
// Row loads go through a per-warp ring of kRing slots in shared memory, filled by
// cp.async kLead rows ahead of the arithmetic: each lane copies its own 16-byte pieces
// (zero-filled outside the grid and beyond column W - 1 by the copy's source size) and
// reads back only what it copied, so no barrier is needed, and the bytes in flight no
// longer cost registers.  wait_group is the hardware's own wait on the lane's copies.
constexpr int kLead = 3;
constexpr int kRing = kLead + 1;   // the slot being read is never the one being filled
constexpr int kWalkWarps = 4;      // 128-thread blocks

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sa), "l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_lead() { asm volatile("cp.async.wait_group %0;" ::"n"(kLead) : "memory"); }

// bytes of the lane's float4 at (r, j) that lie in the grid (0, 4, 8, 12 or 16)
__device__ __forceinline__ int row_bytes(const Grid& f, int r, int j) {
  if (r < 0 || r >= f.H || j < 0 || j >= f.W) return 0;
  const int n = f.W - j;
  return n >= 4 ? 16 : 4 * n;
}

// one slot of the down walker's ring: U, V, D^-1, b of one row (float4 per lane)
struct DownSlot {
  float4 U[32], V[32], D[32], B[32];
};

__device__ __forceinline__ void down_issue(DownSlot& sl, const Grid& f, int r, int j, int lane) {
  const int nb = row_bytes(f, r, j);
  const size_t o = nb ? (size_t)r * f.ld + j : 0;
  cp_async16(&sl.U[lane], f.U + o, nb);
  cp_async16(&sl.V[lane], f.V + o, nb);
  cp_async16(&sl.D[lane], f.Dinv + o, nb);
  cp_async16(&sl.B[lane], f.b + o, nb);
}

// pre-smoothing + residual + restriction for the coarse rows [RB band, RB band + RB)
__global__ void __launch_bounds__(kWalkWarps * 32) k_mg_down_w(Grid f, Grid c, int RB, const MapState* S) {
  if (skip_map(S)) return;
  extern __shared__ float4 wsm4[];
  int seg, band, j, lane;
  if (!walk_warp(f.W, (c.H + RB - 1) / RB, seg, band, j, lane)) return;
  DownSlot* ring = reinterpret_cast<DownSlot*>(wsm4) + (threadIdx.x >> 5) * kRing;
  const bool out = lane >= 1 && lane <= 30 && j < f.W;
  const int I0 = band * RB, I1 = min(c.H, I0 + RB);
  const int r0 = 2 * I0, r1 = min(f.H, 2 * I1);
  const int rb = r0 - 2, re = r1 + 1;  // rows walked
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  // rows r-1, r-2, r-3 of the window (m1, m2, m3)
  float4 Um1 = z, Um2 = z, Vm1 = z, Vm2 = z, Vm3 = z, Dm1 = z, Bm1 = z, Bm2 = z;
  float4 X1m1 = z, X1m2 = z, X2m2 = z, X2m3 = z;
  float lo = 0.f, hi = 0.f;
#pragma unroll
  for (int k = 0; k < kLead; ++k) {
    if (rb + k <= re) down_issue(ring[k], f, rb + k, j, lane);
    cp_commit();
  }
  for (int r = rb; r <= re; ++r) {
    if (r + kLead <= re) down_issue(ring[(r + kLead - rb) % kRing], f, r + kLead, j, lane);
    cp_commit();
    cp_wait_lead();
    const DownSlot& sl = ring[(r - rb) % kRing];
    const float4 U = sl.U[lane], V = sl.V[lane], D = sl.D[lane], B = sl.B[lane];
    const float4 X1 = make_float4(kOmegaF * D.x * B.x, kOmegaF * D.y * B.y, kOmegaF * D.z * B.z, kOmegaF * D.w * B.w);
    // x2 at row q = r - 1
    const int q = r - 1;
    float4 X2 = z;
    if (q >= r0 - 1 && q >= 0 && q < f.H) {
      X2 = jac4(X1m1, Dm1, Bm1, arow(X1m2, X1m1, X1, Um1, Vm1, Vm2, lane));
      if (out && q >= r0 && q < r1) *reinterpret_cast<float4*>(f.x + (size_t)q * f.ld + j) = X2;
    }
    // residual at row p = r - 2, summed over the aggregate's two columns and two rows
    const int p = r - 2;
    if (p >= r0 && p < r1) {
      const float4 a = arow(X2m3, X2m2, X2, Um2, Vm2, Vm3, lane);
      if ((p & 1) == 0) {
        lo = (Bm2.x - a.x) + (Bm2.y - a.y);
        hi = (Bm2.z - a.z) + (Bm2.w - a.w);
      } else {
        lo += (Bm2.x - a.x) + (Bm2.y - a.y);
        hi += (Bm2.z - a.z) + (Bm2.w - a.w);
      }
      if (out && ((p & 1) || p + 1 >= f.H))
        *reinterpret_cast<float2*>(c.b + (size_t)(p >> 1) * c.ld + (j >> 1)) = make_float2(lo, hi);
    }
    Vm3 = Vm2; Vm2 = Vm1; Vm1 = V;
    Um2 = Um1; Um1 = U;
    Dm1 = D;
    Bm2 = Bm1; Bm1 = B;
    X1m2 = X1m1; X1m1 = X1;
    X2m3 = X2m2; X2m2 = X2;
  }
}

// one slot of the up walker's ring: U, V, D^-1, b, x of row r, the coarse x of its
// aggregates, and on the map's grid the mask and FP64 r of row r - 2
struct UpSlot {
  float4 U[32], V[32], D[32], B[32], X[32];
  float2 XC[32];
  uchar4 MK[32];
  double2 RA[32], RB[32];
};

template <int MODE>
__device__ __forceinline__ void up_issue(UpSlot& sl, const Grid& f, const Grid& c, const float* xc,
                                         const uint8_t* mask, const double* rv, int r, int j, int lane) {
  const int nb = row_bytes(f, r, j);
  const size_t o = nb ? (size_t)r * f.ld + j : 0;
  cp_async16(&sl.U[lane], f.U + o, nb);
  cp_async16(&sl.V[lane], f.V + o, nb);
  cp_async16(&sl.D[lane], f.Dinv + o, nb);
  cp_async16(&sl.B[lane], f.b + o, nb);
  cp_async16(&sl.X[lane], f.x + o, nb);
  cp_async8(&sl.XC[lane], nb ? xc + (size_t)(r >> 1) * c.ld + (j >> 1) : xc, nb ? 8 : 0);
  if (MODE != kUpCoarse) {
    const int p = r - 2;
    const int pb = row_bytes(f, p, j);
    const size_t op = pb ? (size_t)p * f.ld + j : 0;
    if (mask) cp_async4(&sl.MK[lane], mask + op, pb ? 4 : 0);
    if (MODE == kUp64 && rv) {
      cp_async16(&sl.RA[lane], rv + op, pb ? 16 : 0);
      cp_async16(&sl.RB[lane], rv + op + (pb ? 2 : 0), pb ? 16 : 0);
    }
  }
}

// prolongation + correction + both post-sweeps for the rows [R band, R band + R); modes
// and outputs as k_mg_up_t (the dot phase's arrival counted per warp).
template <int MODE>
__global__ void __launch_bounds__(kWalkWarps * 32) k_mg_up_w(Grid f, Grid c, const float* __restrict__ xc, int R,
                                                             const uint8_t* mask, double* s,
                                                             const double* __restrict__ rv, float* s32,
                                                             const PcgArgs* pa, const MapState* S, int ph) {
  constexpr bool MAP = MODE != kUpCoarse;
  if (skip_map(S)) return;
  extern __shared__ float4 wsm4[];
  int seg, band, j, lane;
  const int bands = (f.H + R - 1) / R;
  if (!walk_warp(f.W, bands, seg, band, j, lane)) return;
  UpSlot* ring = reinterpret_cast<UpSlot*>(wsm4) + (threadIdx.x >> 5) * kRing;
  const bool out = lane >= 1 && lane <= 30 && j < f.W;
  const int i0 = band * R, i1 = min(f.H, i0 + R);
  const int rb = i0 - 2, re = i1 + 1;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 Um1 = z, Um2 = z, Vm1 = z, Vm2 = z, Vm3 = z, Dm1 = z, Dm2 = z, Bm1 = z, Bm2 = z;
  float4 XPm1 = z, XPm2 = z, Tm2 = z, Tm3 = z;
  double rs = 0.0, rr = 0.0;
  DF rs32;
#pragma unroll
  for (int k = 0; k < kLead; ++k) {
    if (rb + k <= re) up_issue<MODE>(ring[k], f, c, xc, mask, rv, rb + k, j, lane);
    cp_commit();
  }
  for (int r = rb; r <= re; ++r) {
    if (r + kLead <= re) up_issue<MODE>(ring[(r + kLead - rb) % kRing], f, c, xc, mask, rv, r + kLead, j, lane);
    cp_commit();
    cp_wait_lead();
    const UpSlot& sl = ring[(r - rb) % kRing];
    const float4 U = sl.U[lane], V = sl.V[lane], D = sl.D[lane], B = sl.B[lane];
    float4 XP = sl.X[lane];
    if (r >= 0 && r < f.H && j >= 0 && j < f.W) {
      const float2 e = sl.XC[lane];
      XP = make_float4(XP.x + kCCF * e.x, XP.y + kCCF * e.x, XP.z + kCCF * e.y, XP.w + kCCF * e.y);
      if (j + 1 >= f.W) XP.y = 0.f;
      if (j + 2 >= f.W) XP.z = 0.f;
      if (j + 3 >= f.W) XP.w = 0.f;
    }
    // t at row q = r - 1
    const int q = r - 1;
    float4 T = z;
    if (q >= i0 - 1 && q >= 0 && q < f.H) T = jac4(XPm1, Dm1, Bm1, arow(XPm2, XPm1, XP, Um1, Vm1, Vm2, lane));
    // s at row p = r - 2
    const int p = r - 2;
    if (p >= i0 && p < i1) {
      const float4 v = jac4(Tm2, Dm2, Bm2, arow(Tm3, Tm2, T, Um2, Vm2, Vm3, lane));
      const size_t o = (size_t)p * f.ld + j;
      if (MODE == kUpCoarse) {
        if (out) *reinterpret_cast<float4*>(f.t + o) = v;
      } else if (out) {
        const uchar4 mk = mask ? sl.MK[lane] : make_uchar4(0, 0, 0, 0);
        if (MODE == kUp32) {
          const float4 sv = make_float4(mk.x ? 0.f : v.x, mk.y ? 0.f : v.y, mk.z ? 0.f : v.z, mk.w ? 0.f : v.w);
          *reinterpret_cast<float4*>(s32 + o) = sv;
          if (pa) {
            // r is the cycle's right-hand side (zero beyond column W - 1, as is s there);
            // r^T r comes per tile from the kernels that wrote r
            rs32.add_prod(Bm2.x, sv.x);
            rs32.add_prod(Bm2.y, sv.y);
            rs32.add_prod(Bm2.z, sv.z);
            rs32.add_prod(Bm2.w, sv.w);
          }
        } else {
          // the map's grid: FP64 s, 0 on masked pixels and nothing beyond column W - 1
          const double sv[4] = {mk.x ? 0.0 : (double)v.x, mk.y ? 0.0 : (double)v.y, mk.z ? 0.0 : (double)v.z,
                                mk.w ? 0.0 : (double)v.w};
          if (j + 4 <= f.W) {
            *reinterpret_cast<double2*>(s + o) = make_double2(sv[0], sv[1]);
            *reinterpret_cast<double2*>(s + o + 2) = make_double2(sv[2], sv[3]);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (j + k < f.W) s[o + k] = sv[k];
          }
          if (rv) {
            const double2 ra = sl.RA[lane], rb2 = sl.RB[lane];
            const double rk[4] = {ra.x, ra.y, rb2.x, rb2.y};
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (j + k < f.W) {
                rs = fma(rk[k], sv[k], rs);
                rr = fma(rk[k], rk[k], rr);
              }
          }
        }
      }
    }
    Vm3 = Vm2; Vm2 = Vm1; Vm1 = V;
    Um2 = Um1; Um1 = U;
    Dm2 = Dm1; Dm1 = D;
    Bm2 = Bm1; Bm1 = B;
    XPm2 = XPm1; XPm1 = XP;
    Tm3 = Tm2; Tm2 = T;
  }
  if (MAP && pa) {
    const PcgArgs a = *pa;
    const int nseg = (f.W + kSegOut - 1) / kSegOut;
    if (MODE == kUp32) rs = rs32.value();
    warp_arrive_fcg(a, a.maps[0], a.st, band * nseg + seg, nseg * bands, rs, rr, lane, ph, MODE == kUp32);
  }
}

constexpr size_t kDownRingSmem = (size_t)kWalkWarps * kRing * sizeof(DownSlot);
constexpr size_t kUpRingSmem = (size_t)kWalkWarps * kRing * sizeof(UpSlot);

// level 0 without the fused kernels (grids narrower than 64 columns): the FP64 s rounded to FP32
__global__ void k_mg_to32(const double* __restrict__ s, float* s32, Grid g, const MapState* S) {
  if (skip_map(S)) return;
  MG_LOOP(t, (long long)g.H * g.W) {
    const size_t o = (size_t)(t / g.W) * g.ld + (t % g.W);
    s32[o] = (float)s[o];
  }
}

// The grids from index lt down (each at most kTailMax unknowns, together at
// most kTailPx) in one block, in shared memory: U, V, D^-1 copied in, the
// right-hand side of grid lt read from global memory, the whole rest of the
// cycle (down, coarsest sweeps, up) with block barriers between the steps, x of
// grid lt written back.  Same arithmetic as the per-grid kernels.
constexpr int kTailMax = 4096;
constexpr int kTailPx = 5600;
constexpr int kTailThreads = 1024;

struct TailGrids {
  int n;                  // grids in the tail
  Grid g[12];             // their global-memory descriptors (U, V, Dinv filled by mg_setup)
  int off[12];            // element offset of each grid inside the shared arrays
};

__device__ __forceinline__ float tail_ax(const float* U, const float* V, int H, int W, int i, int j,
                                         const float* x) {
  const int o = i * W + j;
  float acc = 0.f;
  float d = U[o] + V[o];
  if (j + 1 < W) acc -= U[o] * x[o + 1];
  if (j > 0) {
    d += U[o - 1];
    acc -= U[o - 1] * x[o - 1];
  }
  if (i + 1 < H) acc -= V[o] * x[o + W];
  if (i > 0) {
    d += V[o - W];
    acc -= V[o - W] * x[o - W];
  }
  return d * x[o] + acc;
}

// Shared-memory grids of the tail: grid l at offset off[l] of each array, row-major H x W.
struct TailSmem {
  float *U, *V, *D, *x, *b, *t;
};

// f(i, j) over grid (H, W).  WARPS = 32: the whole block, rows by warp and columns
// by lane (no per-element index division).  WARPS = 8: the first 256 threads, one
// unknown per thread (grids of at most kTailWarpPx unknowns), synchronised by a
// named barrier so the other warps never wait on these steps.
constexpr int kTailSmallThreads = 256;
template <int WARPS, class F>
__device__ __forceinline__ void tail_for(int H, int W, int warp, int lane, const F& f) {
  if (WARPS == kTailThreads / 32) {
    for (int i = warp; i < H; i += WARPS)
      for (int j = lane; j < W; j += 32) f(i, j);
  } else {
    const int k = warp * 32 + lane;
    if (k < H * W) {
      const int i = k / W;
      f(i, k - i * W);
    }
  }
}

template <int WARPS>
__device__ __forceinline__ void tail_sync() {
  if (WARPS == kTailThreads / 32) __syncthreads();
  else asm volatile("bar.sync 1, %0;" ::"n"(kTailSmallThreads) : "memory");
}

// Down-step of tail grid l (pre-sweeps, residual, restriction into grid l+1).
template <int WARPS>
__device__ __forceinline__ void tail_down(const TailGrids& tg, const TailSmem& sm, int l, int warp, int lane) {
  const int H = tg.g[l].H, W = tg.g[l].W, o0 = tg.off[l];
  const float* U = sm.U + o0;
  const float* V = sm.V + o0;
  const float* D = sm.D + o0;
  float* x = sm.x + o0;
  float* b = sm.b + o0;
  float* t = sm.t + o0;
  tail_for<WARPS>(H, W, warp, lane, [&](int i, int j) { t[i * W + j] = kOmegaF * D[i * W + j] * b[i * W + j]; });
  tail_sync<WARPS>();
  tail_for<WARPS>(H, W, warp, lane, [&](int i, int j) {
    const int k = i * W + j;
    x[k] = t[k] + kOmegaF * D[k] * (b[k] - tail_ax(U, V, H, W, i, j, t));
  });
  tail_sync<WARPS>();
  const int Hc = tg.g[l + 1].H, Wc = tg.g[l + 1].W;
  float* bc = sm.b + tg.off[l + 1];
  tail_for<WARPS>(Hc, Wc, warp, lane, [&](int I, int J) {
    float acc = 0.f;
    for (int i = 2 * I; i <= 2 * I + 1 && i < H; ++i)
      for (int j = 2 * J; j <= 2 * J + 1 && j < W; ++j) acc += b[i * W + j] - tail_ax(U, V, H, W, i, j, x);
    bc[I * Wc + J] = acc;
  });
  tail_sync<WARPS>();
}

// Up-step of tail grid l (correction from grid l+1, two post-sweeps).
template <int WARPS>
__device__ __forceinline__ void tail_up(const TailGrids& tg, const TailSmem& sm, int l, int warp, int lane) {
  const int H = tg.g[l].H, W = tg.g[l].W, o0 = tg.off[l];
  const float* U = sm.U + o0;
  const float* V = sm.V + o0;
  const float* D = sm.D + o0;
  float* x = sm.x + o0;
  float* b = sm.b + o0;
  float* t = sm.t + o0;
  const int Wc = tg.g[l + 1].W;
  const float* xc = sm.x + tg.off[l + 1];
  tail_for<WARPS>(H, W, warp, lane, [&](int i, int j) { x[i * W + j] += kCCF * xc[(i >> 1) * Wc + (j >> 1)]; });
  tail_sync<WARPS>();
  tail_for<WARPS>(H, W, warp, lane, [&](int i, int j) {
    const int k = i * W + j;
    t[k] = x[k] + kOmegaF * D[k] * (b[k] - tail_ax(U, V, H, W, i, j, x));
  });
  tail_sync<WARPS>();
  tail_for<WARPS>(H, W, warp, lane, [&](int i, int j) {
    const int k = i * W + j;
    x[k] = t[k] + kOmegaF * D[k] * (b[k] - tail_ax(U, V, H, W, i, j, t));
  });
  tail_sync<WARPS>();
}

// Coarsest tail grid: thirty sweeps from zero, result in x.  The grid has at most
// kCoarseMax <= 32 unknowns, so warp 0 holds one unknown per lane in a register and
// takes its four neighbours by shuffle: thirty sweeps without a barrier or a
// shared-memory round trip between them, the same terms in the same order as tail_ax.
static_assert(kCoarseMax <= 32, "the coarsest grid fits one warp");
template <int WARPS>
__device__ __forceinline__ void tail_coarsest(const TailGrids& tg, const TailSmem& sm, int l, int warp, int lane) {
  const int H = tg.g[l].H, W = tg.g[l].W, o0 = tg.off[l];
  if (warp == 0) {
    const bool in = lane < H * W;
    const int k = in ? lane : 0;  // lanes past the grid mirror unknown 0 and store nothing
    const int i = k / W, j = k - i * W;
    const bool hx = j + 1 < W, hw = j > 0, hs = i + 1 < H, hn = i > 0;
    const float u = sm.U[o0 + k], v = sm.V[o0 + k];
    const float uw = hw ? sm.U[o0 + k - 1] : 0.f, vn = hn ? sm.V[o0 + k - W] : 0.f;
    float d = u + v;
    if (hw) d += uw;
    if (hn) d += vn;
    const float dk = sm.D[o0 + k], bk = sm.b[o0 + k];
    const int le = hx ? k + 1 : k, lw = hw ? k - 1 : k, ls = hs ? k + W : k, ln = hn ? k - W : k;
    float x = 0.f;
    for (int s = 0; s < kCoarseSweeps; ++s) {
      const float xe = __shfl_sync(kFull, x, le);
      const float xw = __shfl_sync(kFull, x, lw);
      const float xs = __shfl_sync(kFull, x, ls);
      const float xn = __shfl_sync(kFull, x, ln);
      float acc = 0.f;
      if (hx) acc -= u * xe;
      if (hw) acc -= uw * xw;
      if (hs) acc -= v * xs;
      if (hn) acc -= vn * xn;
      const float ax = d * x + acc;
      x = x + kOmegaF * dk * (bk - ax);
    }
    if (in) sm.x[o0 + k] = x;
  }
  tail_sync<WARPS>();
}

// Grids of at most this many unknowns run on the first kTailSmallThreads threads.
constexpr int kTailWarpPx = kTailSmallThreads;

__global__ void __launch_bounds__(kTailThreads) k_mg_tail(TailGrids tg, const MapState* S) {
  if (skip_map(S)) return;
  extern __shared__ float smem[];
  const int tot = tg.off[tg.n - 1] + tg.g[tg.n - 1].H * tg.g[tg.n - 1].W;
  TailSmem sm;
  sm.U = smem;
  sm.V = sm.U + tot;
  sm.D = sm.V + tot;
  sm.x = sm.D + tot;
  sm.b = sm.x + tot;
  sm.t = sm.b + tot;
  // load weights of every tail grid and the right-hand side of the first, all loads of
  // a thread in flight together (the shared arrays are contiguous over the grids)
  {
    constexpr int kq = (kTailPx + kTailThreads - 1) / kTailThreads;
    float ru[kq], rv[kq], rd[kq], rb[kq];
#pragma unroll
    for (int q = 0; q < kq; ++q) {
      const int k = threadIdx.x + kTailThreads * q;
      ru[q] = rv[q] = rd[q] = rb[q] = 0.f;
      if (k < tot) {
        int l = 0;
        while (l + 1 < tg.n && k >= tg.off[l + 1]) ++l;
        const Grid& g = tg.g[l];
        const int e = k - tg.off[l];
        const size_t o = (size_t)(e / g.W) * g.ld + e % g.W;
        ru[q] = g.U[o];
        rv[q] = g.V[o];
        rd[q] = g.Dinv[o];
        if (l == 0) rb[q] = g.b[o];
      }
    }
#pragma unroll
    for (int q = 0; q < kq; ++q) {
      const int k = threadIdx.x + kTailThreads * q;
      if (k < tot) {
        sm.U[k] = ru[q];
        sm.V[k] = rv[q];
        sm.D[k] = rd[q];
        if (k < tg.g[0].H * tg.g[0].W) sm.b[k] = rb[q];
      }
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = tg.n;
  // leading grids of more than kTailWarpPx unknowns: the whole block; the rest (always
  // including the coarsest, at most 16 unknowns): the first 8 warps, one unknown each
  constexpr int kSmallWarps = kTailSmallThreads / 32;
  int nb = 0;
  while (nb < L && tg.g[nb].H * tg.g[nb].W > kTailWarpPx) ++nb;
  for (int l = 0; l < nb && l + 1 < L; ++l) tail_down<kTailThreads / 32>(tg, sm, l, warp, lane);
  if (warp < kSmallWarps) {
    for (int l = nb; l + 1 < L; ++l) tail_down<kSmallWarps>(tg, sm, l, warp, lane);
    tail_coarsest<kSmallWarps>(tg, sm, L - 1, warp, lane);
    for (int l = L - 2; l >= nb; --l) tail_up<kSmallWarps>(tg, sm, l, warp, lane);
  }
  __syncthreads();
  for (int l = (nb < L - 1 ? nb : L - 1) - 1; l >= 0; --l) tail_up<kTailThreads / 32>(tg, sm, l, warp, lane);
  const Grid& g0 = tg.g[0];
  tail_for<kTailThreads / 32>(g0.H, g0.W, warp, lane,
                              [&](int i, int j) { g0.x[(size_t)i * g0.ld + j] = sm.x[i * g0.W + j]; });
}

}  // namespace mg

using namespace mg;

struct MgPlan {
  std::vector<Grid> g;   // FP32 grids; g[0] has the map's size and pitch
  // per grid: kind of the fused kernels (kPerStep, kWalk, kTile) and their rows (walker:
  // coarse rows per band down, rows per band up; tile: rows per tile down (even) and up)
  std::vector<int> kind, rows_down, rows_up;
  int dots_units = 0;    // warps (walker) or blocks (tile) of the map grid's up kernel when it
                         // also does the dot phase (0: it does not)
  int lt = -1;           // first grid handled by the shared-memory tail kernel (-1: none)
  TailGrids tail{};
  size_t tail_smem = 0;
  const double *U0, *V0, *Dinv0, *r0;  // the map's FP64 planes
  double* s0;
  void* mem = nullptr;
  int nsm = 1;
};

static size_t fbytes(size_t elems) { return (elems * 4 + 255) & ~(size_t)255; }

size_t mg_bytes(int H, int W) {
  const int pitch = (W + 63) / 64 * 64;
  size_t bytes = 2 * fbytes((size_t)H * pitch);  // x, t of the map's grid (U, V, D^-1, b are the map's FP32 planes)
  int h = H, w = W;
  while ((long long)h * w > kCoarseMax) {
    h = (h + 1) / 2;
    w = (w + 1) / 2;
    bytes += 6 * fbytes((size_t)h * ((w + 3) / 4 * 4));
  }
  return bytes + 256;
}

constexpr int kVecMinW = 64;  // grids at least this wide use the fused kernels
enum { kPerStep = 0, kWalk = 1, kTile = 2 };

// Rows per walker band: at least rmin, and no more warps than target.
static int walk_rows(int rows, int W, int rmin, long long target) {
  const long long nseg = (W + kSegOut - 1) / kSegOut;
  int R = rmin;
  while (nseg * ((rows + R - 1) / R) > target) ++R;
  return R;
}

static unsigned walk_blocks(const Grid& f, int rows, int R) {
  const long long warps = (long long)((f.W + kSegOut - 1) / kSegOut) * ((rows + R - 1) / R);
  return (unsigned)((warps + kWalkWarps - 1) / kWalkWarps);
}

// Rows per tile: the most (up to kTileMaxRows) that still give every SM two blocks,
// 2 at least; even for the down kernel, whose coarse rows must not straddle tiles.
static int tile_rows(int H, int W, int nsm, bool even) {
  const long long nseg = (W + kSegOut - 1) / kSegOut;
  int TR = kTileMaxRows;
  while (TR > 2 && nseg * ((H + TR - 1) / TR) < 2LL * nsm) TR -= even ? 2 : 1;
  return TR;
}

static unsigned tile_blocks(const Grid& f, int TR) {
  return (unsigned)(((f.W + kSegOut - 1) / kSegOut) * ((f.H + TR - 1) / TR));
}

MgPlan* mg_create(const MapDesc& M, void* mem, int nsm, int ntiles) {
  MgPlan* p = new MgPlan();
  p->mem = mem;
  p->nsm = nsm;
  p->U0 = M.f.U;
  p->V0 = M.f.V;
  p->Dinv0 = M.f.Dinv;
  p->r0 = M.f.r;
  p->s0 = M.f.s;
  char* q = static_cast<char*>(mem);
  auto take = [&](size_t elems) {
    float* r = reinterpret_cast<float*>(q);
    q += fbytes(elems);
    return r;
  };
  Grid g0{};
  g0.H = M.H;
  g0.W = M.W;
  g0.ld = M.pitch;
  const size_t n0 = (size_t)M.H * M.pitch;
  // the map's grid uses the map's FP32 planes for its weights, D^-1 and right-hand side
  // (the FP32 residual of the mixed flexible CG is the cycle's input as it stands)
  g0.U = M.h.U;
  g0.V = M.h.V;
  g0.Dinv = M.h.Dinv;
  g0.b = M.h.r;
  g0.x = take(n0);
  g0.t = take(n0);
  p->g.push_back(g0);
  while ((long long)p->g.back().H * p->g.back().W > kCoarseMax) {
    const Grid& f = p->g.back();
    Grid c{};
    c.H = (f.H + 1) / 2;
    c.W = (f.W + 1) / 2;
    c.ld = (c.W + 3) / 4 * 4;
    const size_t n = (size_t)c.H * c.ld;
    c.U = take(n);
    c.V = take(n);
    c.Dinv = take(n);
    c.x = take(n);
    c.b = take(n);
    c.t = take(n);
    p->g.push_back(c);
  }
  // fused kernels (walkers or tiles) on every grid at least kVecMinW wide; the map grid's
  // up kernel carries the dot phase if its warps or blocks fit the plan's per-tile partial
  // arrays
  // dynamic shared memory above 48 KB is an attribute of the function on the current
  // device: set on every plan creation (the plan's device is current here)
  {
    cudaFuncSetAttribute(k_mg_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(6 * kTailPx * sizeof(float)));
    cudaFuncSetAttribute(k_mg_down_t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    cudaFuncSetAttribute(k_mg_up_t<kUpCoarse>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    cudaFuncSetAttribute(k_mg_up_t<kUp64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    cudaFuncSetAttribute(k_mg_up_t<kUp32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    cudaFuncSetAttribute(k_mg_down_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDownRingSmem);
    cudaFuncSetAttribute(k_mg_up_w<kUpCoarse>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpRingSmem);
    cudaFuncSetAttribute(k_mg_up_w<kUp64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpRingSmem);
    cudaFuncSetAttribute(k_mg_up_w<kUp32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpRingSmem);
  }
  // one resident wave of each walker (the ring's shared memory limits the up walker to
  // three blocks per SM): more warps than that run as a second, mostly idle wave
  int occ_down = 0, occ_up = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_down, k_mg_down_w, kWalkWarps * 32, kDownRingSmem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_up, k_mg_up_w<kUp32>, kWalkWarps * 32, kUpRingSmem);
  const long long wave_down = (long long)(occ_down > 0 ? occ_down : 1) * kWalkWarps * nsm;
  const long long wave_up = (long long)(occ_up > 0 ? occ_up : 1) * kWalkWarps * nsm;
  // walkers where even two-row bands fill a wave, tiles on the smaller grids (see the
  // walker section for the measurements)
  const long long wave = wave_up < wave_down ? wave_up : wave_down;
  for (size_t l = 0; l < p->g.size(); ++l) {
    const Grid& f = p->g[l];
    const long long nseg = (f.W + kSegOut - 1) / kSegOut;
    int kind = kPerStep, rd = 0, ru = 0;
    if (l + 1 < p->g.size() && f.W >= kVecMinW) {
      if (nseg * ((f.H + 1) / 2) >= wave) {
        kind = kWalk;
        rd = walk_rows(p->g[l + 1].H, f.W, 1, wave_down);
        ru = walk_rows(f.H, f.W, 2, l == 0 ? (wave_up < ntiles ? wave_up : ntiles) : wave_up);
      } else {
        kind = kTile;
        rd = tile_rows(f.H, f.W, nsm, true);
        ru = tile_rows(f.H, f.W, nsm, false);
      }
    }
    p->kind.push_back(kind);
    p->rows_down.push_back(rd);
    p->rows_up.push_back(ru);
  }
  if (p->kind[0] != kPerStep) {
    const long long n = p->kind[0] == kWalk
                            ? (long long)((M.W + kSegOut - 1) / kSegOut) * ((M.H + p->rows_up[0] - 1) / p->rows_up[0])
                            : (long long)tile_blocks(p->g[0], p->rows_up[0]);
    if (n >= kArriveGroups && n <= ntiles) p->dots_units = (int)n;
  }

  // the tail: the smallest suffix of grids, from the first with at most kTailMax unknowns,
  // if it fits the shared-memory budget and there is a grid before it
  const int L = (int)p->g.size();
  for (int l = 1; l < L; ++l) {
    if ((long long)p->g[l].H * p->g[l].W > kTailMax) continue;
    int tot = 0;
    for (int k = l; k < L; ++k) tot += p->g[k].H * p->g[k].W;
    if (tot <= kTailPx && L - l <= 12) {
      p->lt = l;
      p->tail.n = L - l;
      int off = 0;
      for (int k = l; k < L; ++k) {
        p->tail.g[k - l] = p->g[k];
        p->tail.off[k - l] = off;
        off += p->g[k].H * p->g[k].W;
      }
      p->tail_smem = (size_t)6 * off * sizeof(float);
    }
    break;
  }
  return p;
}

void mg_destroy(MgPlan* p) { delete p; }

bool mg_fuses_dots(const MgPlan& p) { return p.dots_units > 0; }

static unsigned row_blocks(const Grid& f, int rows) {
  const long long warps = (long long)rows * ((f.W + 127) / 128);
  return (unsigned)((warps + 7) / 8);
}

static int mg_blocks(const MgPlan& p, long long n) {
  const long long b = (n + 255) / 256;
  const long long cap = 8LL * p.nsm;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// FP32 level 0 and the coarse grids for the current weights (once per inner solve).
cudaError_t mg_setup(const MgPlan& p, const MapState* S, cudaStream_t st, bool level0) {
  const Grid& g0 = p.g[0];
  if (level0) k_mg_level0<<<mg_blocks(p, (long long)g0.H * g0.W), 256, 0, st>>>(p.U0, p.V0, p.Dinv0, g0, S);
  // one launch per coarse grid while it has more than kCoarsenSmall unknowns, then one
  // block for all the smaller ones (same arithmetic per aggregate); one block walking a
  // 128^2 grid serialised its memory latency (38 us for the grids of 16384 and fewer)
  constexpr long long kCoarsenSmall = 1024;
  size_t l = 0;
  for (; l + 1 < p.g.size(); ++l) {
    const Grid& c = p.g[l + 1];
    if ((long long)c.H * c.W <= kCoarsenSmall && p.g.size() - l <= 16) break;
    k_mg_coarsen<<<mg_blocks(p, (long long)c.H * c.W), 256, 0, st>>>(p.g[l], c, S);
  }
  if (l + 1 < p.g.size()) {
    CoarsenList cl{};
    cl.n = (int)(p.g.size() - l);
    for (int k = 0; k < cl.n; ++k) cl.g[k] = p.g[l + k];
    k_mg_coarsen_small<<<1, 1024, 0, st>>>(cl, S);
  }
  return cudaGetLastError();
}

// s = V-cycle(r) on the map's planes; mask zeroes s.
float* mg_input(const MgPlan& p) { return p.g[0].b; }

// The up step of grid l; on the map's grid (l = 0) it writes s (FP64, or FP32 into
// s32) and, with dots, carries the flexible CG's dot phase ph.
static void up_level(const MgPlan& p, int l, int stop, const uint8_t* mask, const MapState* S, cudaStream_t st,
                     const PcgArgs* dots, float* s32, int ph) {
  const Grid& f = p.g[l];
  if (p.kind[l] != kPerStep) {
    // the coarse grid's corrected solution: the t plane if a fused kernel made it, else x
    const Grid& c = p.g[l + 1];
    const float* xc = (l + 1 < stop && p.kind[l + 1] != kPerStep) ? c.t : c.x;
    const int R = p.rows_up[l];
    const bool d = l == 0 && dots && p.dots_units > 0;
    const PcgArgs* pa = d ? dots : nullptr;
    const int mode = l > 0 ? kUpCoarse : (s32 ? kUp32 : kUp64);
    const double* rv = (mode == kUp64 && d) ? p.r0 : nullptr;
    double* s64 = mode == kUp64 ? p.s0 : nullptr;
    const uint8_t* mk = l == 0 ? mask : nullptr;
    float* o32 = mode == kUp32 ? s32 : nullptr;
    if (p.kind[l] == kWalk) {
      const unsigned nb = walk_blocks(f, f.H, R);
      const unsigned nt = kWalkWarps * 32;
      if (mode == kUp32) k_mg_up_w<kUp32><<<nb, nt, kUpRingSmem, st>>>(f, c, xc, R, mk, s64, rv, o32, pa, S, ph);
      else if (mode == kUp64) k_mg_up_w<kUp64><<<nb, nt, kUpRingSmem, st>>>(f, c, xc, R, mk, s64, rv, o32, pa, S, ph);
      else k_mg_up_w<kUpCoarse><<<nb, nt, kUpRingSmem, st>>>(f, c, xc, R, mk, s64, rv, o32, pa, S, ph);
    } else {
      const unsigned nb = tile_blocks(f, R);
      if (mode == kUp32) k_mg_up_t<kUp32><<<nb, kTileThreads, kTileSmem, st>>>(f, c, xc, R, mk, s64, rv, o32, pa, S, ph);
      else if (mode == kUp64) k_mg_up_t<kUp64><<<nb, kTileThreads, kTileSmem, st>>>(f, c, xc, R, mk, s64, rv, o32, pa, S, ph);
      else k_mg_up_t<kUpCoarse><<<nb, kTileThreads, kTileSmem, st>>>(f, c, xc, R, mk, s64, rv, o32, pa, S, ph);
    }
    return;
  }
  if (f.W >= kVecMinW) {
    k_mg_sweep_v<kSrcXP><<<row_blocks(f, f.H), 256, 0, st>>>(f, p.g[l + 1], f.t, nullptr, nullptr, S);
    k_mg_sweep_v<kSrcT><<<row_blocks(f, f.H), 256, 0, st>>>(f, Grid{}, f.x, l == 0 ? mask : nullptr,
                                                             l == 0 ? p.s0 : nullptr, S);
  } else {
    k_mg_post1<<<mg_blocks(p, (long long)f.H * f.W), 256, 0, st>>>(f, p.g[l + 1], S);
    k_mg_post2<<<mg_blocks(p, (long long)f.H * f.W), 256, 0, st>>>(f, l == 0 ? mask : nullptr,
                                                                  l == 0 ? p.s0 : nullptr, S);
  }
  // the map's grid without fused kernels: the FP64 s rounded into s32
  if (l == 0 && s32) k_mg_to32<<<mg_blocks(p, (long long)f.H * f.W), 256, 0, st>>>(p.s0, s32, f, S);
}

cudaError_t mg_apply(const MgPlan& p, const uint8_t* mask, const MapState* S, cudaStream_t st, bool packed,
                     const PcgArgs* dots, float* s32, bool dots_init, int part) {
  const int ph = dots_init ? kPhResInit : kPhFcg;
  const int L = (int)p.g.size();
  const Grid& g0 = p.g[0];
  const int stop = p.lt > 0 ? p.lt : L - 1;  // grids [0, stop) by per-grid kernels
  if (part == 2) {
    // the map grid's last step alone
    if (L == 1) {
      k_mg_post2<<<mg_blocks(p, (long long)g0.H * g0.W), 256, 0, st>>>(g0, mask, p.s0, S);
      if (s32) k_mg_to32<<<mg_blocks(p, (long long)g0.H * g0.W), 256, 0, st>>>(p.s0, s32, g0, S);
    } else {
      up_level(p, 0, stop, mask, S, st, dots, s32, ph);
    }
    return cudaGetLastError();
  }
  if (!packed) k_mg_rhs_v<<<mg_blocks(p, (long long)g0.H * ((g0.W + 3) / 4)), 256, 0, st>>>(p.r0, g0, S);
  if (L == 1) {
    k_mg_coarsest<<<1, 256, 0, st>>>(g0, S);
    if (part == 0) {
      k_mg_post2<<<mg_blocks(p, (long long)g0.H * g0.W), 256, 0, st>>>(g0, mask, p.s0, S);
      if (s32) k_mg_to32<<<mg_blocks(p, (long long)g0.H * g0.W), 256, 0, st>>>(p.s0, s32, g0, S);
    }
    return cudaGetLastError();
  }
  for (int l = 0; l < stop; ++l) {
    const Grid& f = p.g[l];
    if (p.kind[l] == kWalk) {
      const Grid& c = p.g[l + 1];
      k_mg_down_w<<<walk_blocks(f, c.H, p.rows_down[l]), kWalkWarps * 32, kDownRingSmem, st>>>(f, c, p.rows_down[l], S);
    } else if (p.kind[l] == kTile) {
      const Grid& c = p.g[l + 1];
      k_mg_down_t<<<tile_blocks(f, p.rows_down[l]), kTileThreads, kTileSmem, st>>>(f, c, p.rows_down[l], S);
    } else if (f.W >= kVecMinW) {
      k_mg_sweep_v<kSrcX1><<<row_blocks(f, f.H), 256, 0, st>>>(f, Grid{}, f.x, nullptr, nullptr, S);
      k_mg_res_v<<<row_blocks(f, p.g[l + 1].H), 256, 0, st>>>(f, p.g[l + 1], S);
    } else {
      k_mg_pre<<<mg_blocks(p, (long long)f.H * f.W), 256, 0, st>>>(f, S);
      k_mg_res<<<mg_blocks(p, (long long)p.g[l + 1].H * p.g[l + 1].W), 256, 0, st>>>(f, p.g[l + 1], S);
    }
  }
  if (p.lt > 0) {
    k_mg_tail<<<1, kTailThreads, p.tail_smem, st>>>(p.tail, S);
  } else {
    k_mg_coarsest<<<1, 256, 0, st>>>(p.g[L - 1], S);
  }
  for (int l = stop - 1; l >= (part == 1 ? 1 : 0); --l) up_level(p, l, stop, mask, S, st, dots, s32, ph);
  return cudaGetLastError();
}

int mg_levels(const MgPlan& p) { return (int)p.g.size(); }

}  // namespace ulp
