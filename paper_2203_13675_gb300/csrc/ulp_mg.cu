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

__global__ void __launch_bounds__(kTailThreads) k_mg_tail(TailGrids tg, const MapState* S) {
  if (skip_map(S)) return;
  extern __shared__ float sm[];
  const int tot = tg.off[tg.n - 1] + tg.g[tg.n - 1].H * tg.g[tg.n - 1].W;
  float* sU = sm;
  float* sV = sU + tot;
  float* sD = sV + tot;
  float* sx = sD + tot;
  float* sb = sx + tot;
  float* st = sb + tot;
  // load weights of every tail grid and the right-hand side of the first
  for (int l = 0; l < tg.n; ++l) {
    const Grid& g = tg.g[l];
    const int n = g.H * g.W;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const size_t o = (size_t)(k / g.W) * g.ld + k % g.W;
      sU[tg.off[l] + k] = g.U[o];
      sV[tg.off[l] + k] = g.V[o];
      sD[tg.off[l] + k] = g.Dinv[o];
      if (l == 0) sb[k] = g.b[o];
    }
  }
  __syncthreads();
  // down
  for (int l = 0; l + 1 < tg.n; ++l) {
    const int H = tg.g[l].H, W = tg.g[l].W, n = H * W, o0 = tg.off[l];
    const float* U = sU + o0;
    const float* V = sV + o0;
    const float* D = sD + o0;
    float* x = sx + o0;
    float* b = sb + o0;
    float* t = st + o0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) t[k] = kOmegaF * D[k] * b[k];  // first sweep
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x)
      x[k] = t[k] + kOmegaF * D[k] * (b[k] - tail_ax(U, V, H, W, k / W, k % W, t));
    __syncthreads();
    const int Hc = tg.g[l + 1].H, Wc = tg.g[l + 1].W;
    float* bc = sb + tg.off[l + 1];
    for (int k = threadIdx.x; k < Hc * Wc; k += blockDim.x) {
      const int I = k / Wc, J = k % Wc;
      float acc = 0.f;
      for (int i = 2 * I; i <= 2 * I + 1 && i < H; ++i)
        for (int j = 2 * J; j <= 2 * J + 1 && j < W; ++j) acc += b[i * W + j] - tail_ax(U, V, H, W, i, j, x);
      bc[k] = acc;
    }
    __syncthreads();
  }
  // coarsest: sweeps from zero, x and t ping-pong
  {
    const int l = tg.n - 1;
    const int H = tg.g[l].H, W = tg.g[l].W, n = H * W, o0 = tg.off[l];
    const float* U = sU + o0;
    const float* V = sV + o0;
    const float* D = sD + o0;
    float* b = sb + o0;
    float* src = sx + o0;
    float* dst = st + o0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) src[k] = 0.f;
    __syncthreads();
    for (int s = 0; s < kCoarseSweeps; ++s) {
      for (int k = threadIdx.x; k < n; k += blockDim.x)
        dst[k] = src[k] + kOmegaF * D[k] * (b[k] - tail_ax(U, V, H, W, k / W, k % W, src));
      __syncthreads();
      float* tmp = src;
      src = dst;
      dst = tmp;
    }
    if (src != sx + o0) {
      for (int k = threadIdx.x; k < n; k += blockDim.x) sx[o0 + k] = src[k];
      __syncthreads();
    }
  }
  // up
  for (int l = tg.n - 2; l >= 0; --l) {
    const int H = tg.g[l].H, W = tg.g[l].W, n = H * W, o0 = tg.off[l];
    const float* U = sU + o0;
    const float* V = sV + o0;
    const float* D = sD + o0;
    float* x = sx + o0;
    float* b = sb + o0;
    float* t = st + o0;
    const int Wc = tg.g[l + 1].W;
    const float* xc = sx + tg.off[l + 1];
    for (int k = threadIdx.x; k < n; k += blockDim.x) x[k] += kCCF * xc[(k / W >> 1) * Wc + ((k % W) >> 1)];
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x)
      t[k] = x[k] + kOmegaF * D[k] * (b[k] - tail_ax(U, V, H, W, k / W, k % W, x));
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x)
      x[k] = t[k] + kOmegaF * D[k] * (b[k] - tail_ax(U, V, H, W, k / W, k % W, t));
    __syncthreads();
  }
  const Grid& g0 = tg.g[0];
  for (int k = threadIdx.x; k < g0.H * g0.W; k += blockDim.x)
    g0.x[(size_t)(k / g0.W) * g0.ld + k % g0.W] = sx[k];
}

}  // namespace mg

using namespace mg;

struct MgPlan {
  std::vector<Grid> g;   // FP32 grids; g[0] has the map's size and pitch
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
  size_t bytes = 6 * fbytes((size_t)H * pitch);
  int h = H, w = W;
  while ((long long)h * w > kCoarseMax) {
    h = (h + 1) / 2;
    w = (w + 1) / 2;
    bytes += 6 * fbytes((size_t)h * w);
  }
  return bytes + 256;
}

MgPlan* mg_create(const MapDesc& M, void* mem, int nsm) {
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
  g0.U = take(n0);
  g0.V = take(n0);
  g0.Dinv = take(n0);
  g0.x = take(n0);
  g0.b = take(n0);
  g0.t = take(n0);
  p->g.push_back(g0);
  while ((long long)p->g.back().H * p->g.back().W > kCoarseMax) {
    const Grid& f = p->g.back();
    Grid c{};
    c.H = (f.H + 1) / 2;
    c.W = (f.W + 1) / 2;
    c.ld = c.W;
    const size_t n = (size_t)c.H * c.W;
    c.U = take(n);
    c.V = take(n);
    c.Dinv = take(n);
    c.x = take(n);
    c.b = take(n);
    c.t = take(n);
    p->g.push_back(c);
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

static int mg_blocks(const MgPlan& p, long long n) {
  const long long b = (n + 255) / 256;
  const long long cap = 8LL * p.nsm;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// FP32 level 0 and the coarse grids for the current weights (once per inner solve).
cudaError_t mg_setup(const MgPlan& p, const MapState* S, cudaStream_t st) {
  const Grid& g0 = p.g[0];
  k_mg_level0<<<mg_blocks(p, (long long)g0.H * g0.W), 256, 0, st>>>(p.U0, p.V0, p.Dinv0, g0, S);
  for (size_t l = 0; l + 1 < p.g.size(); ++l) {
    const Grid& c = p.g[l + 1];
    k_mg_coarsen<<<mg_blocks(p, (long long)c.H * c.W), 256, 0, st>>>(p.g[l], c, S);
  }
  return cudaGetLastError();
}

// s = V-cycle(r) on the map's planes; mask zeroes s.
cudaError_t mg_apply(const MgPlan& p, const uint8_t* mask, const MapState* S, cudaStream_t st) {
  const int L = (int)p.g.size();
  const Grid& g0 = p.g[0];
  k_mg_rhs<<<mg_blocks(p, (long long)g0.H * g0.W), 256, 0, st>>>(p.r0, g0, S);
  if (L == 1) {
    k_mg_coarsest<<<1, 256, 0, st>>>(g0, S);
    k_mg_post2<<<mg_blocks(p, (long long)g0.H * g0.W), 256, 0, st>>>(g0, mask, p.s0, S);
    return cudaGetLastError();
  }
  const int stop = p.lt > 0 ? p.lt : L - 1;  // grids [0, stop) by per-grid kernels
  for (int l = 0; l < stop; ++l) {
    const Grid& f = p.g[l];
    k_mg_pre<<<mg_blocks(p, (long long)f.H * f.W), 256, 0, st>>>(f, S);
    k_mg_res<<<mg_blocks(p, (long long)p.g[l + 1].H * p.g[l + 1].W), 256, 0, st>>>(f, p.g[l + 1], S);
  }
  if (p.lt > 0) {
    static bool attr = false;
    if (!attr) {
      const cudaError_t e = cudaFuncSetAttribute(k_mg_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(6 * kTailPx * sizeof(float)));
      if (e != cudaSuccess) return e;
      attr = true;
    }
    k_mg_tail<<<1, kTailThreads, p.tail_smem, st>>>(p.tail, S);
  } else {
    k_mg_coarsest<<<1, 256, 0, st>>>(p.g[L - 1], S);
  }
  for (int l = stop - 1; l >= 0; --l) {
    const Grid& f = p.g[l];
    k_mg_post1<<<mg_blocks(p, (long long)f.H * f.W), 256, 0, st>>>(f, p.g[l + 1], S);
    k_mg_post2<<<mg_blocks(p, (long long)f.H * f.W), 256, 0, st>>>(f, l == 0 ? mask : nullptr,
                                                                  l == 0 ? p.s0 : nullptr, S);
  }
  return cudaGetLastError();
}

int mg_levels(const MgPlan& p) { return (int)p.g.size(); }

}  // namespace ulp
