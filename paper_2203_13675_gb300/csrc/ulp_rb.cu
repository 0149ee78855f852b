// ulp_rb.cu -- SSOR(omega) and ILU(0) with the unknowns in red-black order.
//
// The paper's triangular preconditioners (Sec. 2 items 3-5) are defined for an
// ordering it leaves open; in natural row-major order their solves are a
// wavefront across the whole grid.  With red pixels (i + j even) first and
// black ones after, the 5-point stencil couples only opposite colours, and
// each triangular solve becomes one fully parallel pass per colour:
//   SSOR:   black  s_b = c w (r_b + sum_red w_bk y_k) / D_b,  y_k = w r_k / D_k
//           red    s_r = c y_r + (w / D_r) sum_black w_rk s_k
//           (c = (2 - w) / w; D = 0 counts as 1; the red pass uses the scaled
//           black values, which is the same expression)
//   ILU(0): pivots p_red = a_kk, p_black = a_bb - sum_red w_bk^2 / p_k (guarded
//           as in the natural order), once per inner solve;
//           black  s_b = (r_b + sum_red w_bk r_k / p_k) / p_b
//           red    s_r = (r_r + sum_black w_rk s_k) / p_r
// (w_bk the edge weight U or V between the pixels; a_bk = -w_bk.)  IC(0) in
// this order is the same M.  FP64 throughout, as the natural-order sweeps.
#include "ulp_host.h"

namespace ulp {

namespace rb {

struct RbArgs {
  int H, W, pitch, color;  // pixels of this colour: (i + j) % 2 == color (0 red, 1 black)
  const double *U, *V, *D, *r;
  double* s;
  double* piv;             // ILU: 1 / pivot per pixel
  double omega;
};

#define RB_LOOP(t, n) for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (n); t += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ bool rb_skip(const MapState* S) { return S && *(volatile const int*)&S->done; }

// the k-th pixel of row i with colour c: j = 2k + ((i + c) & 1)
__device__ __forceinline__ bool rb_pixel(const RbArgs& a, long long t, int& i, int& j) {
  const int per = (a.W + 1) / 2;
  i = (int)(t / per);
  j = 2 * (int)(t % per) + ((i + a.color) & 1);
  return j < a.W;
}

// sum over the 4 neighbours of (i, j) of w * f(neighbour offset)
template <class F>
__device__ __forceinline__ double nbr_sum(const RbArgs& a, int i, int j, size_t o, const F& f) {
  double acc = 0.0;
  if (j + 1 < a.W) acc = fma(a.U[o], f(o + 1), acc);
  if (j > 0) acc = fma(a.U[o - 1], f(o - 1), acc);
  if (i + 1 < a.H) acc = fma(a.V[o], f(o + a.pitch), acc);
  if (i > 0) acc = fma(a.V[o - a.pitch], f(o - a.pitch), acc);
  return acc;
}

__device__ __forceinline__ double ssor_diag(double d) { return d > 0.0 ? d : 1.0; }

__global__ void k_rbssor_black(RbArgs a, const MapState* S) {
  if (rb_skip(S)) return;
  const double w = a.omega, c = (2.0 - w) / w;
  RB_LOOP(t, (long long)a.H * ((a.W + 1) / 2)) {
    int i, j;
    if (!rb_pixel(a, t, i, j)) continue;
    const size_t o = (size_t)i * a.pitch + j;
    const double acc = nbr_sum(a, i, j, o, [&](size_t q) { return w * a.r[q] / ssor_diag(a.D[q]); });
    a.s[o] = c * (w * (a.r[o] + acc) / ssor_diag(a.D[o]));
  }
}

__global__ void k_rbssor_red(RbArgs a, const MapState* S) {
  if (rb_skip(S)) return;
  const double w = a.omega, c = (2.0 - w) / w;
  RB_LOOP(t, (long long)a.H * ((a.W + 1) / 2)) {
    int i, j;
    if (!rb_pixel(a, t, i, j)) continue;
    const size_t o = (size_t)i * a.pitch + j;
    const double d = ssor_diag(a.D[o]);
    const double acc = nbr_sum(a, i, j, o, [&](size_t q) { return a.s[q]; });
    a.s[o] = c * (w * a.r[o] / d) + (w / d) * acc;
  }
}

__device__ __forceinline__ double guard_pivot(double p, double akk) {
  return (p > 1e-12 * akk && p > 0.0) ? p : (akk > 0.0 ? akk : 1.0);
}

// pivots: red pixels first (a_kk), black from them (two launches: color 0, then 1)
__global__ void k_rbilu_piv(RbArgs a, const MapState* S) {
  if (rb_skip(S)) return;
  RB_LOOP(t, (long long)a.H * ((a.W + 1) / 2)) {
    int i, j;
    if (!rb_pixel(a, t, i, j)) continue;
    const size_t o = (size_t)i * a.pitch + j;
    const double akk = a.D[o];
    double p = akk;
    if (a.color == 1) {
      auto wsq = [&](double w, size_t q) { return w * w * a.piv[q]; };
      if (j + 1 < a.W) p -= wsq(a.U[o], o + 1);
      if (j > 0) p -= wsq(a.U[o - 1], o - 1);
      if (i + 1 < a.H) p -= wsq(a.V[o], o + a.pitch);
      if (i > 0) p -= wsq(a.V[o - a.pitch], o - a.pitch);
    }
    a.piv[o] = 1.0 / guard_pivot(p, akk);
  }
}

__global__ void k_rbilu_black(RbArgs a, const MapState* S) {
  if (rb_skip(S)) return;
  RB_LOOP(t, (long long)a.H * ((a.W + 1) / 2)) {
    int i, j;
    if (!rb_pixel(a, t, i, j)) continue;
    const size_t o = (size_t)i * a.pitch + j;
    const double acc = nbr_sum(a, i, j, o, [&](size_t q) { return a.piv[q] * a.r[q]; });
    a.s[o] = (a.r[o] + acc) * a.piv[o];
  }
}

__global__ void k_rbilu_red(RbArgs a, const MapState* S) {
  if (rb_skip(S)) return;
  RB_LOOP(t, (long long)a.H * ((a.W + 1) / 2)) {
    int i, j;
    if (!rb_pixel(a, t, i, j)) continue;
    const size_t o = (size_t)i * a.pitch + j;
    const double acc = nbr_sum(a, i, j, o, [&](size_t q) { return a.s[q]; });
    a.s[o] = (a.r[o] + acc) * a.piv[o];
  }
}

}  // namespace rb

using namespace rb;

static RbArgs rb_args(const Plan& pl, int color) {
  const MapDesc& M = pl.hmaps[0];
  RbArgs a{};
  a.H = M.H;
  a.W = M.W;
  a.pitch = M.pitch;
  a.color = color;
  a.U = M.f.U;
  a.V = M.f.V;
  a.D = M.f.D;
  a.r = M.f.r;
  a.s = M.f.s;
  a.piv = M.f.piv;
  a.omega = pl.opt.omega;
  return a;
}

static int rb_blocks(const Plan& pl, const RbArgs& a) {
  const long long n = (long long)a.H * ((a.W + 1) / 2);
  const long long b = (n + 255) / 256, cap = 8LL * pl.nsm;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// ILU(0) pivots for the current weights (once per inner solve); nothing for SSOR
cudaError_t rb_setup(const Plan& pl, int kind, const MapState* S, cudaStream_t st) {
  if (kind == ULP_PRECOND_RBILU) {
    const RbArgs red = rb_args(pl, 0), black = rb_args(pl, 1);
    k_rbilu_piv<<<rb_blocks(pl, red), 256, 0, st>>>(red, S);
    k_rbilu_piv<<<rb_blocks(pl, black), 256, 0, st>>>(black, S);
  }
  return cudaGetLastError();
}

// s = M^-1 r on the map's planes: the black pass, then the red pass
cudaError_t rb_apply(const Plan& pl, int kind, const MapState* S, cudaStream_t st) {
  const RbArgs red = rb_args(pl, 0), black = rb_args(pl, 1);
  if (kind == ULP_PRECOND_RBSSOR) {
    k_rbssor_black<<<rb_blocks(pl, black), 256, 0, st>>>(black, S);
    k_rbssor_red<<<rb_blocks(pl, red), 256, 0, st>>>(red, S);
  } else {
    k_rbilu_black<<<rb_blocks(pl, black), 256, 0, st>>>(black, S);
    k_rbilu_red<<<rb_blocks(pl, red), 256, 0, st>>>(red, S);
  }
  return cudaGetLastError();
}

}  // namespace ulp
