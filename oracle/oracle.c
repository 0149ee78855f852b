/*
 * oracle.c -- plain, slow FP64 CPU oracle of the L^p-norm phase-unwrapping
 * method of arXiv 2203.13675 (Legarda-Saenz, Brito-Loeza, Espinosa-Romero).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load it.  It shares nothing with the CUDA
 * library: no headers, helpers, tables or constants.
 *
 * The method is an iteration (IRLS around PCG) with no faster closed form, so
 * this file takes Algorithm 1's steps in the paper's order and notation:
 *   wrapped differences (Sec. 2.1)  ->  U, V (Eq. UV)  ->  A, b in CSR (Eq. Axb)
 *   ->  M from A (Sec. 2 list of preconditioners)  ->  PCG (Algorithm 1, after
 *   Shewchuk)  ->  outer error (Algorithm 1).
 * Readings of points the paper leaves open are marked READING.
 * Single thread, no blocking, no fusion, sequential sums in natural order.
 * Build with -ffp-contract=off so every operation rounds as written.
 */
#define _POSIX_C_SOURCE 199309L  /* clock_gettime: the set-up time of the preconditioner */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* Wall-clock seconds (monotonic), for the set-up share the paper reports (Sec. 3). */
static double orc_now(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static const double ORC_PI = 3.14159265358979323846;

/* Eq. (wrapped): psi = phi + 2 pi k with -pi < psi <= pi.  W(x) is the
 * representative of x modulo 2 pi in (-pi, pi]; x = +-pi both map to +pi. */
double orc_wrap(double x) {
  double k = ceil((x - ORC_PI) / (2.0 * ORC_PI));
  return x - (2.0 * ORC_PI) * k;
}

/* Sec. 2.1, wrapped differences.  Delta^x acts along j (columns), Delta^y
 * along i (rows), both as forward differences on every edge inside the grid.
 * READING: the paper's last-column/last-row "backward" case only multiplies
 * U_{i,W-1} = 0 and V_{H-1,j} = 0 (zero-flux boundary condition of
 * Eq. ecuacion), so those ghost entries are stored as 0. */
void orc_wrapped_diffs(const double* psi, int H, int W, double* dx, double* dy) {
  for (int i = 0; i < H; ++i) {
    for (int j = 0; j < W; ++j) {
      long k = (long)i * W + j;
      dx[k] = (j + 1 < W) ? orc_wrap(psi[k + 1] - psi[k]) : 0.0;
      dy[k] = (i + 1 < H) ? orc_wrap(psi[k + W] - psi[k]) : 0.0;
    }
  }
}

/* Eq. (UV): U_{i,j} = tau / (|phi_{i,j+1} - phi_{i,j} - Delta^x_{i,j}|^{2-p} + tau),
 * V likewise along i.  READING: an edge leaving the grid, or touching a masked
 * pixel, carries weight 0 (zero flux).  pow(0, 0) = 1, so p = 2 gives
 * tau / (1 + tau) on every edge. */
static double orc_weight(double resid, double p, double tau) {
  return tau / (pow(fabs(resid), 2.0 - p) + tau);
}

void orc_weights(const double* phi, const double* dx, const double* dy,
                 const uint8_t* mask, int H, int W, double p, double tau,
                 double* U, double* V) {
  for (int i = 0; i < H; ++i) {
    for (int j = 0; j < W; ++j) {
      long k = (long)i * W + j;
      int mk = mask ? (mask[k] != 0) : 0;
      if (j + 1 < W && !mk && !(mask && mask[k + 1])) {
        U[k] = orc_weight(phi[k + 1] - phi[k] - dx[k], p, tau);
      } else {
        U[k] = 0.0;
      }
      if (i + 1 < H && !mk && !(mask && mask[k + W])) {
        V[k] = orc_weight(phi[k + W] - phi[k] - dy[k], p, tau);
      } else {
        V[k] = 0.0;
      }
    }
  }
}

/* Eq. (Axb), row k = (i,j):
 *   -(phi_{i,j+1} U_{i,j} + phi_{i+1,j} V_{i,j} + phi_{i,j-1} U_{i,j-1} + phi_{i-1,j} V_{i-1,j})
 *   + (U_{i,j-1} + U_{i,j} + V_{i-1,j} + V_{i,j}) phi_{i,j}
 *   = Delta^x_{i,j-1} U_{i,j-1} - Delta^x_{i,j} U_{i,j} + Delta^y_{i-1,j} V_{i-1,j} - Delta^y_{i,j} V_{i,j}.
 * Terms whose index leaves the grid are absent.  Every structural entry of the
 * 5-point pattern is stored, even when its value is 0, so nnz = 5HW - 2(H+W). */
long orc_assemble(const double* U, const double* V, const double* dx,
                  const double* dy, int H, int W, long* indptr, int* indices,
                  double* data, double* b) {
  long nnz = 0;
  for (int i = 0; i < H; ++i) {
    for (int j = 0; j < W; ++j) {
      long k = (long)i * W + j;
      double uw = (j > 0) ? U[k - 1] : 0.0;     /* U_{i,j-1} */
      double ue = U[k];                         /* U_{i,j}   */
      double vn = (i > 0) ? V[k - W] : 0.0;     /* V_{i-1,j} */
      double vs = V[k];                         /* V_{i,j}   */
      indptr[k] = nnz;
      if (i > 0) { indices[nnz] = (int)(k - W); data[nnz] = -vn; ++nnz; }
      if (j > 0) { indices[nnz] = (int)(k - 1); data[nnz] = -uw; ++nnz; }
      indices[nnz] = (int)k; data[nnz] = uw + ue + vn + vs; ++nnz;
      if (j + 1 < W) { indices[nnz] = (int)(k + 1); data[nnz] = -ue; ++nnz; }
      if (i + 1 < H) { indices[nnz] = (int)(k + W); data[nnz] = -vs; ++nnz; }
      double bk = 0.0;
      if (j > 0) bk += dx[k - 1] * uw;
      bk -= dx[k] * ue;
      if (i > 0) bk += dy[k - W] * vn;
      bk -= dy[k] * vs;
      b[k] = bk;
    }
  }
  indptr[(long)H * W] = nnz;
  return nnz;
}

void orc_csr_matvec(int n, const long* indptr, const int* indices,
                    const double* data, const double* x, double* y) {
  for (int r = 0; r < n; ++r) {
    double acc = 0.0;
    for (long t = indptr[r]; t < indptr[r + 1]; ++t) acc += data[t] * x[indices[t]];
    y[r] = acc;
  }
}

static double orc_dot(long n, const double* a, const double* b) {
  double acc = 0.0;
  for (long t = 0; t < n; ++t) acc += a[t] * b[t];
  return acc;
}

/* ------------------------------------------------------------------------ */
/* Preconditioners (Sec. 2, list items 1-5, plus the Fourier-basis Poisson   */
/* solver of Sec. 1 used as a fixed M).                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int kind, H, W, n;
  const long* indptr;
  const int* indices;
  const double* data;
  double omega;
  const uint8_t* mask;
  double* diag;     /* Jacobi / SSOR: a_kk (guarded) */
  double* fact;     /* ILU(0): unit-L and U in A's pattern; IC(0): L in A's pattern */
  long* dpos;       /* position of the diagonal in each row */
  double* ch;       /* DCT: orthonormal DCT-II matrix, H x H */
  double* cw;       /* DCT: W x W */
  double* lam;      /* DCT: eigenvalues, H x W */
  double* tmp;      /* DCT scratch, H x W */
  double* tmp2;
  int mg_levels;    /* MG: number of grids, level 0 = the fine grid */
  int mg_h[32], mg_w[32];
  double* mg_u[32]; /* MG: edge weights and diagonal per level */
  double* mg_v[32];
  double* mg_d[32];
  double* mg_x[32]; /* MG: work vectors per level (iterate, right-hand side, scratch) */
  double* mg_b[32];
  double* mg_t[32];
} orc_precond;

/* Position of column c in CSR row r, or -1 if (r,c) is not in the pattern. */
static long orc_find(const orc_precond* P, int r, int c) {
  for (long t = P->indptr[r]; t < P->indptr[r + 1]; ++t)
    if (P->indices[t] == c) return t;
  return -1;
}

/* READING (paper silent): a pivot that is not clearly positive (a zero row
 * from masked pixels, or the last node of a chain-shaped component, where
 * the factorisation of a singular block reaches 0) is replaced by the
 * original diagonal a_kk, or by 1 when a_kk = 0.  M stays SPD. */
static double orc_guard_pivot(double piv, double akk) {
  if (piv > 1e-12 * akk && piv > 0.0) return piv;
  return (akk > 0.0) ? akk : 1.0;
}

/* ILU(0): incomplete LU with the sparsity pattern of A (no fill), IKJ
 * variant of Gaussian elimination restricted to the pattern. */
static void orc_ilu0_setup(orc_precond* P) {
  long nnz = P->indptr[P->n];
  memcpy(P->fact, P->data, sizeof(double) * nnz);
  for (int i = 0; i < P->n; ++i) {
    for (long pk = P->indptr[i]; pk < P->indptr[i + 1]; ++pk) {
      int k = P->indices[pk];
      if (k >= i) break;
      P->fact[pk] /= P->fact[P->dpos[k]];            /* l_ik = a_ik / u_kk */
      for (long pj = pk + 1; pj < P->indptr[i + 1]; ++pj) {
        int j = P->indices[pj];
        if (j <= k) continue;
        long kj = orc_find(P, k, j);
        if (kj >= 0) P->fact[pj] -= P->fact[pk] * P->fact[kj];
      }
    }
    P->fact[P->dpos[i]] = orc_guard_pivot(P->fact[P->dpos[i]], P->data[P->dpos[i]]);
  }
}

static void orc_ilu0_apply(const orc_precond* P, const double* r, double* s) {
  /* L y = r with unit diagonal, then U s = y. */
  for (int i = 0; i < P->n; ++i) {
    double acc = r[i];
    for (long t = P->indptr[i]; t < P->dpos[i]; ++t) acc -= P->fact[t] * s[P->indices[t]];
    s[i] = acc;
  }
  for (int i = P->n - 1; i >= 0; --i) {
    double acc = s[i];
    for (long t = P->dpos[i] + 1; t < P->indptr[i + 1]; ++t) acc -= P->fact[t] * s[P->indices[t]];
    s[i] = acc / P->fact[P->dpos[i]];
  }
}

/* IC(0): A ~ L L^T with L restricted to the lower pattern of A, row-oriented
 * (left-looking) Cholesky. */
static void orc_ic0_setup(orc_precond* P) {
  long nnz = P->indptr[P->n];
  memset(P->fact, 0, sizeof(double) * nnz);
  for (int i = 0; i < P->n; ++i) {
    for (long pj = P->indptr[i]; pj < P->dpos[i]; ++pj) {
      int j = P->indices[pj];
      double acc = P->data[pj];
      /* subtract sum_{k<j} L_ik L_jk over columns present in both rows */
      for (long pk = P->indptr[i]; pk < pj; ++pk) {
        int k = P->indices[pk];
        long jk = orc_find(P, j, k);
        if (jk >= 0) acc -= P->fact[pk] * P->fact[jk];
      }
      P->fact[pj] = acc / P->fact[P->dpos[j]];
    }
    double v = P->data[P->dpos[i]];
    for (long pk = P->indptr[i]; pk < P->dpos[i]; ++pk) v -= P->fact[pk] * P->fact[pk];
    P->fact[P->dpos[i]] = sqrt(orc_guard_pivot(v, P->data[P->dpos[i]]));
  }
}

static void orc_ic0_apply(const orc_precond* P, const double* r, double* s) {
  /* L y = r */
  for (int i = 0; i < P->n; ++i) {
    double acc = r[i];
    for (long t = P->indptr[i]; t < P->dpos[i]; ++t) acc -= P->fact[t] * s[P->indices[t]];
    s[i] = acc / P->fact[P->dpos[i]];
  }
  /* L^T s = y, column-oriented on the rows of L */
  for (int i = P->n - 1; i >= 0; --i) {
    s[i] = s[i] / P->fact[P->dpos[i]];
    for (long t = P->indptr[i]; t < P->dpos[i]; ++t) s[P->indices[t]] -= P->fact[t] * s[i];
  }
}

/* SSOR(omega): M = omega/(2-omega) (D/omega + L)(D/omega)^{-1}(D/omega + L^T),
 * L the strict lower triangle of A.  READING: the paper's "SOR factorization"
 * must be symmetric for CG, hence SSOR; a zero diagonal is replaced by 1. */
static void orc_ssor_apply(const orc_precond* P, const double* r, double* s) {
  double w = P->omega;
  for (int i = 0; i < P->n; ++i) {
    double acc = r[i];
    for (long t = P->indptr[i]; t < P->dpos[i]; ++t) acc -= P->data[t] * s[P->indices[t]];
    s[i] = acc / (P->diag[i] / w);
  }
  for (int i = 0; i < P->n; ++i) s[i] = (P->diag[i] / w) * s[i];
  for (int i = P->n - 1; i >= 0; --i) {
    double acc = s[i];
    for (long t = P->dpos[i] + 1; t < P->indptr[i + 1]; ++t) acc -= P->data[t] * s[P->indices[t]];
    s[i] = acc / (P->diag[i] / w);
  }
  for (int i = 0; i < P->n; ++i) s[i] = s[i] * ((2.0 - w) / w);
}

/* ------------------------------------------------------------------------ */
/* Red-black orderings (multicolour; the paper leaves the ordering open).    */
/* Red pixels (i + j even) come first, then black; the 5-point stencil only  */
/* couples the two colours, so both triangular solves reduce to one pass per */
/* colour.  The formulas are the natural-order ones of SSOR and ILU(0) taken */
/* in that order of the unknowns.                                             */
/* ------------------------------------------------------------------------ */
static int orc_is_red(const orc_precond* P, int k) { return ((k / P->W) + (k % P->W)) % 2 == 0; }

/* SSOR(omega) in red-black order: forward (D/w + L) y = r with red first
 * (y_red = w r / D, y_black = w (r - A_br y_red) / D), z = (D/w) y, backward
 * (D/w + L^T) s = z with black first (s_black = y_black, s_red = y_red - w
 * A_rb s_black / D), times (2 - w)/w.  A zero diagonal is replaced by 1. */
static void orc_rbssor_apply(const orc_precond* P, const double* r, double* s) {
  double w = P->omega;
  int n = P->n;
  for (int k = 0; k < n; ++k)
    if (orc_is_red(P, k)) s[k] = r[k] / (P->diag[k] / w);
  for (int k = 0; k < n; ++k) {
    if (orc_is_red(P, k)) continue;
    double acc = r[k];
    for (long t = P->indptr[k]; t < P->indptr[k + 1]; ++t)
      if (P->indices[t] != k) acc -= P->data[t] * s[P->indices[t]];  /* all neighbours are red */
    s[k] = acc / (P->diag[k] / w);
  }
  /* z = (D/w) y and the black rows of the backward solve give s_black = y_black */
  for (int k = 0; k < n; ++k) {
    if (!orc_is_red(P, k)) continue;
    double acc = (P->diag[k] / w) * s[k];
    for (long t = P->indptr[k]; t < P->indptr[k + 1]; ++t)
      if (P->indices[t] != k) acc -= P->data[t] * s[P->indices[t]];  /* all neighbours are black */
    s[k] = acc / (P->diag[k] / w);
  }
  for (int k = 0; k < n; ++k) s[k] = s[k] * ((2.0 - w) / w);
}

/* ILU(0) in red-black order: the red pivots are a_kk (no red-red coupling);
 * a black pivot is a_bb - sum over its red neighbours k of a_bk a_kb / a_kk
 * (the fill a red elimination would put into the black-black block falls on
 * the diagonal only), guarded as in the natural order.  L y = r (y_red = r,
 * y_black = r - A_br D_red^-1 y_red), U s = y (s_black = y / p, s_red =
 * (y - A_rb s_black) / a_kk).  IC(0) in this order is the same M. */
static void orc_rbilu_setup(orc_precond* P) {
  for (int k = 0; k < P->n; ++k) {
    double akk = P->data[P->dpos[k]];
    if (orc_is_red(P, k)) {
      P->fact[k] = orc_guard_pivot(akk, akk);
    }
  }
  for (int k = 0; k < P->n; ++k) {
    if (orc_is_red(P, k)) continue;
    double akk = P->data[P->dpos[k]];
    double piv = akk;
    for (long t = P->indptr[k]; t < P->indptr[k + 1]; ++t) {
      int j = P->indices[t];
      if (j == k) continue;
      long tj = orc_find(P, j, k);
      piv -= P->data[t] * P->data[tj] / P->fact[j];
    }
    P->fact[k] = orc_guard_pivot(piv, akk);
  }
}

static void orc_rbilu_apply(const orc_precond* P, const double* r, double* s) {
  int n = P->n;
  /* y_red = r_red, s_black = (r_black - sum a_bk y_k / p_k) / p_black */
  for (int k = 0; k < n; ++k) {
    if (orc_is_red(P, k)) continue;
    double acc = r[k];
    for (long t = P->indptr[k]; t < P->indptr[k + 1]; ++t) {
      int j = P->indices[t];
      if (j != k) acc -= P->data[t] / P->fact[j] * r[j];
    }
    s[k] = acc / P->fact[k];
  }
  for (int k = 0; k < n; ++k) {
    if (!orc_is_red(P, k)) continue;
    double acc = r[k];
    for (long t = P->indptr[k]; t < P->indptr[k + 1]; ++t) {
      int j = P->indices[t];
      if (j != k) acc -= P->data[t] * s[j];
    }
    s[k] = acc / P->fact[k];
  }
}

/* Orthonormal DCT-II matrix C[k][x] = c_k cos(pi k (x + 1/2) / n). */
static void orc_dct_matrix(int n, double* C) {
  for (int k = 0; k < n; ++k) {
    double ck = (k == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n);
    for (int x = 0; x < n; ++x) C[(long)k * n + x] = ck * cos(ORC_PI * k * (x + 0.5) / n);
  }
}

/* Fourier-basis Poisson solver (Sec. 1, Green-function/Fourier approach):
 * s = Pi L^+ r, L the unit-weight Neumann 5-point Laplacian, whose
 * eigenvectors are products of DCT-II vectors with eigenvalues
 * (2 - 2 cos(pi k / H)) + (2 - 2 cos(pi l / W)); the zero mode is dropped and
 * Pi zeroes masked pixels.  Written as explicit matrix products. */
static void orc_dct_apply(const orc_precond* P, const double* r, double* s) {
  int H = P->H, W = P->W;
  /* tmp = C_H r */
  for (int k = 0; k < H; ++k)
    for (int j = 0; j < W; ++j) {
      double acc = 0.0;
      for (int i = 0; i < H; ++i) acc += P->ch[(long)k * H + i] * r[(long)i * W + j];
      P->tmp[(long)k * W + j] = acc;
    }
  /* tmp2 = tmp C_W^T, then divide by the eigenvalues */
  for (int k = 0; k < H; ++k)
    for (int l = 0; l < W; ++l) {
      double acc = 0.0;
      for (int j = 0; j < W; ++j) acc += P->tmp[(long)k * W + j] * P->cw[(long)l * W + j];
      double lam = P->lam[(long)k * W + l];
      P->tmp2[(long)k * W + l] = (k == 0 && l == 0) ? 0.0 : acc / lam;
    }
  /* tmp = C_H^T tmp2 */
  for (int i = 0; i < H; ++i)
    for (int l = 0; l < W; ++l) {
      double acc = 0.0;
      for (int k = 0; k < H; ++k) acc += P->ch[(long)k * H + i] * P->tmp2[(long)k * W + l];
      P->tmp[(long)i * W + l] = acc;
    }
  /* s = tmp C_W */
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) {
      double acc = 0.0;
      for (int l = 0; l < W; ++l) acc += P->tmp[(long)i * W + l] * P->cw[(long)l * W + j];
      long k = (long)i * W + j;
      s[k] = (P->mask && P->mask[k]) ? 0.0 : acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Multigrid (Sec. 1 names multigrid with the Fourier methods as the fast    */
/* solvers of this system): one V-cycle of aggregation multigrid as a fixed  */
/* SPD-in-practice M.  Grids: 2x2 aggregates, Galerkin coarse operators      */
/* A_{l+1} = P^T A_l P (again 5-point weighted Laplacians, orc_mg_coarsen),   */
/* down to at most ORC_MG_COARSE_MAX unknowns.  Smoother: damped Jacobi,      */
/* weight ORC_MG_OMEGA, ORC_MG_NU sweeps before and after the coarse          */
/* correction (the same count, so the cycle is symmetric); the correction is */
/* scaled by ORC_MG_CC (over-correction for piecewise-constant P); the        */
/* coarsest grid gets ORC_MG_COARSE_SWEEPS sweeps from zero.                  */
/* ------------------------------------------------------------------------ */
void orc_mg_coarsen(const double* U, const double* V, int H, int W, double* Uc, double* Vc) {
  int Hc = (H + 1) / 2, Wc = (W + 1) / 2;
  for (int I = 0; I < Hc; ++I)
    for (int J = 0; J < Wc; ++J) {
      double u = 0.0, v = 0.0;
      /* edge between aggregates (I,J) and (I,J+1): the fine edges (i, 2J+1)-(i, 2J+2) */
      if (2 * J + 2 < W)
        for (int i = 2 * I; i <= 2 * I + 1 && i < H; ++i) u += U[(long)i * W + 2 * J + 1];
      /* edge between aggregates (I,J) and (I+1,J): the fine edges (2I+1, j)-(2I+2, j) */
      if (2 * I + 2 < H)
        for (int j = 2 * J; j <= 2 * J + 1 && j < W; ++j) v += V[(long)(2 * I + 1) * W + j];
      Uc[(long)I * Wc + J] = u;
      Vc[(long)I * Wc + J] = v;
    }
}

/* y = A x on a grid given by its edge weights (Eq. Axb's operator). */
static void orc_grid_matvec(const double* U, const double* V, const double* D, int H, int W,
                            const double* x, double* y) {
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) {
      long k = (long)i * W + j;
      double acc = D[k] * x[k];
      if (j + 1 < W) acc -= U[k] * x[k + 1];
      if (j > 0) acc -= U[k - 1] * x[k - 1];
      if (i + 1 < H) acc -= V[k] * x[k + W];
      if (i > 0) acc -= V[k - W] * x[k - W];
      y[k] = acc;
    }
}

/* nu damped-Jacobi sweeps x <- x + omega D^-1 (b - A x) (D = 0: no update). */
static void orc_mg_smooth(const orc_precond* P, int l, const double* b, double* x, int nu) {
  int H = P->mg_h[l], W = P->mg_w[l];
  long n = (long)H * W;
  double* Ax = P->mg_t[l];
  for (int s = 0; s < nu; ++s) {
    orc_grid_matvec(P->mg_u[l], P->mg_v[l], P->mg_d[l], H, W, x, Ax);
    for (long k = 0; k < n; ++k)
      if (P->mg_d[l][k] > 0.0) x[k] += ORC_MG_OMEGA * (b[k] - Ax[k]) / P->mg_d[l][k];
  }
}

/* x = V-cycle(l) applied to b (x starts at 0). */
static void orc_mg_vcycle(const orc_precond* P, int l, const double* b, double* x) {
  int H = P->mg_h[l], W = P->mg_w[l];
  long n = (long)H * W;
  for (long k = 0; k < n; ++k) x[k] = 0.0;
  if (l == P->mg_levels - 1) {
    orc_mg_smooth(P, l, b, x, ORC_MG_COARSE_SWEEPS);
    return;
  }
  orc_mg_smooth(P, l, b, x, ORC_MG_NU);
  /* restrict the residual: b_c = P^T (b - A x), the sum over each aggregate */
  double* r = P->mg_t[l];
  orc_grid_matvec(P->mg_u[l], P->mg_v[l], P->mg_d[l], H, W, x, r);
  int Hc = P->mg_h[l + 1], Wc = P->mg_w[l + 1];
  double* bc = P->mg_b[l + 1];
  for (long k = 0; k < (long)Hc * Wc; ++k) bc[k] = 0.0;
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) {
      long k = (long)i * W + j;
      bc[(long)(i / 2) * Wc + j / 2] += b[k] - r[k];
    }
  double* xc = P->mg_x[l + 1];
  orc_mg_vcycle(P, l + 1, bc, xc);
  /* prolong and correct: x += cc P x_c */
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) x[(long)i * W + j] += ORC_MG_CC * xc[(long)(i / 2) * Wc + j / 2];
  orc_mg_smooth(P, l, b, x, ORC_MG_NU);
}

static int orc_mg_setup(orc_precond* P) {
  int H = P->H, W = P->W;
  long n = (long)H * W;
  /* level 0 weights from the CSR matrix: U_k = -A[k][k+1], V_k = -A[k][k+W] */
  P->mg_levels = 1;
  P->mg_h[0] = H;
  P->mg_w[0] = W;
  P->mg_u[0] = (double*)calloc(n, sizeof(double));
  P->mg_v[0] = (double*)calloc(n, sizeof(double));
  if (!P->mg_u[0] || !P->mg_v[0]) return ORC_INVALID;
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) {
      long k = (long)i * W + j;
      long t;
      if (j + 1 < W && (t = orc_find(P, (int)k, (int)(k + 1))) >= 0) P->mg_u[0][k] = -P->data[t];
      if (i + 1 < H && (t = orc_find(P, (int)k, (int)(k + W))) >= 0) P->mg_v[0][k] = -P->data[t];
    }
  while ((long)P->mg_h[P->mg_levels - 1] * P->mg_w[P->mg_levels - 1] > ORC_MG_COARSE_MAX && P->mg_levels < 32) {
    int l = P->mg_levels - 1;
    int Hc = (P->mg_h[l] + 1) / 2, Wc = (P->mg_w[l] + 1) / 2;
    P->mg_u[l + 1] = (double*)calloc((long)Hc * Wc, sizeof(double));
    P->mg_v[l + 1] = (double*)calloc((long)Hc * Wc, sizeof(double));
    if (!P->mg_u[l + 1] || !P->mg_v[l + 1]) return ORC_INVALID;
    orc_mg_coarsen(P->mg_u[l], P->mg_v[l], P->mg_h[l], P->mg_w[l], P->mg_u[l + 1], P->mg_v[l + 1]);
    P->mg_h[l + 1] = Hc;
    P->mg_w[l + 1] = Wc;
    P->mg_levels += 1;
  }
  for (int l = 0; l < P->mg_levels; ++l) {
    int h = P->mg_h[l], w = P->mg_w[l];
    long m = (long)h * w;
    P->mg_d[l] = (double*)calloc(m, sizeof(double));
    P->mg_x[l] = (double*)calloc(m, sizeof(double));
    P->mg_b[l] = (double*)calloc(m, sizeof(double));
    P->mg_t[l] = (double*)calloc(m, sizeof(double));
    if (!P->mg_d[l] || !P->mg_x[l] || !P->mg_b[l] || !P->mg_t[l]) return ORC_INVALID;
    /* the diagonal of the grid's Laplacian: the sum of its incident edge weights */
    for (int i = 0; i < h; ++i)
      for (int j = 0; j < w; ++j) {
        long k = (long)i * w + j;
        double d = P->mg_u[l][k] + P->mg_v[l][k];
        if (j > 0) d += P->mg_u[l][k - 1];
        if (i > 0) d += P->mg_v[l][k - w];
        P->mg_d[l][k] = d;
      }
  }
  return ORC_OK;
}

static void orc_mg_apply(const orc_precond* P, const double* r, double* s) {
  orc_mg_vcycle(P, 0, r, s);
  if (P->mask)
    for (int k = 0; k < P->n; ++k)
      if (P->mask[k]) s[k] = 0.0;
}

static int orc_precond_setup(orc_precond* P, int kind, int H, int W,
                             const long* indptr, const int* indices,
                             const double* data, double omega,
                             const uint8_t* mask) {
  memset(P, 0, sizeof(*P));
  P->kind = kind; P->H = H; P->W = W; P->n = H * W;
  P->indptr = indptr; P->indices = indices; P->data = data;
  P->omega = omega; P->mask = mask;
  int n = P->n;
  long nnz = indptr[n];
  P->dpos = (long*)malloc(sizeof(long) * n);
  P->diag = (double*)malloc(sizeof(double) * n);
  if (!P->dpos || !P->diag) return ORC_INVALID;
  for (int i = 0; i < n; ++i) {
    P->dpos[i] = orc_find(P, i, i);
    P->diag[i] = data[P->dpos[i]];
  }
  switch (kind) {
    case ORC_M_IDENTITY:
    case ORC_M_JACOBI:
      break;
    case ORC_M_SSOR:
      if (!(omega > 0.0 && omega < 2.0)) return ORC_INVALID;
      for (int i = 0; i < n; ++i) if (!(P->diag[i] > 0.0)) P->diag[i] = 1.0;
      break;
    case ORC_M_ILU0:
      P->fact = (double*)malloc(sizeof(double) * nnz);
      if (!P->fact) return ORC_INVALID;
      orc_ilu0_setup(P);
      break;
    case ORC_M_IC0:
      P->fact = (double*)malloc(sizeof(double) * nnz);
      if (!P->fact) return ORC_INVALID;
      orc_ic0_setup(P);
      break;
    case ORC_M_DCT:
      P->ch = (double*)malloc(sizeof(double) * H * H);
      P->cw = (double*)malloc(sizeof(double) * W * W);
      P->lam = (double*)malloc(sizeof(double) * n);
      P->tmp = (double*)malloc(sizeof(double) * n);
      P->tmp2 = (double*)malloc(sizeof(double) * n);
      if (!P->ch || !P->cw || !P->lam || !P->tmp || !P->tmp2) return ORC_INVALID;
      orc_dct_matrix(H, P->ch);
      orc_dct_matrix(W, P->cw);
      for (int k = 0; k < H; ++k)
        for (int l = 0; l < W; ++l)
          P->lam[(long)k * W + l] = (2.0 - 2.0 * cos(ORC_PI * k / H)) + (2.0 - 2.0 * cos(ORC_PI * l / W));
      break;
    case ORC_M_MG:
      return orc_mg_setup(P);
    case ORC_M_RBSSOR:
      if (!(omega > 0.0 && omega < 2.0)) return ORC_INVALID;
      for (int i = 0; i < n; ++i) if (!(P->diag[i] > 0.0)) P->diag[i] = 1.0;
      break;
    case ORC_M_RBILU:
      P->fact = (double*)malloc(sizeof(double) * n);
      if (!P->fact) return ORC_INVALID;
      orc_rbilu_setup(P);
      break;
    default:
      return ORC_INVALID;
  }
  return ORC_OK;
}

static void orc_precond_free(orc_precond* P) {
  free(P->dpos); free(P->diag); free(P->fact);
  free(P->ch); free(P->cw); free(P->lam); free(P->tmp); free(P->tmp2);
  for (int l = 0; l < P->mg_levels; ++l) {
    free(P->mg_u[l]); free(P->mg_v[l]); free(P->mg_d[l]);
    free(P->mg_x[l]); free(P->mg_b[l]); free(P->mg_t[l]);
  }
}

static void orc_precond_solve(const orc_precond* P, const double* r, double* s) {
  int n = P->n;
  switch (P->kind) {
    case ORC_M_IDENTITY:
      for (int i = 0; i < n; ++i) s[i] = r[i];
      break;
    case ORC_M_JACOBI:
      /* READING: a zero diagonal (isolated or masked pixel) gives s = 0. */
      for (int i = 0; i < n; ++i) s[i] = (P->diag[i] > 0.0) ? r[i] / P->diag[i] : 0.0;
      break;
    case ORC_M_ILU0: orc_ilu0_apply(P, r, s); break;
    case ORC_M_IC0: orc_ic0_apply(P, r, s); break;
    case ORC_M_SSOR: orc_ssor_apply(P, r, s); break;
    case ORC_M_DCT: orc_dct_apply(P, r, s); break;
    case ORC_M_MG: orc_mg_apply(P, r, s); break;
    case ORC_M_RBSSOR: orc_rbssor_apply(P, r, s); break;
    case ORC_M_RBILU: orc_rbilu_apply(P, r, s); break;
  }
}

int orc_precond_apply(int kind, int H, int W, const long* indptr,
                      const int* indices, const double* data, double omega,
                      const uint8_t* mask, const double* r, double* s) {
  orc_precond P;
  int st = orc_precond_setup(&P, kind, H, W, indptr, indices, data, omega, mask);
  if (st == ORC_OK) orc_precond_solve(&P, r, s);
  orc_precond_free(&P);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Inner PCG: Algorithm 1, the "solve Eq. (Axb) using PCG" block.           */
/* ------------------------------------------------------------------------ */
int orc_pcg(int H, int W, const long* indptr, const int* indices,
            const double* data, const double* b, const uint8_t* mask,
            const orc_pcg_opts* o, double* phi, orc_pcg_result* res) {
  int n = H * W;
  long lmax = (o->max_inner > 0) ? o->max_inner : 2L * n;           /* l_max = 2MN */
  long refresh = (o->refresh > 0) ? o->refresh : (long)floor(sqrt((double)n));
  if (refresh < 1) refresh = 1;
  double tol2 = o->tol * o->tol;
  orc_precond P;
  const double t_setup = orc_now();
  int st = orc_precond_setup(&P, o->kind, H, W, indptr, indices, data, o->omega, mask);
  res->setup_s = orc_now() - t_setup;  /* "estimate preconditioning matrix M from A" */
  if (st != ORC_OK) { orc_precond_free(&P); return st; }

  double* r = (double*)malloc(sizeof(double) * n);
  double* d = (double*)malloc(sizeof(double) * n);
  double* q = (double*)malloc(sizeof(double) * n);
  double* s = (double*)malloc(sizeof(double) * n);
  if (!r || !d || !q || !s) { free(r); free(d); free(q); free(s); orc_precond_free(&P); return ORC_INVALID; }

  /* r <- b - A phi ; d <- M^{-1} r ; delta_new <- r^T d ; delta_0 <- delta_new */
  orc_csr_matvec(n, indptr, indices, data, phi, q);
  for (int t = 0; t < n; ++t) r[t] = b[t] - q[t];
  orc_precond_solve(&P, r, d);
  double delta_new = orc_dot(n, r, d);
  double delta_0 = delta_new;
  double bb = orc_dot(n, b, b);
  double rr = orc_dot(n, r, r);
  long l = 0;
  int status = ORC_OK;

  if (bb > 0.0) {
    for (;;) {
      int done = (o->stop_mode == ORC_STOP_PAPER) ? !(delta_new > tol2 * delta_0)
                                                   : !(rr > tol2 * bb);
      if (done) break;
      if (l >= lmax) { status = ORC_MAXITER; break; }
      orc_csr_matvec(n, indptr, indices, data, d, q);             /* q <- A d */
      double dq = orc_dot(n, d, q);
      if (!(dq > 0.0) || !isfinite(dq)) { status = ORC_BREAKDOWN; break; }
      double alpha = delta_new / dq;                              /* alpha <- delta_new / d^T q */
      for (int t = 0; t < n; ++t) phi[t] = phi[t] + alpha * d[t];
      if (l % refresh == 0) {                                     /* true residual */
        orc_csr_matvec(n, indptr, indices, data, phi, q);
        for (int t = 0; t < n; ++t) r[t] = b[t] - q[t];
      } else {
        for (int t = 0; t < n; ++t) r[t] = r[t] - alpha * q[t];
      }
      orc_precond_solve(&P, r, s);                                /* s <- M^{-1} r */
      double delta_old = delta_new;
      delta_new = orc_dot(n, r, s);
      rr = orc_dot(n, r, r);
      double beta = delta_new / delta_old;
      for (int t = 0; t < n; ++t) d[t] = s[t] + beta * d[t];
      l += 1;
    }
  }
  res->iters = l;
  res->status = status;
  res->relres = (bb > 0.0) ? sqrt(rr / bb) : 0.0;
  orc_csr_matvec(n, indptr, indices, data, phi, q);
  double tr = 0.0;
  for (int t = 0; t < n; ++t) { double e = b[t] - q[t]; tr += e * e; }
  res->true_relres = (bb > 0.0) ? sqrt(tr / bb) : sqrt(tr);
  free(r); free(d); free(q); free(s);
  orc_precond_free(&P);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: the outer reweighting loop.                                 */
/* ------------------------------------------------------------------------ */
int orc_unwrap(const double* psi, const uint8_t* mask, int H, int W, double p,
               double tau, const orc_pcg_opts* o, int max_outer,
               double outer_tol, double* phi, orc_unwrap_stats* st) {
  if (H < 2 || W < 2 || !(p >= 0.0 && p <= 2.0) || !(tau > 0.0)) return ORC_INVALID;
  long n = (long)H * W;
  for (long t = 0; t < n; ++t) if (!isfinite(psi[t])) return ORC_INVALID;
  double* dx = (double*)malloc(sizeof(double) * n);
  double* dy = (double*)malloc(sizeof(double) * n);
  double* U = (double*)malloc(sizeof(double) * n);
  double* V = (double*)malloc(sizeof(double) * n);
  double* b = (double*)malloc(sizeof(double) * n);
  double* phin = (double*)malloc(sizeof(double) * n);
  long* indptr = (long*)malloc(sizeof(long) * (n + 1));
  int* indices = (int*)malloc(sizeof(int) * 5 * n);
  double* data = (double*)malloc(sizeof(double) * 5 * n);
  int rc = ORC_OK;
  if (!dx || !dy || !U || !V || !b || !phin || !indptr || !indices || !data) { rc = ORC_INVALID; goto out; }
  memset(st, 0, sizeof(*st));

  orc_wrapped_diffs(psi, H, W, dx, dy);
  int k = 0;
  double error = 1.0;                                   /* k <- 0, error <- 1 */
  while (k < max_outer && error > outer_tol) {
    orc_weights(phi, dx, dy, mask, H, W, p, tau, U, V);         /* Eq. (UV) */
    orc_assemble(U, V, dx, dy, H, W, indptr, indices, data, b); /* Eq. (Axb) */
    memcpy(phin, phi, sizeof(double) * n);                      /* phi^{k+1} <- phi^k */
    orc_pcg_result pr;
    int s = orc_pcg(H, W, indptr, indices, data, b, mask, o, phin, &pr);
    if (s < 0 && s != ORC_BREAKDOWN) { rc = s; goto out; }
    double num = 0.0, den = 0.0;
    for (long t = 0; t < n; ++t) {
      double e = phin[t] - phi[t];
      num += e * e;
      den += phi[t] * phi[t];
    }
    /* READING: ||phi^k|| = 0 (the default phi^0 = 0) makes the error infinite. */
    error = (den > 0.0) ? sqrt(num) / sqrt(den) : INFINITY;
    memcpy(phi, phin, sizeof(double) * n);
    if (k < 64) { st->inner[k] = pr.iters; st->relres[k] = pr.relres; st->outer_err[k] = error; }
    st->inner_total += pr.iters;
    st->setup_s += pr.setup_s;
    if (pr.status == ORC_BREAKDOWN) st->status = ORC_BREAKDOWN;
    else if (pr.status == ORC_MAXITER && st->status == ORC_OK) st->status = ORC_MAXITER;
    k += 1;
  }
  st->outer = k;
  rc = st->status;
out:
  free(dx); free(dy); free(U); free(V); free(b); free(phin);
  free(indptr); free(indices); free(data);
  return rc;
}

/* Congruence post-step (Ghiglia & Pritt): phi_c = phi + W(psi - phi), so that
 * W(phi_c) = psi. */
void orc_congruence(const double* phi, const double* psi, long n, double* out) {
  for (long t = 0; t < n; ++t) out[t] = phi[t] + orc_wrap(psi[t] - phi[t]);
}

/* Q(mu, nu) = ||mu - nu||_2 / (||mu||_2 + ||nu||_2)  (Sec. 3). */
double orc_quality_q(const double* mu, const double* nu, long n) {
  double d = 0.0, a = 0.0, c = 0.0;
  for (long t = 0; t < n; ++t) {
    double e = mu[t] - nu[t];
    d += e * e; a += mu[t] * mu[t]; c += nu[t] * nu[t];
  }
  double den = sqrt(a) + sqrt(c);
  return (den > 0.0) ? sqrt(d) / den : 0.0;
}

/* Eq. (funcional), discretised with the forward differences of Sec. 2.1:
 * J = sum |delta_x^+ phi - Delta^x|^p + |delta_y^+ phi - Delta^y|^p over
 * the edges inside the grid whose endpoints are both unmasked. */
double orc_functional(const double* phi, const double* dx, const double* dy,
                      const uint8_t* mask, int H, int W, double p) {
  double J = 0.0;
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) {
      long k = (long)i * W + j;
      int mk = mask ? (mask[k] != 0) : 0;
      if (j + 1 < W && !mk && !(mask && mask[k + 1])) J += pow(fabs(phi[k + 1] - phi[k] - dx[k]), p);
      if (i + 1 < H && !mk && !(mask && mask[k + W])) J += pow(fabs(phi[k + W] - phi[k] - dy[k]), p);
    }
  return J;
}
