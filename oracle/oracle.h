/*
 * oracle.h -- FP64 single-threaded CPU oracle of the L^p-norm phase-unwrapping
 * method (Legarda-Saenz, Brito-Loeza, Espinosa-Romero, arXiv 2203.13675).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load this library.  It shares no code, header,
 * table or constant with the CUDA library; neither includes the other.
 *
 * Grid convention: H rows (index i, the paper's y direction) by W columns
 * (index j, the paper's x direction); pixel (i,j) lives at k = i*W + j
 * (natural row-major order).  All planes are contiguous row-major doubles.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_M_IDENTITY = 0, /* M = I, Sec. 2 list item 1 */
  ORC_M_JACOBI = 1,   /* M = diag(A), item 2 */
  ORC_M_ILU0 = 2,     /* ILU(0), item 3 */
  ORC_M_IC0 = 3,      /* IC(0), item 4 */
  ORC_M_SSOR = 4,     /* "SOR factorization", item 5, read as SSOR(omega) */
  ORC_M_DCT = 5,      /* unweighted Neumann-Poisson pseudo-inverse (Fourier basis, Sec. 1) */
  ORC_M_MG = 7,       /* one symmetric aggregation-multigrid V-cycle (multigrid, Sec. 1) */
  ORC_M_RBSSOR = 8,   /* SSOR(omega) with the unknowns in red-black order (red: i + j even, first) */
  ORC_M_RBILU = 9     /* ILU(0) = IC(0) with the unknowns in red-black order */
};

/* Multigrid parameters (the method's definition, see orc_mg_*): damped-Jacobi
 * weight, sweeps before and after the coarse correction, the coarse-correction
 * scale, the sweeps on the coarsest grid and its size bound. */
#define ORC_MG_OMEGA (2.0 / 3.0)
#define ORC_MG_NU 2
#define ORC_MG_CC 1.5
#define ORC_MG_COARSE_SWEEPS 30
#define ORC_MG_COARSE_MAX 16

/* Galerkin coarsening of the 5-point weighted Laplacian by 2x2 aggregation:
 * the coarse edge weights of P^T A P, P the piecewise-constant prolongation
 * (aggregate (I,J) = fine rows 2I, 2I+1 and columns 2J, 2J+1, clipped at the
 * border).  Uc, Vc are ((H+1)/2) x ((W+1)/2). */
void orc_mg_coarsen(const double* U, const double* V, int H, int W, double* Uc, double* Vc);

enum { ORC_STOP_RELRES = 0, ORC_STOP_PAPER = 1 };

enum { ORC_OK = 0, ORC_MAXITER = 1, ORC_BREAKDOWN = -3, ORC_INVALID = -1 };

/* Eq. (wrapped): principal value in (-pi, pi]. */
double orc_wrap(double x);

/* Wrapped differences Delta^x, Delta^y (Sec. 2.1, definitions after Eq. gradientep). */
void orc_wrapped_diffs(const double* psi, int H, int W, double* dx, double* dy);

/* Eq. (UV): regularised IRLS weights. mask may be NULL (1 = pixel excluded). */
void orc_weights(const double* phi, const double* dx, const double* dy,
                 const uint8_t* mask, int H, int W, double p, double tau,
                 double* U, double* V);

/* Eq. (Axb): CSR matrix A (structural 5-point pattern, columns ascending) and b.
 * indptr has H*W+1 entries; indices/data have room for 5*H*W entries.
 * Returns nnz. */
long orc_assemble(const double* U, const double* V, const double* dx,
                  const double* dy, int H, int W, long* indptr, int* indices,
                  double* data, double* b);

/* y = A x for a CSR matrix. */
void orc_csr_matvec(int n, const long* indptr, const int* indices,
                    const double* data, const double* x, double* y);

/* Build the preconditioner kind for CSR A and apply it once: s = M^{-1} r. */
int orc_precond_apply(int kind, int H, int W, const long* indptr,
                      const int* indices, const double* data, double omega,
                      const uint8_t* mask, const double* r, double* s);

typedef struct {
  int kind;          /* ORC_M_* */
  int stop_mode;     /* ORC_STOP_* */
  double tol;        /* RELRES: ||r|| <= tol ||b||.  PAPER: delta_new <= tol^2 delta_0 */
  long max_inner;    /* l_max; <= 0 means 2*H*W */
  long refresh;      /* true-residual period; <= 0 means floor(sqrt(H*W)) */
  double omega;      /* SSOR relaxation */
} orc_pcg_opts;

typedef struct {
  long iters;        /* l at exit */
  int status;        /* ORC_OK, ORC_MAXITER or ORC_BREAKDOWN */
  double relres;     /* ||r_l|| / ||b|| of the recurrence residual at exit */
  double true_relres;/* ||b - A phi|| / ||b|| at exit */
  double setup_s;    /* wall time of building M from A (seconds), for the set-up share of Sec. 3 */
} orc_pcg_result;

/* Inner PCG of Algorithm 1 on CSR A, warm-started from phi (overwritten). */
int orc_pcg(int H, int W, const long* indptr, const int* indices,
            const double* data, const double* b, const uint8_t* mask,
            const orc_pcg_opts* o, double* phi, orc_pcg_result* res);

typedef struct {
  int outer;             /* outer passes run */
  int status;            /* worst inner status */
  long inner_total;
  long inner[64];        /* per-outer inner iterations (first 64 passes) */
  double relres[64];
  double outer_err[64];
  double setup_s;        /* summed wall time of building M in every pass (seconds) */
} orc_unwrap_stats;

/* Algorithm 1: IRLS outer loop around the inner PCG.  phi holds phi^0 on
 * entry and the result on exit.  outer_tol <= 0 runs exactly max_outer passes. */
int orc_unwrap(const double* psi, const uint8_t* mask, int H, int W, double p,
               double tau, const orc_pcg_opts* o, int max_outer,
               double outer_tol, double* phi, orc_unwrap_stats* st);

/* Ghiglia-Pritt congruence post-step: phi_c = phi + W(psi - phi). */
void orc_congruence(const double* phi, const double* psi, long n, double* out);

/* Normalised error Q of Sec. 3 (Perlin 2016). */
double orc_quality_q(const double* mu, const double* nu, long n);

/* Discrete L^p functional of Eq. (funcional) with the forward differences. */
double orc_functional(const double* phi, const double* dx, const double* dy,
                      const uint8_t* mask, int H, int W, double p);

#ifdef __cplusplus
}
#endif
#endif
