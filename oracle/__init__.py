"""FP64 CPU oracle of the L^p-norm phase-unwrapping method (arXiv 2203.13675).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
(``paper_2203_13675_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, built with
``-ffp-contract=off``); this module only compiles it with gcc and marshals
numpy arrays through ctypes.  Every function states the passage it follows.

Parity status per function (what pins it, see ``tests/test_oracle_*.py``):
  wrap, wrapped_diffs       -- tie-break/range/periodicity, hand-worked grids
  weights                   -- special cases p = 0, 1, 2, hand-worked grids
  assemble                  -- Table 1 nnz, A1 = 0, sum b = 0, symmetry, edge-energy identity
  precond_apply             -- ILU(0) = IC(0), SSOR(1) = symmetric Gauss-Seidel,
                               Jacobi closed form, DCT apply vs a dense Neumann Laplacian,
                               multigrid: Galerkin coarse operator = P^T A P (dense),
                               symmetric cycle, two-grid limit against a dense solve
  pcg                       -- dense direct solve (<= 16x16), closed-form DCT solve (p = 2),
                               one-iteration convergence with the DCT M at p = 2, finite termination
  unwrap                    -- exact recovery of noiseless phase, M-independence
  congruence, quality_q     -- definitions checked on constructed cases
  functional                -- hand case; shift invariance, degree-p homogeneity, row/column
                               symmetry, zero at a noiseless congruent phase, masked edges free,
                               and at p = 2 its gradient equals (2 / c)(A phi - b) from assemble
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

M_IDENTITY, M_JACOBI, M_ILU0, M_IC0, M_SSOR, M_DCT = range(6)
M_MG = 7
M_RBSSOR, M_RBILU = 8, 9
STOP_RELRES, STOP_PAPER = 0, 1
OK, MAXITER, INVALID, BREAKDOWN = 0, 1, -1, -3


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (no GPU needed)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class PcgOpts(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("stop_mode", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_inner", ctypes.c_long), ("refresh", ctypes.c_long), ("omega", ctypes.c_double)]


class PcgResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_long), ("status", ctypes.c_int), ("relres", ctypes.c_double),
                ("true_relres", ctypes.c_double), ("setup_s", ctypes.c_double)]


class UnwrapStats(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int), ("status", ctypes.c_int), ("inner_total", ctypes.c_long),
                ("inner", ctypes.c_long * 64), ("relres", ctypes.c_double * 64),
                ("outer_err", ctypes.c_double * 64), ("setup_s", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)
_I = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("ORACLE_LIB_OVERRIDE") or build()
            L = ctypes.CDLL(path)
            L.orc_wrap.restype = ctypes.c_double
            L.orc_wrap.argtypes = [ctypes.c_double]
            L.orc_wrapped_diffs.argtypes = [_D, ctypes.c_int, ctypes.c_int, _D, _D]
            L.orc_weights.argtypes = [_D, _D, _D, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, _D, _D]
            L.orc_assemble.restype = ctypes.c_long
            L.orc_assemble.argtypes = [_D, _D, _D, _D, ctypes.c_int, ctypes.c_int, _L, _I, _D, _D]
            L.orc_csr_matvec.argtypes = [ctypes.c_int, _L, _I, _D, _D, _D]
            L.orc_precond_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _L, _I, _D,
                                            ctypes.c_double, _U8, _D, _D]
            L.orc_pcg.argtypes = [ctypes.c_int, ctypes.c_int, _L, _I, _D, _D, _U8,
                                  ctypes.POINTER(PcgOpts), _D, ctypes.POINTER(PcgResult)]
            L.orc_unwrap.argtypes = [_D, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.POINTER(PcgOpts), ctypes.c_int,
                                     ctypes.c_double, _D, ctypes.POINTER(UnwrapStats)]
            L.orc_congruence.argtypes = [_D, _D, ctypes.c_long, _D]
            L.orc_quality_q.restype = ctypes.c_double
            L.orc_quality_q.argtypes = [_D, _D, ctypes.c_long]
            L.orc_functional.restype = ctypes.c_double
            L.orc_functional.argtypes = [_D, _D, _D, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.orc_mg_coarsen.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, _D, _D]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _mask(mask, shape):
    if mask is None:
        return None, None
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    assert m.shape == shape
    return m, m.ctypes.data_as(_U8)


def wrap(x):
    """Eq. (wrapped): principal value in (-pi, pi] (elementwise)."""
    f = lib().orc_wrap
    x = np.asarray(x, dtype=np.float64)
    return np.vectorize(f, otypes=[np.float64])(x) if x.ndim else np.float64(f(float(x)))


def wrapped_diffs(psi):
    """Sec. 2.1: Delta^x (along columns j), Delta^y (along rows i)."""
    psi = _f64(psi)
    H, W = psi.shape
    dx = np.empty_like(psi)
    dy = np.empty_like(psi)
    lib().orc_wrapped_diffs(_d(psi), H, W, _d(dx), _d(dy))
    return dx, dy


def weights(phi, dx, dy, mask=None, p=1.0, tau=0.01):
    """Eq. (UV): U (edges (i,j)-(i,j+1)), V (edges (i,j)-(i+1,j))."""
    phi, dx, dy = _f64(phi), _f64(dx), _f64(dy)
    H, W = phi.shape
    m, mp = _mask(mask, phi.shape)
    U = np.empty_like(phi)
    V = np.empty_like(phi)
    lib().orc_weights(_d(phi), _d(dx), _d(dy), mp, H, W, float(p), float(tau), _d(U), _d(V))
    return U, V


class Csr:
    """CSR matrix of Eq. (Axb) plus its right-hand side b."""

    def __init__(self, H, W, indptr, indices, data, b):
        self.H, self.W = H, W
        self.indptr, self.indices, self.data, self.b = indptr, indices, data, b

    @property
    def nnz(self):
        return int(self.indptr[-1])

    def matvec(self, x):
        x = _f64(x).reshape(-1)
        y = np.empty_like(x)
        lib().orc_csr_matvec(self.H * self.W, self.indptr.ctypes.data_as(_L),
                             self.indices.ctypes.data_as(_I), _d(self.data), _d(x), _d(y))
        return y.reshape(self.H, self.W)

    def dense(self):
        n = self.H * self.W
        A = np.zeros((n, n))
        for r in range(n):
            for t in range(self.indptr[r], self.indptr[r + 1]):
                A[r, self.indices[t]] = self.data[t]
        return A


def assemble(U, V, dx, dy):
    """Eq. (Axb): the 5-point weighted Laplacian A (CSR) and b."""
    U, V, dx, dy = _f64(U), _f64(V), _f64(dx), _f64(dy)
    H, W = U.shape
    n = H * W
    indptr = np.zeros(n + 1, dtype=np.int64)
    indices = np.zeros(5 * n, dtype=np.int32)
    data = np.zeros(5 * n, dtype=np.float64)
    b = np.empty((H, W), dtype=np.float64)
    nnz = lib().orc_assemble(_d(U), _d(V), _d(dx), _d(dy), H, W, indptr.ctypes.data_as(_L),
                             indices.ctypes.data_as(_I), _d(data), _d(b))
    return Csr(H, W, indptr, indices[:nnz].copy(), data[:nnz].copy(), b)


def mg_coarsen(U, V):
    """Galerkin 2x2-aggregation coarsening of the weighted 5-point Laplacian (multigrid M)."""
    U, V = _f64(U), _f64(V)
    H, W = U.shape
    Uc = np.empty(((H + 1) // 2, (W + 1) // 2))
    Vc = np.empty_like(Uc)
    lib().orc_mg_coarsen(_d(U), _d(V), H, W, _d(Uc), _d(Vc))
    return Uc, Vc


def precond_apply(kind, A: Csr, r, omega=1.0, mask=None):
    """Sec. 2 preconditioner list: build M from A and return s = M^{-1} r."""
    r = _f64(r)
    s = np.empty_like(r)
    m, mp = _mask(mask, r.shape)
    rc = lib().orc_precond_apply(int(kind), A.H, A.W, A.indptr.ctypes.data_as(_L),
                                 A.indices.ctypes.data_as(_I), _d(A.data), float(omega), mp,
                                 _d(r), _d(s))
    if rc != OK:
        raise ValueError(f"precond_apply failed: {rc}")
    return s


def pcg(A: Csr, phi0, kind=M_JACOBI, tol=1e-6, max_inner=0, stop_mode=STOP_RELRES, refresh=0,
        omega=1.0, mask=None, b=None):
    """Algorithm 1 inner PCG (Shewchuk's variant), warm-started from phi0."""
    phi = _f64(phi0).copy()
    bb = A.b if b is None else _f64(b)
    m, mp = _mask(mask, phi.shape)
    o = PcgOpts(int(kind), int(stop_mode), float(tol), int(max_inner), int(refresh), float(omega))
    res = PcgResult()
    lib().orc_pcg(A.H, A.W, A.indptr.ctypes.data_as(_L), A.indices.ctypes.data_as(_I),
                  _d(A.data), _d(bb), mp, ctypes.byref(o), _d(phi), ctypes.byref(res))
    return phi, {"iters": res.iters, "status": res.status, "relres": res.relres,
                 "true_relres": res.true_relres, "setup_s": res.setup_s}


def unwrap(psi, mask=None, p=1.0, tau=0.01, kind=M_JACOBI, tol=1e-6, max_outer=5,
           max_inner=0, outer_tol=0.0, stop_mode=STOP_RELRES, refresh=0, omega=1.0, phi0=None):
    """Algorithm 1: IRLS outer loop with the inner PCG; returns (phi, stats)."""
    psi = _f64(psi)
    H, W = psi.shape
    phi = np.zeros_like(psi) if phi0 is None else _f64(phi0).copy()
    m, mp = _mask(mask, psi.shape)
    o = PcgOpts(int(kind), int(stop_mode), float(tol), int(max_inner), int(refresh), float(omega))
    st = UnwrapStats()
    rc = lib().orc_unwrap(_d(psi), mp, H, W, float(p), float(tau), ctypes.byref(o),
                          int(max_outer), float(outer_tol), _d(phi), ctypes.byref(st))
    if rc == INVALID:
        raise ValueError("invalid arguments")
    k = st.outer
    stats = {"status": rc, "outer": k, "inner_total": st.inner_total,
             "inner": list(st.inner[:min(k, 64)]), "relres": list(st.relres[:min(k, 64)]),
             "outer_err": list(st.outer_err[:min(k, 64)]), "setup_s": st.setup_s}
    return phi, stats


def congruence(phi, psi):
    """Ghiglia-Pritt congruence post-step phi + W(psi - phi)."""
    phi, psi = _f64(phi), _f64(psi)
    out = np.empty_like(phi)
    lib().orc_congruence(_d(phi), _d(psi), phi.size, _d(out))
    return out


def quality_q(mu, nu):
    """Normalised error Q of Sec. 3."""
    mu, nu = _f64(mu), _f64(nu)
    return lib().orc_quality_q(_d(mu), _d(nu), mu.size)


def functional(phi, dx, dy, mask=None, p=1.0):
    """Eq. (funcional) with forward differences (monitoring only)."""
    phi, dx, dy = _f64(phi), _f64(dx), _f64(dy)
    H, W = phi.shape
    m, mp = _mask(mask, phi.shape)
    return lib().orc_functional(_d(phi), _d(dx), _d(dy), mp, H, W, float(p))
