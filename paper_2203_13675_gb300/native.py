"""Thin ctypes binding of libunwrap_lp.so (include/unwrap_lp.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Arrays are torch tensors (CUDA for device pointers, CPU for the
host-pointer form of ``unwrap_lp``); torch supplies memory and streams.
There is no CPU fallback: if the library is missing the import fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

PRECOND = {"identity": 0, "jacobi": 1, "ilu0": 2, "ic0": 3, "ssor": 4, "dct": 5, "learned": 6, "mg": 7, "rbssor": 8,
           "rbilu": 9}
ULP_OK, ULP_WARN_MAXITER = 0, 1
ULP_ERR_INVALID, ULP_ERR_CUDA, ULP_ERR_BREAKDOWN, ULP_ERR_TIMEOUT, ULP_ERR_NOMEM, ULP_ERR_UNSUPPORTED = \
    -1, -2, -3, -4, -5, -6
ULP_STOP_RELRES, ULP_STOP_PAPER = 0, 1
ULP_PRECISION_FP64, ULP_PRECISION_MIXED = 0, 1
ULP_PHI0_ZERO, ULP_PHI0_USER = 0, 1

EXPORTED = ["ulp_options_default", "ulp_last_error", "unwrap_lp", "ulp_plan_create",
            "ulp_plan_create_batched", "ulp_plan_destroy", "ulp_unwrap", "ulp_unwrap_batched",
            "ulp_plan_last_status", "ulp_wrapped_diffs", "ulp_weights", "ulp_matvec",
            "ulp_precond_apply", "ulp_pcg", "ulp_plan_counters", "ulp_pcg_noalloc",
            "ulp_autotune", "ulp_unet_param_count", "ulp_unet_create", "ulp_unet_destroy",
            "ulp_unet_set_params", "ulp_unet_get_params", "ulp_unet_save", "ulp_unet_load",
            "ulp_unet_apply", "ulp_unet_forward", "ulp_unet_loss_grad", "ulp_unet_train_step",
            "ulp_unet_harvest", "ulp_plan_set_unet"]


class UlpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"unwrap_lp status {status}: {msg}")
        self.status = status


class ulp_options(ctypes.Structure):
    _fields_ = [("stop_mode", ctypes.c_int), ("outer_tol", ctypes.c_double),
                ("refresh", ctypes.c_longlong), ("omega", ctypes.c_double),
                ("precision", ctypes.c_int), ("phi0_mode", ctypes.c_int),
                ("tile_rows", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("spin_timeout_s", ctypes.c_double), ("profile", ctypes.c_int), ("graph", ctypes.c_int),
                ("stall_window", ctypes.c_int)]


class ulp_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer", ctypes.c_int), ("inner_total", ctypes.c_longlong),
                ("inner", ctypes.c_longlong * 64), ("relres", ctypes.c_double * 64),
                ("outer_err", ctypes.c_double * 64), ("fallbacks", ctypes.c_int), ("setup_ms", ctypes.c_double)]

    def as_dict(self):
        k = min(self.outer, 64)
        return {"status": self.status, "outer": self.outer, "inner_total": self.inner_total,
                "inner": list(self.inner[:k]), "relres": list(self.relres[:k]),
                "outer_err": list(self.outer_err[:k]), "fallbacks": self.fallbacks, "setup_ms": self.setup_ms}


class ulp_counters(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("solver_launches", ctypes.c_longlong),
                ("solver_ms", ctypes.c_double), ("timed_launches", ctypes.c_longlong),
                ("phase_ms", ctypes.c_double * 6), ("phase_launches", ctypes.c_longlong * 6),
                ("graph_start_kernels", ctypes.c_longlong), ("graph_body_kernels", ctypes.c_longlong)]


class ulp_map(ctypes.Structure):
    _fields_ = [("psi", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("phi", ctypes.c_void_p),
                ("p", ctypes.c_double), ("eps", ctypes.c_double)]


_lib = None


def load(path: str | None = None):
    """Loads the library (built in-tree by paper_2203_13675_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    V, I, D, P = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    L.ulp_options_default.argtypes = [ctypes.POINTER(ulp_options)]
    L.ulp_options_default.restype = None
    L.ulp_last_error.restype = ctypes.c_char_p
    L.unwrap_lp.argtypes = [P, I, I, D, D, I, D, I, I, P]
    L.ulp_plan_create.argtypes = [I, I, ctypes.POINTER(ulp_options), ctypes.POINTER(V)]
    L.ulp_plan_create_batched.argtypes = [I, ctypes.POINTER(I), ctypes.POINTER(I),
                                          ctypes.POINTER(ulp_options), ctypes.POINTER(V)]
    L.ulp_plan_destroy.argtypes = [V]
    L.ulp_plan_destroy.restype = None
    L.ulp_unwrap.argtypes = [V, P, P, D, D, I, D, I, I, P, V, ctypes.POINTER(ulp_stats)]
    L.ulp_unwrap_batched.argtypes = [V, ctypes.POINTER(ulp_map), I, D, I, I, V, ctypes.POINTER(ulp_stats)]
    L.ulp_plan_last_status.argtypes = [V, ctypes.POINTER(ulp_stats)]
    L.ulp_plan_counters.argtypes = [V, I, ctypes.POINTER(ulp_counters)]
    L.ulp_wrapped_diffs.argtypes = [P, I, I, P, P, V]
    L.ulp_weights.argtypes = [P, P, P, P, I, I, D, D, P, P, P, V]
    L.ulp_matvec.argtypes = [P, P, P, I, I, P, V]
    L.ulp_precond_apply.argtypes = [I, P, P, P, I, I, D, P, P, V]
    L.ulp_pcg.argtypes = [P, P, P, I, I, I, D, I, ctypes.POINTER(ulp_options), P, V,
                          ctypes.POINTER(ulp_stats)]
    L.ulp_pcg_noalloc.argtypes = [P, P, P, I, I, I, D, I, P, V, ctypes.POINTER(ulp_stats)]
    L.ulp_autotune.argtypes = [I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ulp_map), I, I, I,
                               ctypes.c_char_p, ctypes.POINTER(ulp_options)]
    LL = ctypes.c_ulonglong
    L.ulp_unet_param_count.argtypes = []
    L.ulp_unet_create.argtypes = [LL, ctypes.POINTER(V)]
    L.ulp_unet_destroy.argtypes = [V]
    L.ulp_unet_destroy.restype = None
    L.ulp_unet_set_params.argtypes = [V, P]
    L.ulp_unet_get_params.argtypes = [V, P]
    L.ulp_unet_save.argtypes = [V, ctypes.c_char_p]
    L.ulp_unet_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(V)]
    L.ulp_unet_apply.argtypes = [V, P, P, P, P, I, I, P, V]
    L.ulp_unet_forward.argtypes = [V, I, I, I, P, P, P, P, V]
    L.ulp_unet_loss_grad.argtypes = [V, I, I, I, P, P, P, P, ctypes.POINTER(D), P, V]
    L.ulp_unet_train_step.argtypes = [V, I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(I), I, I,
                                      P, P, P, P, ctypes.c_float, ctypes.POINTER(D), V]
    L.ulp_unet_harvest.argtypes = [P, P, P, I, I, I, D, I, ctypes.POINTER(I), P, P, V]
    L.ulp_plan_set_unet.argtypes = [V, V]
    _lib = L
    return L


def last_error() -> str:
    return load().ulp_last_error().decode()


def _check(rc):
    if rc < 0:
        raise UlpError(rc, last_error())
    return rc


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype=torch.float64):
    assert t.is_cuda and t.dtype == dtype and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _precond(p):
    return PRECOND[p] if isinstance(p, str) else int(p)


def ulp_options_default(**overrides) -> ulp_options:
    o = ulp_options()
    load().ulp_options_default(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def unwrap_lp(psi, p=1.0, eps=1e-2, precond="jacobi", tol=1e-6, max_outer=5, max_inner=0, phi=None):
    """unwrap_lp(): whole method, host (CPU tensor) or device (CUDA tensor) buffers."""
    H, W = psi.shape
    assert psi.dtype == torch.float64 and psi.is_contiguous()
    if phi is None:
        phi = torch.empty_like(psi)
    rc = load().unwrap_lp(_ptr(psi), H, W, float(p), float(eps), _precond(precond), float(tol),
                          int(max_outer), int(max_inner), _ptr(phi))
    _check(rc)
    return phi, rc


class Plan:
    """Owns a ulp_plan (device workspace for one size or one batch of sizes)."""

    def __init__(self, H, W=None, options: ulp_options | None = None, sizes=None, **opt):
        L = load()
        self._h = ctypes.c_void_p()
        o = options or ulp_options_default(**opt)
        if sizes is not None:
            n = len(sizes)
            Ha = (ctypes.c_int * n)(*[s[0] for s in sizes])
            Wa = (ctypes.c_int * n)(*[s[1] for s in sizes])
            _check(L.ulp_plan_create_batched(n, Ha, Wa, ctypes.byref(o), ctypes.byref(self._h)))
            self.sizes = list(sizes)
        else:
            _check(L.ulp_plan_create(int(H), int(W), ctypes.byref(o), ctypes.byref(self._h)))
            self.sizes = [(H, W)]
        self.options = o

    def close(self):
        if self._h:
            load().ulp_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def unwrap(self, psi, mask=None, p=1.0, eps=1e-2, precond="jacobi", tol=1e-6, max_outer=5,
               max_inner=0, phi=None, stream=None, stats=True):
        """ulp_unwrap(): returns (phi, stats dict or None)."""
        _dev(psi)
        if mask is not None:
            _dev(mask, torch.uint8)
        if phi is None:
            phi = torch.empty_like(psi)
        st = ulp_stats() if stats else None
        rc = load().ulp_unwrap(self._h, _ptr(psi), _ptr(mask), float(p), float(eps), _precond(precond),
                               float(tol), int(max_outer), int(max_inner), _ptr(phi), _stream(stream),
                               ctypes.byref(st) if st is not None else None)
        _check(rc)
        return phi, (st.as_dict() if st is not None else None)

    def unwrap_batched(self, maps, precond="jacobi", tol=1e-6, max_outer=5, max_inner=0, stream=None,
                       stats=True):
        """ulp_unwrap_batched(): maps = list of dicts with psi, mask, phi, p, eps (CUDA tensors)."""
        n = len(maps)
        arr = (ulp_map * n)()
        for t, m in enumerate(maps):
            arr[t].psi = m["psi"].data_ptr()
            arr[t].mask = m["mask"].data_ptr() if m.get("mask") is not None else None
            arr[t].phi = m["phi"].data_ptr()
            arr[t].p = float(m["p"])
            arr[t].eps = float(m.get("eps", 1e-2))
        st = (ulp_stats * n)() if stats else None
        rc = load().ulp_unwrap_batched(self._h, arr, _precond(precond), float(tol), int(max_outer),
                                       int(max_inner), _stream(stream), st)
        _check(rc)
        return rc, ([s.as_dict() for s in st] if st is not None else None)

    def set_unet(self, net):
        """ulp_plan_set_unet(): the network used by precond="learned" (None detaches)."""
        _check(load().ulp_plan_set_unet(self._h, net._h if net is not None else None))
        self._unet = net  # keep it alive while the plan may use it

    def counters(self, reset=False):
        """ulp_plan_counters(): kernel launches, solver launches, (profile=1) solver ms and
        (profile=2, flexible CG) per-phase ms and counts keyed A, B, R, M, D, U."""
        c = ulp_counters()
        _check(load().ulp_plan_counters(self._h, int(bool(reset)), ctypes.byref(c)))
        names = ("A", "B", "R", "M", "D", "U")
        return {"kernel_launches": c.kernel_launches, "solver_launches": c.solver_launches,
                "solver_ms": c.solver_ms, "timed_launches": c.timed_launches,
                "phase_ms": {n: c.phase_ms[k] for k, n in enumerate(names)},
                "phase_launches": {n: c.phase_launches[k] for k, n in enumerate(names)},
                "graph_start_kernels": c.graph_start_kernels, "graph_body_kernels": c.graph_body_kernels}

    def last_status(self):
        """ulp_plan_last_status(): (worst status over the maps, stats of the first map)."""
        st = ulp_stats()
        rc = load().ulp_plan_last_status(self._h, ctypes.byref(st))
        return rc, st.as_dict()


def _map_array(maps):
    arr = (ulp_map * len(maps))()
    for t, m in enumerate(maps):
        arr[t].psi = m["psi"].data_ptr()
        arr[t].mask = m["mask"].data_ptr() if m.get("mask") is not None else None
        arr[t].phi = m["phi"].data_ptr()
        arr[t].p = float(m["p"])
        arr[t].eps = float(m.get("eps", 1e-2))
    return arr


def ulp_autotune(maps, precond="jacobi", precision=ULP_PRECISION_FP64, iters=40, cache_path=None):
    """ulp_autotune(): fastest tile_rows / blocks_per_sm for these maps (returns ulp_options)."""
    n = len(maps)
    Ha = (ctypes.c_int * n)(*[m["psi"].shape[0] for m in maps])
    Wa = (ctypes.c_int * n)(*[m["psi"].shape[1] for m in maps])
    best = ulp_options()
    _check(load().ulp_autotune(n, Ha, Wa, _map_array(maps), _precond(precond), int(precision), int(iters),
                               cache_path.encode() if cache_path else None, ctypes.byref(best)))
    return best


def ulp_wrapped_diffs(psi, stream=None):
    H, W = psi.shape
    _dev(psi)
    dx = torch.empty_like(psi)
    dy = torch.empty_like(psi)
    _check(load().ulp_wrapped_diffs(_ptr(psi), H, W, _ptr(dx), _ptr(dy), _stream(stream)))
    return dx, dy


def ulp_weights(phi, dx, dy, mask=None, p=1.0, eps=1e-2, stream=None, U=None, V=None, b=None):
    """U, V, b: optional contiguous output tensors (views into larger buffers allowed)."""
    H, W = phi.shape
    U = torch.empty_like(phi) if U is None else _dev(U)
    V = torch.empty_like(phi) if V is None else _dev(V)
    b = torch.empty_like(phi) if b is None else _dev(b)
    _check(load().ulp_weights(_ptr(_dev(phi)), _ptr(_dev(dx)), _ptr(_dev(dy)),
                              _ptr(mask), H, W, float(p), float(eps), _ptr(U), _ptr(V), _ptr(b),
                              _stream(stream)))
    return U, V, b


def ulp_matvec(U, V, x, stream=None):
    H, W = x.shape
    y = torch.empty_like(x)
    _check(load().ulp_matvec(_ptr(_dev(U)), _ptr(_dev(V)), _ptr(_dev(x)), H, W, _ptr(y), _stream(stream)))
    return y


def ulp_precond_apply(precond, U, V, r, mask=None, omega=1.0, stream=None):
    H, W = r.shape
    s = torch.empty_like(r)
    _check(load().ulp_precond_apply(_precond(precond), _ptr(_dev(U)), _ptr(_dev(V)), _ptr(mask), H, W,
                                    float(omega), _ptr(_dev(r)), _ptr(s), _stream(stream)))
    return s


def ulp_pcg(U, V, b, phi, precond="jacobi", tol=1e-6, max_inner=0, stream=None, **opt):
    H, W = b.shape
    o = ulp_options_default(**opt)
    st = ulp_stats()
    rc = load().ulp_pcg(_ptr(_dev(U)), _ptr(_dev(V)), _ptr(_dev(b)), H, W, _precond(precond), float(tol),
                        int(max_inner), ctypes.byref(o), _ptr(_dev(phi)), _stream(stream), ctypes.byref(st))
    _check(rc)
    return phi, st.as_dict()


def ulp_pcg_noalloc(U, V, b, phi, precond="jacobi", tol=1e-6, max_inner=0, stream=None):
    """ulp_pcg_noalloc(): ulp_pcg without any device allocation (static workspace)."""
    H, W = b.shape
    st = ulp_stats()
    rc = load().ulp_pcg_noalloc(_ptr(_dev(U)), _ptr(_dev(V)), _ptr(_dev(b)), H, W, _precond(precond),
                                float(tol), int(max_inner), _ptr(_dev(phi)), _stream(stream), ctypes.byref(st))
    _check(rc)
    return phi, st.as_dict()


# ---------------------------------------------------------------- learned preconditioner
class Unet:
    """Owns a ulp_unet (the learned preconditioner's parameters and workspace)."""

    def __init__(self, seed=0, path=None):
        L = load()
        h = ctypes.c_void_p()
        if path is not None:
            _check(L.ulp_unet_load(os.fsencode(path), ctypes.byref(h)))
        else:
            _check(L.ulp_unet_create(int(seed), ctypes.byref(h)))
        self._h = h

    @staticmethod
    def param_count() -> int:
        return load().ulp_unet_param_count()

    def close(self):
        if getattr(self, "_h", None):
            load().ulp_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        """params: host float32 array-like of param_count() values (canonical order)."""
        t = torch.as_tensor(params, dtype=torch.float32).contiguous().cpu()
        assert t.numel() == self.param_count()
        _check(load().ulp_unet_set_params(self._h, ctypes.c_void_p(t.data_ptr())))

    def get_params(self):
        t = torch.empty(self.param_count(), dtype=torch.float32)
        _check(load().ulp_unet_get_params(self._h, ctypes.c_void_p(t.data_ptr())))
        return t

    def save(self, path):
        _check(load().ulp_unet_save(self._h, os.fsencode(path)))

    def apply(self, r, U, V, mask=None, s=None, stream=None):
        H, W = r.shape
        if s is None:
            s = torch.empty_like(r)
        _check(load().ulp_unet_apply(self._h, _ptr(_dev(r)), _ptr(_dev(U)), _ptr(_dev(V)),
                                     _ptr(mask) if mask is not None else None, H, W, _ptr(_dev(s)),
                                     _stream(stream)))
        return s

    def forward(self, r, U, V, stream=None):
        B, H, W = r.shape
        y = torch.empty((B, H, W), dtype=torch.float32, device=r.device)
        _check(load().ulp_unet_forward(self._h, B, H, W, _ptr(_dev(r)), _ptr(_dev(U)), _ptr(_dev(V)),
                                       _ptr(y), _stream(stream)))
        return y

    def loss_grad(self, r, U, V, e, stream=None):
        B, H, W = r.shape
        g = torch.empty(self.param_count(), dtype=torch.float32, device=r.device)
        loss = ctypes.c_double()
        _check(load().ulp_unet_loss_grad(self._h, B, H, W, _ptr(_dev(r)), _ptr(_dev(U)), _ptr(_dev(V)),
                                         _ptr(_dev(e)), ctypes.byref(loss), _ptr(g), _stream(stream)))
        return loss.value, g

    def train_step(self, pair_idx, sys_idx, r, e, U, V, lr=1e-3, stream=None, want_loss=True):
        """One Adam step on pairs r[pair_idx] -> e[pair_idx] with weights U[sys_idx], V[sys_idx];
        returns the batch loss (which synchronises), or None with want_loss=False."""
        _, H, W = r.shape
        B = len(pair_idx)
        pi = (ctypes.c_longlong * B)(*[int(x) for x in pair_idx])
        si = (ctypes.c_int * B)(*[int(x) for x in sys_idx])
        loss = ctypes.c_double()
        _check(load().ulp_unet_train_step(self._h, B, pi, si, H, W, _ptr(_dev(r)), _ptr(_dev(e)),
                                          _ptr(_dev(U)), _ptr(_dev(V)), float(lr),
                                          ctypes.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None


def ulp_unet_harvest(U, V, b, iters, precond="jacobi", tol_star=1e-10, r_out=None, e_out=None, stream=None):
    """Training pairs (b - A phi_l, phi* - phi_l) for PCG iterates phi_l after iters[k] iterations."""
    H, W = b.shape
    n = len(iters)
    if r_out is None:
        r_out = torch.empty((n, H, W), dtype=torch.float64, device=b.device)
    if e_out is None:
        e_out = torch.empty((n, H, W), dtype=torch.float64, device=b.device)
    it = (ctypes.c_int * n)(*[int(x) for x in iters])
    _check(load().ulp_unet_harvest(_ptr(_dev(U)), _ptr(_dev(V)), _ptr(_dev(b)), H, W, _precond(precond),
                                   float(tol_star), n, it, _ptr(_dev(r_out)), _ptr(_dev(e_out)),
                                   _stream(stream)))
    return r_out, e_out
