"""GB300 (sm_103a) L^p-norm phase unwrapping (arXiv 2203.13675).

The method (Algorithm 1 of the paper: IRLS reweighting around a preconditioned
conjugate-gradient solve of the weighted 5-point system) runs in hand-written
CUDA kernels behind the C ABI declared in include/unwrap_lp.h.  This package
holds the build step, the ctypes binding (``native``) and the seeded synthetic
input generator (``synth``).
"""
from . import synth  # noqa: F401

__all__ = ["synth", "native", "build"]
