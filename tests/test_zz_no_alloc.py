"""ulp_pcg_noalloc: the allocation-free inner solve, checked against ulp_pcg.

Callers whose device memory is owned by another allocator, or whose loop
cannot afford cudaMalloc/cudaFree, use ulp_pcg_noalloc (static workspace in
the library) instead of ulp_pcg (temporary workspace per call).  Both must
give the same solve: iteration counts within +-2 and the solution within
1e-8 rad RMS after removing the mean, the tolerances of the FP64 PCG parity
tests.  Two calls in a row exercise a workspace that still holds the previous
call's contents.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_13675_gb300 import native, synth

pytestmark = pytest.mark.gpu


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _system(H, W, seed, p):
    m = synth.phase_map(H, W, seed, noise=0.7, mask_frac=0.05, ramp=0.1)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, m.mask, p, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    return _cuda(U), _cuda(V), _cuda(A.b)


def _rms(a, b):
    e = (a - b).double().cpu().numpy()
    e = e - e.mean()
    return float(np.sqrt(np.mean(e ** 2)))


@pytest.mark.parametrize("kind", ["jacobi", "identity"])
@pytest.mark.parametrize("H,W,p", [(200, 129, 0.5), (256, 256, 1.0)])
def test_noalloc_matches_existing_entry_point(kind, H, W, p):
    U, V, b = _system(H, W, 40 + H, p)
    U2, V2, b2 = _system(H, W, 90 + H, 0.0)  # a second, different system
    zeros = lambda: torch.zeros(H, W, dtype=torch.float64, device="cuda")  # noqa: E731
    ref1, st1 = native.ulp_pcg(U, V, b, zeros(), kind, 1e-6)
    ref2, st2 = native.ulp_pcg(U2, V2, b2, zeros(), kind, 1e-6)
    # two calls in a row on the shared static workspace, then a third with other inputs
    for _ in range(2):
        got, st = native.ulp_pcg_noalloc(U, V, b, zeros(), kind, 1e-6)
        assert st["status"] == 0
        assert abs(st["inner"][0] - st1["inner"][0]) <= 2, (st["inner"], st1["inner"])
        assert _rms(got, ref1) < 1e-8
    got, st = native.ulp_pcg_noalloc(U2, V2, b2, zeros(), kind, 1e-6)
    assert abs(st["inner"][0] - st2["inner"][0]) <= 2 and _rms(got, ref2) < 1e-8


def test_noalloc_rejects_oversize_grid():
    H, W = 257, 256
    t = torch.zeros(H, W, dtype=torch.float64, device="cuda")
    with pytest.raises(native.UlpError) as e:
        native.ulp_pcg_noalloc(t, t, t, t.clone(), "jacobi", 1e-6)
    assert e.value.status == native.ULP_ERR_INVALID and "65536" in str(e.value)
