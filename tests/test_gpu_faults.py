"""Failure paths of the solver, made on the host -- no GPU fault, trap or hang.

Every wait inside a kernel is bounded by options.spin_timeout_s (the grid
barriers of the persistent solvers and the band exchange of the wavefront
sweeps).  A bound of one nanosecond makes the first wait that spans a tick of
the GPU's timer give up: the kernel records the error, every other block sees
it at its next wait and leaves, and the call returns ULP_ERR_TIMEOUT.  The next
call with the default bound must then run normally and match the oracle, which
shows that the timed-out kernel left nothing behind (the barrier and the
exchange rows are reset at every launch).

Breakdown (Algorithm 1 divides by d^T q = d^T A d, which a symmetric positive
semi-definite A keeps non-negative): weights made negative on every edge give a
negative semi-definite A, so d^T A d <= 0 at the first step, and both the oracle
and the library stop with a breakdown status at iteration 0.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_13675_gb300 import native, synth

pytestmark = pytest.mark.gpu

KIND = {"identity": oracle.M_IDENTITY, "jacobi": oracle.M_JACOBI, "ilu0": oracle.M_ILU0, "mg": oracle.M_MG}


def _cuda(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _system(H, W, seed, sign=1.0):
    m = synth.phase_map(H, W, seed, noise=0.5)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, None, 1.0, 0.01)
    U, V = sign * U, sign * V
    return U, V, oracle.assemble(U, V, dx, dy)


def _rms(a, b):
    e = a - b
    e = e - e.mean()
    return float(np.sqrt(np.mean(e ** 2)))


@pytest.mark.parametrize("precond", ["jacobi", "ilu0"])
def test_bounded_wait_runs_out_then_the_next_call_is_clean(precond):
    H, W = 64, 64
    U, V, A = _system(H, W, 5)
    phi = torch.zeros((H, W), dtype=torch.float64, device="cuda")
    with pytest.raises(native.UlpError) as ei:
        native.ulp_pcg(_cuda(U), _cuda(V), _cuda(A.b), phi, precond=precond, tol=1e-8, spin_timeout_s=1e-9)
    assert ei.value.status == native.ULP_ERR_TIMEOUT, ei.value
    assert "wait ran out" in native.last_error()
    # the same solve with the default bound, in the same process and context
    phi = torch.zeros((H, W), dtype=torch.float64, device="cuda")
    _, st = native.ulp_pcg(_cuda(U), _cuda(V), _cuda(A.b), phi, precond=precond, tol=1e-8)
    ref, rst = oracle.pcg(A, np.zeros((H, W)), kind=KIND[precond], tol=1e-8)
    assert st["status"] == native.ULP_OK, st
    assert abs(st["inner"][0] - rst["iters"]) <= 2, (st, rst)
    assert _rms(phi.cpu().numpy(), ref) < 1e-6


def test_bounded_wait_runs_out_in_the_mixed_persistent_solver():
    """The mixed-precision persistent Jacobi PCG through a plan: a plan whose bound is
    one nanosecond reports ULP_ERR_TIMEOUT; a plan with the default bound, created and
    run right after, unwraps the same map like the oracle."""
    H, W = 64, 64
    m = synth.phase_map(H, W, 8, noise=0.4)
    psi = _cuda(m.psi)
    plan = native.Plan(H, W, outer_tol=0.0, precision=native.ULP_PRECISION_MIXED, spin_timeout_s=1e-9)
    with pytest.raises(native.UlpError) as ei:
        plan.unwrap(psi, None, p=1.0, precond="jacobi", tol=1e-6, max_outer=2)
    assert ei.value.status == native.ULP_ERR_TIMEOUT, ei.value
    plan.close()
    plan = native.Plan(H, W, outer_tol=0.0, precision=native.ULP_PRECISION_MIXED)
    phi, st = plan.unwrap(psi, None, p=1.0, precond="jacobi", tol=1e-6, max_outer=2)
    ref, rst = oracle.unwrap(m.psi, None, p=1.0, kind=oracle.M_JACOBI, tol=1e-6, max_outer=2)
    assert st["status"] == native.ULP_OK, st
    assert _rms(phi.cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("precond,precision", [("identity", native.ULP_PRECISION_FP64),
                                               ("jacobi", native.ULP_PRECISION_FP64),
                                               ("ilu0", native.ULP_PRECISION_FP64),
                                               ("mg", native.ULP_PRECISION_FP64),
                                               ("mg", native.ULP_PRECISION_MIXED)])
def test_indefinite_system_breaks_down_like_the_oracle(precond, precision):
    H, W = 48, 48
    U, V, A = _system(H, W, 3, sign=-1.0)
    _, rst = oracle.pcg(A, np.zeros((H, W)), kind=KIND[precond], tol=1e-8)
    assert rst["status"] == oracle.BREAKDOWN and rst["iters"] == 0, rst
    phi = torch.zeros((H, W), dtype=torch.float64, device="cuda")
    with pytest.raises(native.UlpError) as ei:
        native.ulp_pcg(_cuda(U), _cuda(V), _cuda(A.b), phi, precond=precond, tol=1e-8, precision=precision)
    assert ei.value.status == native.ULP_ERR_BREAKDOWN, ei.value
    assert "breakdown" in native.last_error()
    # nothing is left waiting: a positive-definite solve right after runs normally
    U2, V2, A2 = _system(H, W, 3)
    phi = torch.zeros((H, W), dtype=torch.float64, device="cuda")
    _, st = native.ulp_pcg(_cuda(U2), _cuda(V2), _cuda(A2.b), phi, precond=precond, tol=1e-8, precision=precision)
    assert st["status"] == native.ULP_OK, st


def test_noalloc_breakdown_sets_the_last_error():
    H, W = 48, 48
    U, V, A = _system(H, W, 3, sign=-1.0)
    phi = torch.zeros((H, W), dtype=torch.float64, device="cuda")
    with pytest.raises(native.UlpError) as ei:
        native.ulp_pcg_noalloc(_cuda(U), _cuda(V), _cuda(A.b), phi, precond="jacobi", tol=1e-8)
    assert ei.value.status == native.ULP_ERR_BREAKDOWN, ei.value
    assert "breakdown" in native.last_error()
