"""The outer loop of Algorithm 1 under a large k_max.

Every pass decides on the device whether it runs; a pass after the outer stop does
nothing.  With more than 8 passes the call looks, after every 8, whether any map is
still in its outer loop and enqueues no further pass once none is.  These tests check
that this changes nothing in the result: a call under the paper's k_max = 500 (Sec. 3)
returns the same phase, bit for bit, and the same statistics as the same call with
k_max equal to the passes it ran; and a call whose outer loop never stops runs all of
its passes.
"""
import pytest
import torch

from paper_2203_13675_gb300 import experiment_table1 as t1
from paper_2203_13675_gb300 import native

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precond", ["mg", "jacobi"])
def test_paper_k_max_gives_the_result_of_the_passes_it_ran(precond):
    cols, rows = 320, 240
    m = t1.make_map(cols, rows)
    psi = torch.from_numpy(m.psi).cuda()
    plan = native.Plan(rows, cols, outer_tol=1e-6, stop_mode=native.ULP_STOP_PAPER)
    phi_a, st_a = plan.unwrap(psi, None, p=1.0, precond=precond, tol=0.005, max_outer=500, max_inner=0)
    n = st_a["outer"]
    assert st_a["status"] == 0, st_a
    assert 1 <= n < 8, st_a  # the outer loop stops within the first look
    phi_b, st_b = plan.unwrap(psi, None, p=1.0, precond=precond, tol=0.005, max_outer=n, max_inner=0)
    assert st_b["outer"] == n, (st_a, st_b)
    assert st_b["inner"] == st_a["inner"], (st_a["inner"], st_b["inner"])
    assert torch.equal(phi_a, phi_b)
    plan.close()


def test_outer_loop_that_never_stops_runs_every_pass():
    """At 160x120 the paper's criteria never meet the outer tolerance (all 500 passes run,
    for every preconditioner): 20 passes, past two looks of the host, all run."""
    cols, rows = 160, 120
    m = t1.make_map(cols, rows)
    psi = torch.from_numpy(m.psi).cuda()
    plan = native.Plan(rows, cols, outer_tol=1e-6, stop_mode=native.ULP_STOP_PAPER)
    _, st = plan.unwrap(psi, None, p=1.0, precond="mg", tol=0.005, max_outer=20, max_inner=0)
    assert st["status"] == 0, st
    assert st["outer"] == 20, st
    plan.close()
