"""Feasibility restoration on the GPU (Wachter & Biegler 2006, Section 3.3; for the square
constraint system of problem (10): damped Newton on c(z) = 0 with d fixed, until the
filter augmented with the failed iterate accepts a point with theta reduced by
1 - gamma_theta -- the oracle's IPM.restoration, pinned on the CPU).

The problems: single-scenario instances of the training distribution with the objective
unscaled (w = 1), solved from the inlet-copy start, where the line search of about one
in eight falls below alpha_min.  Which ones stall depends on rounding (the oracle's own
trajectories differ between machines there), so the GPU is checked by what fixes the
answer: a rescued problem converges (E_0 <= 1e-8) to the diameter that its states
determine (d* = max sqrt(4 V R T / (pi u P)), the oracle's check on the GPU's point), the
same as its w = 100 solve, and its batch result equals its solve alone.
"""
import numpy as np
import pytest

import absorber_inputs as ai
from oracle import checks

pytestmark = pytest.mark.gpu
P = ai.PARAMS


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_15420_gb300 import build
    build.build()
    from paper_2607_15420_gb300 import binding
    binding.lib()
    return binding


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def batch_runs(B):
    F = ai.make_feeds(400, 11, stream=3)
    feeds = [F[:, i:i + 1] for i in range(400)]
    batch = B.Batch(P, feeds)
    off = batch.ipm_solve(B.default_options(obj_scaling=1.0, init=1, resto_max=0))
    on = batch.ipm_solve(B.default_options(obj_scaling=1.0, init=1))
    return feeds, off, on


def test_restoration_rescues_stalled_line_searches(B, batch_runs):
    feeds, off, on = batch_runs
    fails_off = {i for i, r in enumerate(off) if r.status != 0}
    fails_on = {i for i, r in enumerate(on) if r.status != 0}
    assert all(off[i].status == -5 for i in fails_off)       # stalls are line-search failures
    assert all(r.resto_phases == 0 for r in off)
    assert fails_on < fails_off                                # some rescued, none lost
    rescued = sorted(fails_off - fails_on)
    for i in rescued:
        assert on[i].resto_phases >= 1 and on[i].E0 <= 1e-8
    # problems whose line search never failed take the same steps with restoration on
    for i in range(0, 400, 37):
        if i not in fails_off:
            assert on[i].iters == off[i].iters and on[i].d == off[i].d and on[i].resto_phases == 0


def test_rescued_problems_reach_the_optimum(B, batch_runs):
    import torch
    feeds, off, on = batch_runs
    rescued = sorted({i for i, r in enumerate(off) if r.status != 0} - {i for i, r in enumerate(on) if r.status != 0})
    assert rescued
    for i in rescued[:3]:
        F = feeds[i]
        prob = B.Problem(P, F)
        x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
        alone = prob.ipm_solve(B.default_options(obj_scaling=1.0, init=1), x_out=x)
        # the batch ran this problem exactly as alone
        assert alone.status == 0 and alone.iters == on[i].iters and alone.d == on[i].d
        Z, d = prob.from_soa(host(x))
        dmin, _ = checks.minimum_diameter(P, F, Z)
        assert abs(d - dmin) <= 1e-8 * dmin
        ref = prob.ipm_solve(B.default_options(obj_scaling=100.0, init=1))
        assert ref.status == 0 and abs(ref.d - d) <= 1e-6 * d
    # graph replay takes the same restoration steps as the eager run
    F = feeds[rescued[0]]
    prob = B.Problem(P, F)
    runs = [prob.ipm_solve(B.default_options(obj_scaling=1.0, init=1, graphs=g)) for g in (0, 1, 1, 1)]
    assert runs[-1].graph_replays == 1
    for r in runs[1:]:
        assert r.status == 0 and r.iters == runs[0].iters and r.d == runs[0].d and r.resto_phases == runs[0].resto_phases
