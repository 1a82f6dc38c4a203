"""The point the GPU solve returns, checked by the oracle's independent functions.

E_0 (Wachter & Biegler 2006, Eq. (5) at mu = 0, with the s_max = 100 scaling) is
recomputed by oracle/checks.kkt_error from the GPU's primal point x, row multipliers y
and bound multipliers z_L, z_U (all of the unscaled problem min d), with the constraint
Jacobian by complex step -- nothing of the GPU's own residuals or reductions enters it.
Bound: E_0 <= 1e-8, the paper's solver tolerance.

The 500-scenario workload (uniform +-10 % feeds, seed 1) is also compared with the
oracle's own solve, stored by tests/golden/make_c1_golden.py (which calls only
oracle/): d* to 1e-6 relative, the sampled scenarios' stage states to 1e-5 (scaled by
max(1, |z|)), the same number of iterations up to 3."""
import json
import math
import os

import numpy as np
import pytest

import absorber_inputs as ai
from oracle import checks, model

pytestmark = pytest.mark.gpu
P = ai.PARAMS
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_s500_seed1.json")


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


def _solve_and_point(B, F, opt, learned_net=None):
    """Solve on the GPU; return the result and the returned KKT point as host arrays
    (Z, d, lambda, z_L, z_U, z_L(d), z_U(d))."""
    import torch
    prob = B.Problem(P, F)
    x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    y = torch.zeros(prob.n_row, dtype=torch.float64, device="cuda")
    if learned_net is None:
        res = prob.ipm_solve(opt, x_out=x, y_out=y)
    else:
        res = B.ipm_solve_learned(prob, learned_net, opt, x_out=x, y_out=y)
    zl = torch.zeros_like(x)
    zu = torch.zeros_like(x)
    zd = prob.bound_multipliers(zl, zu)
    Z, d = prob.from_soa(host(x))
    lam, _ = prob.from_soa(host(y))
    ZL, zld = prob.from_soa(host(zl))
    ZU, zud = prob.from_soa(host(zu))
    assert zld == zd[0] and zud == zd[1]
    return prob, res, (Z, d, lam, ZL, ZU, zld, zud)


def _kkt(F, pt, chunk=None):
    Z, d, lam, ZL, ZU, zld, zud = pt
    return checks.kkt_error(P, F, d, Z, lam, ZL, ZU, zld, zud, chunk=chunk)


def test_kkt_error_recomputed_s10(B):
    F = ai.make_feeds(10, 0)
    prob, res, pt = _solve_and_point(B, F, B.default_options())
    assert res.status == 0 and res.E0 <= 1e-8
    E0 = _kkt(F, pt)
    assert E0 <= 1e-8, E0
    # the bound multipliers are those of the bounds that exist, complementary at the point
    lo, hi, dlo, dhi = model.bounds(P, 10)
    Z, d, lam, ZL, ZU, zld, zud = pt
    assert np.all(ZL[~np.isfinite(lo)] == 0.0) and np.all(ZU[~np.isfinite(hi)] == 0.0)
    assert np.all(ZL[np.isfinite(lo)] > 0.0) and np.all(ZU[np.isfinite(hi)] > 0.0)
    assert zld > 0.0 and zud > 0.0


def test_kkt_error_recomputed_s10_mixed_precision(B):
    F = ai.make_feeds(10, 0)
    prob, res, pt = _solve_and_point(B, F, B.default_options(precision=1, max_refine=8))
    assert res.status == 0
    assert _kkt(F, pt) <= 1e-8


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_s500_fp64_matches_stored_oracle_solve(B, golden):
    F = ai.make_feeds(golden["S"], golden["seed"], dist=golden["dist"])
    prob, res, pt = _solve_and_point(B, F, B.default_options())
    assert res.status == 0 and res.E0 <= 1e-8
    assert abs(res.d - golden["d"]) <= 1e-6 * golden["d"], (res.d, golden["d"])
    Z = pt[0]
    for s in golden["sample"]:
        zo = np.asarray(golden["Z"][str(s)])
        assert np.max(np.abs(Z[s] - zo) / np.maximum(1.0, np.abs(zo))) <= 1e-5, s
    assert abs(res.iters - golden["iters"]) <= 3, (res.iters, golden["iters"])
    # one active hydraulic row carries the objective: sum of the hydraulic multipliers
    lam = pt[2]
    lh = lam.reshape(golden["S"], model.N, model.NV)[:, :, model.NV - 1].sum()
    assert abs(lh - golden["lam_hydraulic_sum"]) <= 1e-6 * abs(golden["lam_hydraulic_sum"])
    assert _kkt(F, pt, chunk=100) <= 1e-8


def test_kkt_error_recomputed_full_size_s5000_mixed(B):
    # the 5000-scenario workload with FP32 factors + FP64 refinement from the default
    # start: E_0 of the returned point from the definitions
    F = ai.workload_feeds("absorber-S5000-tn5-seed2")
    prob, res, pt = _solve_and_point(B, F, B.default_options(precision=1, max_refine=8))
    assert res.status == 0 and res.E0 <= 1e-8
    E0 = _kkt(F, pt, chunk=250)
    assert E0 <= 1e-8, E0
    dmin, _ = checks.minimum_diameter(P, F, pt[0])
    assert abs(pt[1] - dmin) <= 1e-8 * dmin
    # stationarity in d: u_max pi d / 2 * (sum of hydraulic multipliers) = 1 + z_U - z_L
    lam = pt[2]
    lh = lam.reshape(5000, model.N, model.NV)[:, :, model.NV - 1].sum()
    assert abs(P["u_max"] * math.pi * pt[1] / 2.0 * lh - (1.0 - pt[5] + pt[6])) <= 1e-6


def test_bound_multipliers_need_a_solve(B):
    import torch
    F = ai.make_feeds(3, 0)
    prob = B.Problem(P, F)
    z = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    with pytest.raises(B.AbsorberError) as e:
        prob.bound_multipliers(z, z.clone())
    assert e.value.status == -1


def test_injected_inertia_failure(B):
    # Algorithm IC cannot succeed when delta_w_max is below the first trial delta_w and the
    # Schur scalar is negative: a warm start whose row multipliers are scaled far up makes
    # the Lagrangian Hessian strongly indefinite (S_d is linear in lambda for large lambda,
    # so one of the two signs makes it negative); the solve stops with ABS_ERR_INERTIA
    import torch
    F = ai.make_feeds(4, 0)
    prob = B.Problem(P, F)
    x0 = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    prob.ipm_solve(B.default_options(max_iter=0), x_out=x0)     # the default start
    rng = np.random.default_rng(3)
    lam = rng.standard_normal((4, model.NS))
    statuses = []
    for sign in (1.0, -1.0):
        y = torch.from_numpy(prob.to_soa(sign * 1e8 * lam)).cuda()
        r = prob.ipm_solve(B.default_options(dw_max=1e-30), warm_x=x0, warm_y=y)
        statuses.append(r.status)
        if r.status == -4:
            assert r.iters == 0
    assert -4 in statuses, statuses


def test_injected_linesearch_failure(B):
    # from the inlet-copy start of this one-scenario problem the first full trial step of
    # iteration 0 is rejected (the oracle backtracks there too); with one trial allowed, no
    # second-order correction and no restoration the line search fails: ABS_ERR_LINESEARCH
    F = ai.make_feeds(1, 0)
    prob = B.Problem(P, F)
    r = prob.ipm_solve(B.default_options(init=1, max_ls=1, soc_max=0, resto_max=0))
    assert r.status == -5 and r.iters == 0 and r.resto_phases == 0, (r.status, r.iters)
    # with feasibility restoration the same crippled line search still reaches the optimum
    rr = prob.ipm_solve(B.default_options(init=1, max_ls=1, soc_max=0))
    ok = prob.ipm_solve(B.default_options(init=1))
    assert ok.status == 0
    assert rr.status == 0 and rr.resto_phases >= 1 and abs(rr.d - ok.d) <= 1e-6 * ok.d
