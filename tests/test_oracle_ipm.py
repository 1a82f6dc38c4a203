"""Oracle interior-point solve (oracle/ipm.py) pinned by what the problem fixes
independently of the solver: the KKT conditions recomputed from definitions, the
closed-form optimal diameter, conservation laws, the square MESH system, symmetry."""
import math

import numpy as np
import pytest

import absorber_inputs as ai
from oracle import checks, ipm, model

P = ai.PARAMS


@pytest.fixture(scope="module")
def s1():
    F = ai.make_feeds(1, 0)
    return F, ipm.solve(P, F)


@pytest.fixture(scope="module")
def s10():
    F = ai.make_feeds(10, 0)
    return F, ipm.solve(P, F)


def _check_solution(F, r):
    assert r.status == "ok"
    # E_0 <= 1e-8 recomputed from the definitions (complex-step Jacobian)
    assert checks.kkt_error(P, F, r.d, r.Z, r.lam, r.zL, r.zU, r.zLd, r.zUd) <= 1e-8
    # the optimal diameter is the smallest that satisfies every hydraulic row at the
    # (d-independent) MESH states: d* = max sqrt(4 V R T / (pi u P))
    dmin, vol = checks.minimum_diameter(P, F, r.Z)
    assert abs(r.d - dmin) <= 1e-8 * dmin
    # exactly one hydraulic row active (margin within tolerance of zero), the rest slack
    margin = P["u_max"] * math.pi * r.d ** 2 / 4 - vol
    assert margin.min() <= 1e-7 and np.sort(margin.ravel())[1] > 1e-4
    # conservation over the column: elements C, H, N, O and charge; enthalpy
    el_in, el_out, h_in, h_out = checks.column_balances(P, F, r.Z)
    np.testing.assert_allclose(el_out, el_in, rtol=0, atol=1e-8 * np.abs(el_in).max())
    np.testing.assert_allclose(h_out, h_in, rtol=0, atol=1e-7 * np.abs(h_in).max())
    # liquid electroneutral on every stage; compositions closed; fixed entries exactly 0
    assert np.abs(checks.liquid_charge(P, r.Z)).max() <= 1e-10
    full = model.full_layout(P, r.Z)
    np.testing.assert_allclose(full[:, :, 0:11].sum(-1), 1.0, atol=1e-8)
    np.testing.assert_allclose(full[:, :, 11:22].sum(-1), 1.0, atol=1e-8)
    assert np.all(full[:, :, 9:11] == 0.0) and np.all(full[:, :, 11:18] == 0.0)


def test_single_scenario_solution(s1):
    _check_solution(*s1)


def test_ten_scenario_solution(s10):
    _check_solution(*s10)


def test_mesh_square_system_newton(s1):
    F, r = s1
    Z, hist = checks.mesh_newton(P, F, r.Z, r.d)
    assert hist[-1] <= 1e-13
    # quadratic convergence once in the basin: r_{k+1} <= C r_k^2
    for a, b in zip(hist[:-1], hist[1:]):
        if a < 1e-6 and b > 1e-12:
            assert b <= 1e3 * a * a
    # the IPM's states are that root (to within the primal tolerance's reach)
    keep = np.ones(model.NS, dtype=bool)
    keep[model.NV - 1::model.NV] = False
    scale = np.maximum(1.0, np.abs(Z[:, keep]))
    assert np.abs(Z[:, keep] - r.Z[:, keep]).max() / scale.max() <= 1e-6
    dmin, _ = checks.minimum_diameter(P, F, Z)
    assert abs(dmin - r.d) <= 1e-8 * r.d


def test_identical_scenarios_reproduce_single(s1):
    F1, r1 = s1
    S = 3
    F = np.repeat(F1, S, axis=1)
    r = ipm.solve(P, F)
    assert r.status == "ok"
    assert abs(r.d - r1.d) <= 1e-8 * r1.d     # both within the 1e-8 KKT tolerance
    for s in range(S):
        assert np.abs(r.Z[s] - r1.Z[0]).max() <= 1e-6 * np.abs(r1.Z[0]).max()
    hyd = np.arange(model.NV - 1, model.NS, model.NV)
    lh = r.lam[:, hyd]
    np.testing.assert_allclose(lh, np.broadcast_to(lh[0:1], lh.shape), rtol=1e-6, atol=1e-8 * np.abs(lh).max())  # symmetric split
    # the active row's multiplier is split evenly: sum over copies = the single value;
    # inactive rows carry only O(mu) multipliers
    a = int(np.argmax(r1.lam[0, hyd]))
    assert abs(lh[:, a].sum() - r1.lam[0, hyd][a]) <= 1e-5 * r1.lam[0, hyd][a]
    assert np.delete(lh, a, axis=1).max() <= 1e-6


def test_bruteforce_diameter_sweep(s10):
    F, r = s10
    Z, hist = checks.mesh_newton(P, F, r.Z, r.d, iters=4)
    _, vol = checks.minimum_diameter(P, F, Z)
    grid = np.linspace(1.0, 2.0, 201)
    feas = np.array([np.all(P["u_max"] * math.pi * g ** 2 / 4 - vol >= 0) for g in grid])
    # feasibility is monotone in d ...
    first = np.argmax(feas)
    assert feas[first:].all() and not feas[:first].any()
    # ... and the smallest feasible grid point brackets the optimum
    assert grid[first - 1] < r.d <= grid[first]


def test_feasibility_restoration_rescues_a_stalled_line_search():
    # single-scenario problems of the training distribution with the objective unscaled
    # (w = 1) from the inlet-copy start: on this one the line search falls below alpha_min
    # after 21 iterations; restoration (Newton on the square constraint system, d fixed)
    # returns a point the filter accepts and the solve converges to the optimum that the
    # definitions fix
    F = ai.make_feeds(40, 7, stream=3)[:, 32:33]
    r0 = ipm.solve(P, F, ipm.Options(obj_scaling=1.0, init="inlet", resto_max=0))
    assert r0.status == "linesearch"
    r = ipm.solve(P, F, ipm.Options(obj_scaling=1.0, init="inlet"))
    assert sum(1 for h in r.history if h.get("resto")) >= 1
    _check_solution(F, r)
    # the restored point reduced the infeasibility of the failed iterate
    k = next(i for i, h in enumerate(r.history) if h.get("resto"))
    assert r.history[k + 1]["theta"] <= (1 - 1e-5) * r.history[k]["theta"]
    # the optimum does not depend on the objective's scaling: w = 100 reaches it directly
    rs = ipm.solve(P, F, ipm.Options(obj_scaling=100.0, init="inlet"))
    assert rs.status == "ok" and abs(rs.d - r.d) <= 1e-7 * r.d


def test_restoration_reduces_theta_inside_the_bounds():
    # the restoration phase itself, from the failed iterate of the case above: the point
    # it returns has a smaller ||c||_1 by the required factor and stays inside the bounds
    F = ai.make_feeds(40, 7, stream=3)[:, 32:33]
    solver = ipm.IPM(P, F, ipm.Options(obj_scaling=1.0, init="inlet", resto_max=0, max_iter=21))
    r = solver.solve()
    st = solver.state_from_result(r)
    th0 = float(np.abs(model.residuals(P, F, st.Z, st.d)).sum())
    Zr = ipm.IPM(P, F, ipm.Options(obj_scaling=1.0, init="inlet")).restoration(st, r.mu, max(0.99, 1 - r.mu), [],
                                                                               th0)
    assert Zr is not None
    thr = float(np.abs(model.residuals(P, F, Zr, st.d)).sum())
    assert thr <= (1 - 1e-5) * th0
    lo, hi, _, _ = model.bounds(P, 1)
    assert np.all(Zr[np.isfinite(lo)] > lo[np.isfinite(lo)]) and np.all(Zr[np.isfinite(hi)] < hi[np.isfinite(hi)])
