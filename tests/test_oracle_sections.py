"""Oracle pins for a design vector with more than one entry (the general Eq. (8), dim
theta > 1): the column split into K sections of consecutive stages, each with its own
diameter, the objective the stage-weighted sum of the diameters.

What fixes the answer: every scenario's MESH block is square (Section "Degrees of
freedom"), so the stage states at the optimum do not depend on the diameters and each
section's diameter is the smallest that satisfies its own stages' hydraulic rows,
theta_k* = max over scenarios and the section's stages of sqrt(4 V R T / (pi u_max P))
(checks.section_diameters); the largest of them is the one-section optimum d*.  Also:
the K-entry border and Hessian against complex step and the hydraulic rows' closed form,
the K x K Schur solve against the monolithic LDL^T, its inertia against eigenvalue
signs, E_0 from the definitions at the returned point."""
import math

import numpy as np
import pytest

import absorber_inputs as ai
from oracle import checks, ipm, kkt, model

P1 = ai.PARAMS
P2 = dict(ai.PARAMS, n_sections=2)


def test_section_layout():
    assert list(model.stage_sections(1)) == [0] * 10
    assert list(model.stage_sections(2)) == [0] * 5 + [1] * 5
    assert list(model.stage_sections(3)) == [0, 0, 0, 0, 1, 1, 1, 2, 2, 2]
    for K in (1, 2, 3):
        w = model.section_weights(K)
        assert abs(w.sum() - 1.0) <= 1e-15 and np.all(w > 0)


def _iterate(P, S, seed, iters):
    F = ai.make_feeds(S, seed)
    solver = ipm.IPM(P, F, ipm.Options(max_iter=iters))
    r = solver.solve()
    st = solver.state_from_result(r)
    return F, solver, st


def test_border_and_hessian_of_the_sections():
    F, solver, st = _iterate(P2, 2, 0, 2)
    d = np.atleast_1d(st.d)
    assert d.shape == (2,)
    C, J, Jd, W, Wdd = model.derivatives(P2, F, st.Z, d, st.lam)
    assert Jd.shape == (2, model.NS, 2) and Wdd.shape == (2, 2)
    Jc, Jdc = checks.jacobian_complex_step(P2, F, st.Z, d)
    assert np.max(np.abs(Jd - Jdc)) <= 1e-12 * np.max(np.abs(Jdc))
    sec = model.stage_sections(2)
    rows_h = model.NR * np.arange(model.N) + model.NR - 1
    for k in range(2):
        # dc/dtheta_k: -u_max pi theta_k / 2 in the hydraulic rows of section k, 0 elsewhere
        expect = np.zeros((2, model.NS))
        expect[:, rows_h[sec == k]] = -P2["u_max"] * math.pi * d[k] / 2.0
        assert np.max(np.abs(Jd[:, :, k] - expect)) <= 1e-14 * abs(expect).max()
        # d2 (lam^T c)/dtheta_k^2 = -u_max pi / 2 * (sum of the section's hydraulic lam)
        lh = st.lam[:, rows_h[sec == k]].sum(axis=1)
        assert np.max(np.abs(Wdd[:, k] + P2["u_max"] * math.pi / 2.0 * lh)) <= 1e-12 * np.abs(lh).max()


@pytest.mark.parametrize("dw,dc", [(0.0, 0.0), (1e-3, 1e-8)])
def test_schur_on_two_diameters_equals_monolithic(dw, dc):
    F, solver, st = _iterate(P2, 2, 1, 3)
    C, J, Jd, W, Wdd = solver.evaluate(st)
    sig, sigd = solver.sigma(st)
    Kdd = np.diag(Wdd.sum(axis=0) + sigd)
    rng = np.random.default_rng(4)
    rz, rc = rng.standard_normal((2, model.NS)), rng.standard_normal((2, model.NS))
    rd = np.array([0.3, -0.8])
    fac = kkt.SchurKKT(W, sig, J, Jd, Kdd, dw, dc)
    dz, dd, dl = fac.solve(rz, rd, rc)
    dz2, dd2, dl2, inert = kkt.monolithic_solve(W, sig, J, Jd, Kdd, dw, dc, rz, rd, rc)
    x1 = np.concatenate([dd, dz.ravel(), dl.ravel()])
    x2 = np.concatenate([dd2, dz2.ravel(), dl2.ravel()])
    Kmat = kkt.monolithic_matrix(W, sig, J, Jd, Kdd, dw, dc)
    assert np.linalg.norm(x1 - x2) <= max(1e-12, 10 * np.finfo(float).eps * np.linalg.cond(Kmat)) * np.linalg.norm(x2)
    assert fac.inertia() == inert
    ev = np.linalg.eigvalsh(Kmat)
    assert fac.inertia() == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    # the refined solve's residual on the whole bordered system
    z3, d3, l3 = kkt.solve_refined(fac, W, sig, J, Jd, Kdd, dw, dc, rz, rd, rc)
    ez, ed, ec = kkt.kkt_residual(W, sig, J, Jd, Kdd, dw, dc, z3, d3, l3, rz, rd, rc)
    assert max(np.abs(ez).max(), np.abs(ed).max(), np.abs(ec).max()) <= 1e-9 * max(np.abs(rz).max(), 1.0)


def test_two_section_optimum_is_the_sections_closed_form():
    F = ai.make_feeds(4, 0)
    r2 = ipm.solve(P2, F)
    assert r2.status == "ok"
    d2 = np.atleast_1d(r2.d)
    dk = checks.section_diameters(P2, F, r2.Z, 2)
    assert np.all(np.abs(d2 - dk) <= 1e-8 * dk), (d2, dk)
    # the one-section problem's optimum is the largest section diameter
    r1 = ipm.solve(P1, F)
    assert r1.status == "ok"
    assert abs(max(d2) - r1.d) <= 1e-8 * r1.d
    # E_0 from the definitions at the returned point (complex-step Jacobian)
    assert checks.kkt_error(P2, F, d2, r2.Z, r2.lam, r2.zL, r2.zU, r2.zLd, r2.zUd) <= 1e-8
    # the top section carries less gas (CO2 absorbed on the way up): a smaller diameter
    assert d2[1] < d2[0] or d2[0] < d2[1]


def test_identical_scenarios_reproduce_one_scenario_with_sections():
    F1 = ai.make_feeds(1, 3)
    F3 = np.repeat(F1, 3, axis=1)
    opt = ipm.Options(obj_scaling=100.0, init="inlet")
    r1 = ipm.solve(P2, F1, opt)
    r3 = ipm.solve(P2, F3, opt)
    assert r1.status == "ok" and r3.status == "ok"
    assert np.all(np.abs(np.atleast_1d(r3.d) - np.atleast_1d(r1.d)) <= 1e-8 * np.atleast_1d(r1.d))
    assert np.max(np.abs(r3.Z - r1.Z[0][None, :]) / np.maximum(1.0, np.abs(r1.Z[0]))) <= 1e-6
