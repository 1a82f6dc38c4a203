"""Oracle KKT algebra (oracle/kkt.py): Schur-on-d solve against the monolithic dense
LDL^T, inertia against eigenvalue signs, residual of the solve."""
import numpy as np

import absorber_inputs as ai
from oracle import ipm, kkt, model

P = ai.PARAMS


def _iterate(S, seed, iters):
    F = ai.make_feeds(S, seed)
    solver = ipm.IPM(P, F, ipm.Options(max_iter=iters))
    r = solver.solve()
    st = solver.state_from_result(r)
    C, J, Jd, W, Wdd = solver.evaluate(st)
    sig, sigd = solver.sigma(st)
    return solver, st, C, J, Jd, W, Wdd, sig, sigd


def test_schur_equals_monolithic_ldlt():
    solver, st, C, J, Jd, W, Wdd, sig, sigd = _iterate(2, 0, 3)
    rng = np.random.default_rng(0)
    rz, rc = rng.standard_normal((2, model.NS)), rng.standard_normal((2, model.NS))
    rd = 0.7
    Kdd = Wdd.sum() + sigd
    for dw, dc in ((0.0, 0.0), (1e-3, 1e-8)):
        fac = kkt.SchurKKT(W, sig, J, Jd, Kdd, dw, dc)
        dz, dd, dl = fac.solve(rz, rd, rc)
        dz2, dd2, dl2, inert = kkt.monolithic_solve(W, sig, J, Jd, Kdd, dw, dc, rz, rd, rc)
        x1 = np.concatenate([[dd], dz.ravel(), dl.ravel()])
        x2 = np.concatenate([[dd2], dz2.ravel(), dl2.ravel()])
        # both are backward stable; their difference is bounded by cond(K) * eps
        K = kkt.monolithic_matrix(W, sig, J, Jd, Kdd, dw, dc)
        r = np.concatenate([[rd]] + [np.concatenate([rz[s], rc[s]]) for s in range(2)])
        for x in (x1, x2):
            xo = np.empty_like(x)
            xo[0] = x[0]
            for s in range(2):
                o = 1 + 2 * model.NS * s
                xo[o:o + model.NS] = x[1 + model.NS * s:1 + model.NS * (s + 1)]
                xo[o + model.NS:o + 2 * model.NS] = x[1 + 2 * model.NS + model.NS * s:1 + 2 * model.NS + model.NS * (s + 1)]
            berr = np.linalg.norm(K @ xo - r) / (np.linalg.norm(K, 2) * np.linalg.norm(xo) + np.linalg.norm(r))
            assert berr <= 1e-14
        cond = np.linalg.cond(K)
        assert np.linalg.norm(x1 - x2) <= max(1e-12, 10 * np.finfo(float).eps * cond) * np.linalg.norm(x2)
        assert fac.inertia() == inert


def test_inertia_matches_eigenvalue_signs():
    solver, st, C, J, Jd, W, Wdd, sig, sigd = _iterate(1, 3, 2)
    Kdd = Wdd.sum() + sigd
    for dw in (0.0, 1e-2, -5.0):      # a negative shift forces a wrong inertia
        K = kkt.monolithic_matrix(W, sig, J, Jd, Kdd, dw, 0.0)
        ev = np.linalg.eigvalsh(K)
        expect = (int((ev > 0).sum()), int((ev < 0).sum()), 0)
        fac = kkt.SchurKKT(W, sig, J, Jd, Kdd, dw, 0.0)
        assert fac.inertia() == expect
        Ks = kkt.scenario_matrix(W[0], sig[0], J[0], dw, 0.0)
        evs = np.linalg.eigvalsh(Ks)
        assert kkt.BlockLDL(Ks).inertia() == (int((evs > 0).sum()), int((evs < 0).sum()), 0)


def test_newton_direction_solves_full_system():
    solver, st, C, J, Jd, W, Wdd, sig, sigd = _iterate(2, 5, 4)
    mu = 0.1
    dZ, dd, dl, dw, dc, fac = solver.newton_direction(st, mu, C, J, Jd, W, Wdd)
    K = kkt.monolithic_matrix(W, sig, J, Jd, Wdd.sum() + sigd, dw, dc)
    gz, gd = solver.barrier_gradient(st, mu)
    rhs = [-(gd + float(np.sum(Jd * st.lam)))]
    x = [dd]
    for s in range(2):
        rhs += list(-(gz[s] + J[s].T @ st.lam[s])) + list(-C[s])
        x += list(dZ[s]) + list(dl[s])
    res = K @ np.array(x) - np.array(rhs)
    assert np.linalg.norm(res) <= 1e-11 * (np.linalg.norm(rhs) + np.abs(K).max() * np.linalg.norm(x))


def test_refined_schur_solve_matches_monolithic_and_reduces_the_residual():
    # the refined direction of a real iterate (k = 6 of the 10-scenario workload is too
    # large for a monolithic matrix here; two scenarios, k = 4) with a large shift:
    # agreement with the dense monolithic LDL^T solve improves to a few ulps of the
    # solution, and the block-row residual of kkt_residual equals K x - r of the
    # monolithic matrix (a wrong sign or a dropped block would break that equality)
    solver, st, C, J, Jd, W, Wdd, sig, sigd = _iterate(2, 5, 4)
    rng = np.random.default_rng(4)
    rz, rc = rng.standard_normal((2, model.NS)), rng.standard_normal((2, model.NS))
    rd = -0.3
    Kdd = Wdd.sum() + sigd
    for dw, dc in ((1e-1, 0.0), (1e-4, 1e-8)):
        fac = kkt.SchurKKT(W, sig, J, Jd, Kdd, dw, dc)
        x0 = fac.solve(rz, rd, rc)
        x2 = kkt.solve_refined(fac, W, sig, J, Jd, Kdd, dw, dc, rz, rd, rc, steps=2)
        K = kkt.monolithic_matrix(W, sig, J, Jd, Kdd, dw, dc)
        n = model.NS

        def full(x):
            v = np.zeros(1 + 4 * n)
            v[0] = x[1]
            for s in range(2):
                o = 1 + 2 * n * s
                v[o:o + n] = x[0][s]
                v[o + n:o + 2 * n] = x[2][s]
            return v

        r = full((rz, rd, rc))
        for x in (x0, x2):
            ez, ed, ec = kkt.kkt_residual(W, sig, J, Jd, Kdd, dw, dc, *x, rz, rd, rc)
            np.testing.assert_allclose(full((ez, ed, ec)), r - K @ full(x), rtol=0,
                                       atol=1e-12 * np.abs(K).max() * np.abs(full(x)).max())
        res0 = np.linalg.norm(r - K @ full(x0))
        res2 = np.linalg.norm(r - K @ full(x2))
        assert res2 <= res0
        xm = np.linalg.solve(K, r)
        assert np.linalg.norm(full(x2) - xm) <= np.linalg.norm(full(x0) - xm) + 1e-13 * np.linalg.norm(xm)


def test_regularised_block_inertia_matches_eigenvalue_signs():
    # the dual regularisation -dc I (Wachter & Biegler 2006, Section 3.1): the oracle's
    # Bunch-Kaufman inertia of a scenario block against the signs of its eigenvalues, for
    # dc small (the inertia of dc = 0) up to large (that of W + Sigma, indefinite here)
    solver, st, C, J, Jd, W, Wdd, sig, sigd = _iterate(1, 3, 2)
    seen = set()
    for dc in (1e-8, 1e-2, 1.0, 1e6):
        Ks = kkt.scenario_matrix(W[0], sig[0], J[0], 0.0, dc)
        ev = np.linalg.eigvalsh(Ks)
        expect = (int((ev > 0).sum()), int((ev < 0).sum()), 0)
        assert kkt.BlockLDL(Ks).inertia() == expect, dc
        seen.add(expect)
    assert len(seen) > 1    # the range of dc crosses a change of inertia
