"""The regularised block LDL^T of the scenario blocks (kkt_factor with delta_c > 0 or
ABS_PREC_FP64_LDL) against the CPU oracle.

The primal-dual matrix with both regularisations of Wachter & Biegler (2006, Eq. (13) and
Section 3.1), K = [W + Sigma + dw I, J^T; J, -dc I], is factored on the GPU scenario by
scenario by a block LDL^T over the 44 x 44 stage blocks with Bunch-Kaufman pivoting inside
each, and the scenarios eliminated onto d by the scalar Schur complement; the oracle
factors every 440 x 440 scenario block by LAPACK's Bunch-Kaufman (its inertia pinned
against eigenvalue signs, its Schur solve against a monolithic LDL^T).  Checked: the
inertia of the whole matrix, counts equal; S_d to 1e-9; the direction (dz, dd, dlambda)
after FP64 refinement to 1e-10 relative against the oracle's refined Schur solve (the
bound of the block-LU path's direction tests).  With dc large enough the scenario blocks'
own inertia departs from (220, 220, 0) -- W is indefinite at these iterates -- and the
counts must still agree."""
import numpy as np
import pytest

import absorber_inputs as ai
from oracle import ipm, kkt

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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _state(S, seed, k):
    F = ai.make_feeds(S, seed)
    solver = ipm.IPM(P, F)
    if k > 0:
        r = ipm.IPM(P, F, ipm.Options(max_iter=k)).solve()
        st, mu = solver.state_from_result(r), r.mu
    else:
        bc = solver.basecase_start()
        st, mu = solver.initial_state(Z0=bc[0], d0=bc[1]), 0.1
    C, J, Jd, W, Wdd = solver.evaluate(st)
    return F, solver, st, mu, (C, J, Jd, W, Wdd)


@pytest.fixture(scope="module")
def case10():
    return _state(10, 0, 6)


@pytest.fixture(scope="module")
def case37():
    return _state(37, 2, 0)


def _gpu_system(B, case, sig, sigd):
    import torch
    F, solver, st, mu, _ = case
    prob = B.Problem(P, F)
    ld = prob.ld
    x = dev(prob.to_soa(st.Z, st.d))
    lm = dev(prob.to_soa(st.lam))
    jac = torch.zeros(prob.sizes.nnzJ_scen * ld, dtype=torch.float64, device="cuda")
    hes = torch.zeros(prob.sizes.nnzH_scen * ld, dtype=torch.float64, device="cuda")
    prob.eval_grad_jac_hess(x, lm, 1.0, jac=jac, hess=hes)
    sg = dev(prob.to_soa(sig, sigd))
    return prob, x, jac, hes, sg


def _check(B, case, dw, dc, prec=None):
    import torch
    F, solver, st, mu, (C, J, Jd, W, Wdd) = case
    _, _, _, _, _, fac = solver.newton_direction(st, mu, C, J, Jd, W, Wdd, dw=dw, dc=dc)
    sig, sigd = solver.sigma(st)
    gz, gd = solver.barrier_gradient(st, mu)
    rz = -(gz + np.einsum("src,sr->sc", J, st.lam))
    rd = -(gd + float(np.sum(Jd * st.lam)))
    Kdd = float(np.sum(Wdd)) + sigd
    dZ, dd, dl = kkt.solve_refined(fac, W, sig, J, Jd, Kdd, dw, dc, rz, rd, -C, steps=2)
    prob, x, jac, hes, sg = _gpu_system(B, case, sig, sigd)
    inert = prob.kkt_factor(x, jac, hes, sg, delta_w=dw, delta_c=dc,
                            precision=B.PREC_FP64 if prec is None else prec)
    assert inert.n_singular == 0
    assert (inert.n_pos, inert.n_neg, inert.n_zero) == fac.inertia(), ((inert.n_pos, inert.n_neg, inert.n_zero),
                                                                      fac.inertia())
    assert abs(inert.schur_d - fac.Sd) <= 1e-9 * abs(fac.Sd), (inert.schur_d, fac.Sd)
    rx = dev(prob.to_soa(rz, rd))
    rc = dev(prob.to_soa(-C))
    sx, sc = torch.zeros_like(rx), torch.zeros_like(rc)
    info = prob.kkt_solve(rx, rc, sx, sc, max_refine=4, refine_tol=1e-15)
    gz_, gd_ = prob.from_soa(host(sx))
    gl_, _ = prob.from_soa(host(sc))
    xo = np.concatenate([[dd], dZ.ravel(), dl.ravel()])
    xg = np.concatenate([[gd_], gz_.ravel(), gl_.ravel()])
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= 1e-10, (err, info.refine_steps, info.residual)
    return inert, fac


@pytest.mark.parametrize("dw,dc", [(0.0, 1e-8), (1e-4, 1e-8), (0.0, 1e-2), (1e-1, 1.0)])
def test_regularised_direction_s10(B, case10, dw, dc):
    _check(B, case10, dw, dc)


def test_regularised_direction_s37_first_iterate(B, case37):
    # the expected-value start (least-squares multipliers): another matrix, 37 scenarios
    _check(B, case37, 1e-4, 1e-6)


def test_ldl_without_dc_matches_the_block_lu(B, case10):
    # dc = 0 through the block LDL^T: the same inertia and direction as the block LU of J_s
    inert, fac = _check(B, case10, 1e-4, 0.0, prec=B.PREC_FP64_LDL)
    nb = 220 * 10
    assert (inert.n_pos, inert.n_neg) == (nb + (1 if fac.Sd > 0 else 0), nb + (1 if fac.Sd < 0 else 0))


@pytest.mark.parametrize("dc", [1e2, 1e6])
def test_inertia_of_large_dc_follows_the_oracle(B, case10, dc):
    # K_s = [H, J^T; J, -dc I] is congruent to diag(H + J^T J / dc, -dc I): as dc grows the
    # blocks' inertia follows that of H = W + Sigma, indefinite at this iterate (the oracle
    # counts 1849 and 1837 positive eigenvalues of 4401), and at dc = 1e6 S_d is negative
    _check(B, case10, 0.0, dc)


def test_regularisation_arguments(B, case10):
    F, solver, st, mu, (C, J, Jd, W, Wdd) = case10
    sig, sigd = solver.sigma(st)
    prob, x, jac, hes, sg = _gpu_system(B, case10, sig, sigd)
    for kw in (dict(delta_c=-1.0), dict(delta_w=-1.0), dict(delta_c=1e-8, precision=B.PREC_FP32)):
        with pytest.raises(B.AbsorberError) as e:
            prob.kkt_factor(x, jac, hes, sg, **kw)
        assert e.value.status == -1, kw


def _solve_point(B, prob, opt):
    import torch
    x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    y = torch.zeros(prob.n_row, dtype=torch.float64, device="cuda")
    res = prob.ipm_solve(opt, x_out=x, y_out=y)
    zl = torch.zeros_like(x)
    zu = torch.zeros_like(x)
    zd = prob.bound_multipliers(zl, zu)
    Z, d = prob.from_soa(host(x))
    lam, _ = prob.from_soa(host(y))
    ZL, _ = prob.from_soa(host(zl))
    ZU, _ = prob.from_soa(host(zu))
    return res, (Z, d, lam, ZL, ZU, zd[0], zd[1])


@pytest.mark.parametrize("S,seed", [(10, 0), (37, 2)])
def test_ipm_solve_through_the_block_ldlt(B, S, seed):
    # the whole interior-point solve with every scenario block factored by the block LDL^T
    # (Algorithm IC reading every block's inertia from its pivots, each delta_w trial
    # refactored): the optimum of the block-LU path, E_0 <= 1e-8 recomputed by the oracle
    # at the returned point (oracle/checks.kkt_error, complex-step Jacobian)
    from oracle import checks
    F = ai.make_feeds(S, seed)
    prob = B.Problem(P, F)
    r0 = prob.ipm_solve(B.default_options())
    r1, pt = _solve_point(B, prob, B.default_options(kkt=1))
    assert r0.status == 0 and r1.status == 0, (r0.status, r1.status)
    assert abs(r1.d - r0.d) <= 1e-9 * r0.d, (r1.d, r0.d)
    assert abs(r1.iters - r0.iters) <= 2, (r1.iters, r0.iters)
    Z, d, lam, ZL, ZU, zld, zud = pt
    assert checks.kkt_error(P, F, d, Z, lam, ZL, ZU, zld, zud) <= 1e-8
    # graph replay of the same configuration: the eager result bit for bit
    runs = [prob.ipm_solve(B.default_options(kkt=1, graphs=1)) for _ in range(2)]
    assert runs[-1].graph_replays >= 1
    for r in runs:
        assert r.status == 0 and r.iters == r1.iters and r.d == r1.d


def test_batched_block_ldlt_equals_single_solves(B):
    # ragged problems (one of one scenario) side by side: each equals its own solve, and the
    # optimum of the block-LU path wherever that one converges
    feeds = ai.batched_feeds([7, 1, 33, 12], seed=21)
    batch = B.Batch(P, feeds)
    rb = batch.ipm_solve(B.default_options(kkt=1))
    for F, r in zip(feeds, rb):
        prob = B.Problem(P, F)
        rs = prob.ipm_solve(B.default_options(kkt=1))
        assert r.status == rs.status and r.iters == rs.iters and r.d == rs.d, (r.status, rs.status, r.iters, rs.iters)
        rl = prob.ipm_solve(B.default_options())
        if rl.status == 0:
            assert rs.status == 0 and abs(rs.d - rl.d) <= 1e-9 * rl.d, (rs.status, rs.d, rl.d)


def test_block_ldlt_option_checks(B):
    prob = B.Problem(P, ai.make_feeds(2, 0))
    for kw in (dict(kkt=2), dict(kkt=1, precision=1)):
        r = prob.ipm_solve(B.default_options(**kw))
        assert r.status == -1, kw
