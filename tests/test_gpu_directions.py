"""GPU Newton directions against the CPU oracle with the primal regularisation delta_w > 0
(Wachter & Biegler 2006, Algorithm IC: the shifted system [W + Sigma + dw I, J^T; J, 0]),
in both factor precisions, at 10 scenarios and at 600 (past the tile autotuner's
threshold of 256 scenarios, so the tuned launch shapes run), and the mixed-precision
path's FP64 escalation forced from the host.

The GPU applies delta_w only to the Schur scalar and to the products with H (the block
factors of J_s do not depend on it); the oracle factors the whole shifted KKT block by
dense Bunch-Kaufman LDL^T.  Bound: relative error <= 1e-10 of the whole direction
(dz, dd, dlambda) after FP64 refinement, the stated tolerance.  The oracle's direction is
its Schur-reduced solve refined twice in FP64 on the whole system (oracle/kkt.py
solve_refined): at these iterates cond(K) * eps is ~1e-10 to 1e-9, so two unrefined
backward-stable solves (the oracle's Schur and monolithic ones) already differ by that
much; refined, the oracle's direction is the system's solution to far below 1e-10."""
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
    """An iterate of the oracle's method and its derivatives: the k-th iterate (k > 0), or
    the first one (k = 0: the expected-value start with least-squares multipliers)."""
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
def case600():
    return _state(600, 1, 0)


def _check_direction(B, case, dw, prec):
    import torch
    F, solver, st, mu, (C, J, Jd, W, Wdd) = case
    _, _, _, _, _, fac = solver.newton_direction(st, mu, C, J, Jd, W, Wdd, dw=dw, dc=0.0)
    sig, sigd = solver.sigma(st)
    gz, gd = solver.barrier_gradient(st, mu)
    rz = -(gz + np.einsum("src,sr->sc", J, st.lam))
    rd = -(gd + float(np.sum(Jd * st.lam)))
    Kdd = float(np.sum(Wdd)) + sigd
    dZ, dd, dl = kkt.solve_refined(fac, W, sig, J, Jd, Kdd, dw, 0.0, rz, rd, -C, steps=2)
    prob = B.Problem(P, F)
    ld = prob.ld
    x = dev(prob.to_soa(st.Z, st.d))
    lm = dev(prob.to_soa(st.lam))
    jac = torch.zeros(prob.sizes.nnzJ_scen * ld, dtype=torch.float64, device="cuda")
    hes = torch.zeros(prob.sizes.nnzH_scen * ld, dtype=torch.float64, device="cuda")
    prob.eval_grad_jac_hess(x, lm, 1.0, jac=jac, hess=hes)
    # kkt_solve reads jac, hes and sigma again: they must outlive the factorization
    sg = dev(prob.to_soa(sig, sigd))
    inert = prob.kkt_factor(x, jac, hes, sg, delta_w=dw, precision=prec)
    assert inert.n_singular == 0
    assert (inert.n_pos, inert.n_neg, inert.n_zero) == fac.inertia()
    # the Schur scalar with the shift: FP64 to 1e-9; FP32 from FP32 block factors (the
    # refined direction below is the bound that matters)
    assert abs(inert.schur_d - fac.Sd) <= (1e-9 if prec == 0 else 1e-2) * abs(fac.Sd)
    rx = dev(prob.to_soa(rz, rd))
    rc = dev(prob.to_soa(-C))
    sx, sc = torch.zeros_like(rx), torch.zeros_like(rc)
    info = prob.kkt_solve(rx, rc, sx, sc, max_refine=(2 if prec == 0 else 10), refine_tol=1e-15)
    gz_, gd_ = prob.from_soa(host(sx))
    gl_, _ = prob.from_soa(host(sc))
    xo = np.concatenate([[dd], dZ.ravel(), dl.ravel()])
    xg = np.concatenate([[gd_], gz_.ravel(), gl_.ravel()])
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= 1e-10, (err, info.refine_steps, info.residual)
    return prob


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dw", [1e-4, 1e-1])
def test_direction_with_delta_w_s10(B, case10, dw, prec):
    _check_direction(B, case10, dw, prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dw", [1e-4, 1e-1])
def test_direction_with_delta_w_s600_tuned_shapes(B, case600, dw, prec):
    # the first factor/solve launches of this size bucket time every warps-per-block
    # candidate and keep the fastest: the shapes the solves below use are the tuned ones
    prob = _check_direction(B, case600, dw, prec)
    assert prob.S >= 256


def test_forced_fp64_escalation_s10(B):
    # FP32 factors with a refinement target no FP64 refinement reaches in one step: every
    # iteration escalates to FP64 factors, and the solve still reaches the FP64 result
    import torch
    F = ai.make_feeds(10, 0)
    r64 = B.Problem(P, F).ipm_solve(B.default_options())
    assert r64.status == 0
    prob = B.Problem(P, F)
    o = B.default_options(precision=1, max_refine=1, refine_tol=1e-300)
    x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    res = prob.ipm_solve(o, x_out=x)
    assert res.status == 0 and res.E0 <= 1e-8
    assert res.fp64_fallbacks > 0
    assert abs(res.d - r64.d) <= 1e-6 * r64.d
    Z, d = prob.from_soa(host(x))
    assert np.all(np.isfinite(Z)) and d == res.d


def test_partial_per_scenario_escalation_s600(B):
    # FP32 factors with one refinement round and a 1e-9 target: in some iterations the
    # round leaves a few scenarios' rows above the target; only those scenarios are
    # refactored in FP64 (mixed-precision block solves for the rest of the iteration), and
    # the solve reaches the FP64 path's optimum
    F = ai.make_feeds(600, 1)
    r64 = B.Problem(P, F).ipm_solve(B.default_options())
    assert r64.status == 0
    prob = B.Problem(P, F)
    res = prob.ipm_solve(B.default_options(precision=1, max_refine=1, refine_tol=1e-9))
    assert res.status == 0 and res.E0 <= 1e-8
    assert res.fp64_fallbacks > 0
    assert 0 < res.fp64_scenarios < 0.25 * prob.S * res.fp64_fallbacks, (res.fp64_scenarios, res.fp64_fallbacks)
    assert abs(res.d - r64.d) <= 1e-6 * r64.d
    # with the default refinement (8 rounds to 1e-10) nothing escalates on this workload
    r8 = prob.ipm_solve(B.default_options(precision=1, max_refine=8))
    assert r8.status == 0 and r8.fp64_scenarios == 0 and r8.fp64_fallbacks == 0


@pytest.mark.parametrize("dw", [0.0, 1e-1])
def test_tensor_core_factor_direction_s10(B, case10, dw):
    # FP32 stage-block inverses by the blocked Gauss-Jordan with tensor-core trailing updates:
    # after FP64 refinement the direction meets the same 1e-10 bound
    _check_direction(B, case10, dw, 3)


def test_tensor_core_factor_direction_s600(B, case600):
    _check_direction(B, case600, 1e-4, 3)


@pytest.mark.parametrize("S,seed", [(37, 2), (600, 1)])
def test_tensor_core_factor_solve(B, S, seed):
    # the interior-point solve with the tensor-core factor kernel reaches the same optimum as
    # with the SIMT Gauss-Jordan kernel and the FP64 path
    F = ai.make_feeds(S, seed)
    prob = B.Problem(P, F)
    r64 = prob.ipm_solve(B.default_options())
    rs = prob.ipm_solve(B.default_options(precision=1, max_refine=8))
    rt = prob.ipm_solve(B.default_options(precision=1, max_refine=8, factor_kernel=1))
    assert r64.status == rs.status == rt.status == 0
    assert rt.E0 <= 1e-8
    assert abs(rt.d - r64.d) <= 1e-6 * r64.d and abs(rt.d - rs.d) <= 1e-6 * rs.d
    assert abs(rt.iters - rs.iters) <= 2
