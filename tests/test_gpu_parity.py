"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same seeded
inputs.  Tolerances: derivative values to 1e-11 relative (row-scaled: both sides
evaluate the same closed forms in FP64, differing only in libm rounding and summation
order); Newton directions to 1e-10 relative (the stated bound); objective d* to 1e-6
relative and E_0 <= 1e-8 (the stated bounds)."""
import math

import numpy as np
import pytest

import absorber_inputs as ai
from oracle import checks, ipm, model

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


def _iterate(S, seed, dist="uniform", k=None):
    """An interior iterate: the oracle's k-th IPM iterate (k given), or a perturbed start."""
    F = ai.make_feeds(S, seed, dist=dist)
    if k is not None:
        r = ipm.IPM(P, F, ipm.Options(max_iter=k)).solve()
        return F, r
    Z, d = model.initial_point(P, F)
    rng = np.random.default_rng(seed + 100)
    Zs = Z.reshape(S, model.N, model.NV)
    Zs[:, :, :13] = np.abs(Zs[:, :, :13]) * rng.uniform(0.5, 1.5, Zs[:, :, :13].shape) + 0.05
    Zs[:, :, model.IT] = rng.uniform(3.1, 3.5, (S, model.N))
    Zs[:, :, model.IE:model.IE + 5] = rng.normal(0, 1e-3, (S, model.N, 5))
    Zs[:, :, model.IS] = rng.uniform(0.1, 2.0, (S, model.N))
    lam = rng.standard_normal((S, model.NS))
    return F, (Zs.reshape(S, model.NS), 1.37, lam)


def _eval_gpu(B, prob, Z, d, lam):
    import torch
    ld = prob.ld
    x = dev(prob.to_soa(Z, d))
    lm = dev(prob.to_soa(lam))
    c = torch.zeros(prob.n_row, dtype=torch.float64, device="cuda")
    jac = torch.zeros(prob.sizes.nnzJ_scen * ld, dtype=torch.float64, device="cuda")
    hes = torch.zeros(prob.sizes.nnzH_scen * ld, dtype=torch.float64, device="cuda")
    grad = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    f = prob.eval_grad_jac_hess(x, lm, 1.0, grad=grad, c=c, jac=jac, hess=hes, want_f=True)
    return f, host(grad), host(c), host(jac), host(hes), (x, lm, c, jac, hes)


def _rowscaled_close(g, o, rows, tol, floor=0.0):
    """|g - o| <= tol * (|o| + max |o| over the entry's row) + floor."""
    rmax = np.zeros((g.shape[0], rows.max() + 1))
    for s in range(g.shape[0]):
        np.maximum.at(rmax[s], rows, np.abs(o[s]))
    bound = tol * (np.abs(o) + rmax[:, rows]) + floor
    bad = np.abs(g - o) > bound
    assert not bad.any(), (np.argwhere(bad)[:5], g[bad][:5], o[bad][:5])


def _check_eval(B, F, Z, d, lam, sample=None):
    prob = B.Problem(P, F)
    f, grad, c, jac, hes, _ = _eval_gpu(B, prob, Z, d, lam)
    jr, jc, hr, hc = prob.pattern()
    idx = np.arange(F.shape[1]) if sample is None else sample
    Co, J, Jd, W, Wdd = model.derivatives(P, F[:, idx], Z[idx], d, lam[idx])
    Cg, _ = prob.from_soa(c)
    Jg = prob.values_to_scen(jac, len(jr))[idx]
    Hg = prob.values_to_scen(hes, len(hr))[idx]
    Jf = np.concatenate([J, Jd[:, :, None]], axis=2)
    Jo = Jf[:, jr, jc]
    Wf = np.zeros((len(idx), model.NS + 1, model.NS + 1))
    Wf[:, :model.NS, :model.NS] = W
    Wf[:, model.NS, model.NS] = Wdd
    Ho = Wf[:, hr, hc]
    assert f == d and grad[-1] == 1.0 and np.all(grad[:-1][:model.NS * prob.ld] == 0)
    # a residual is a difference of terms of size up to ~1e2 (ln K, enthalpy flows,
    # Henry products): 1e-12 absolute is ~1e2 ulps of those terms
    _rowscaled_close(Cg[idx], Co, np.arange(model.NS), 1e-11, floor=1e-12)
    _rowscaled_close(Jg, Jo, jr, 1e-11)
    _rowscaled_close(Hg, Ho, hr, 1e-11)
    return prob


def test_eval_parity_small(B):
    F, (Z, d, lam) = _iterate(10, 0)
    _check_eval(B, F, Z, d, lam)


def test_eval_parity_ragged_and_single(B):
    for S in (1, 33, 70):        # one scenario; ragged tails past one / two warps
        F, (Z, d, lam) = _iterate(S, S)
        _check_eval(B, F, Z, d, lam)


def test_eval_parity_full_size_sampled(B):
    F, (Z, d, lam) = _iterate(5000, 2, dist="truncnorm")
    rng = np.random.default_rng(5)
    sample = np.sort(np.concatenate([[0, 4999], rng.choice(np.arange(1, 4999), 30, replace=False)]))
    _check_eval(B, F, Z, d, lam, sample)


def _direction_case(S, seed, k):
    F, r = _iterate(S, seed, k=k)
    solver = ipm.IPM(P, F)
    st = solver.state_from_result(r)
    C, J, Jd, W, Wdd = solver.evaluate(st)
    mu = r.mu
    dZ, dd, dl, dw, dc, fac = solver.newton_direction(st, mu, C, J, Jd, W, Wdd, dw=0.0, dc=0.0)
    sig, sigd = solver.sigma(st)
    gz, gd = solver.barrier_gradient(st, mu)
    rz = -(gz + np.einsum("src,sr->sc", J, st.lam))
    rd = -(gd + float(np.sum(Jd * st.lam)))
    return F, st, sig, sigd, rz, rd, -C, (dZ, dd, dl), fac


@pytest.mark.parametrize("prec", [0, 1])
def test_newton_direction_parity(B, prec):
    import torch
    F, st, sig, sigd, rz, rd, rc, (dZ, dd, dl), fac = _direction_case(10, 0, 6)
    prob = B.Problem(P, F)
    _, _, _, _, _, (x, lm, c, jac, hes) = _eval_gpu(B, prob, st.Z, st.d, st.lam)
    sg = dev(prob.to_soa(sig, sigd))
    inert = prob.kkt_factor(x, jac, hes, sg, precision=prec)
    assert inert.n_singular == 0
    o_in = fac.inertia()
    assert (inert.n_pos, inert.n_neg, inert.n_zero) == o_in
    # FP64: the Schur scalar to 1e-9; FP32: q = J^-1 b comes from FP32 factors (a few
    # ulps of float times the block condition number ~1e5); the refined direction below
    # must still meet 1e-10
    assert abs(inert.schur_d - fac.Sd) <= (1e-9 if prec == 0 else 1e-2) * abs(fac.Sd)
    rx = dev(prob.to_soa(rz, rd))
    rcd = dev(prob.to_soa(rc))
    sx = torch.zeros_like(rx)
    sc = torch.zeros_like(rcd)
    info = prob.kkt_solve(rx, rcd, sx, sc, max_refine=2 if prec == 0 else 10, refine_tol=1e-15)
    gz_, gd_ = prob.from_soa(host(sx))
    gl_, _ = prob.from_soa(host(sc))
    xo = np.concatenate([[dd], dZ.ravel(), dl.ravel()])
    xg = np.concatenate([[gd_], gz_.ravel(), gl_.ravel()])
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= 1e-10, (err, info.refine_steps, info.residual)


def test_fp32_direction_before_and_after_refinement(B):
    # the FP32 stage-block inverses alone give the direction to FP32 accuracy times the
    # blocks' condition numbers; the FP64 refinement then reaches 1e-10 in a few steps
    import torch
    F, st, sig, sigd, rz, rd, rc, (dZ, dd, dl), fac = _direction_case(10, 0, 6)
    prob = B.Problem(P, F)
    _, _, _, _, _, (x, lm, c, jac, hes) = _eval_gpu(B, prob, st.Z, st.d, st.lam)
    sg = dev(prob.to_soa(sig, sigd))
    inert = prob.kkt_factor(x, jac, hes, sg, precision=1)
    assert inert.n_singular == 0
    rx = dev(prob.to_soa(rz, rd))
    rcd = dev(prob.to_soa(rc))
    xo = np.concatenate([[dd], dZ.ravel(), dl.ravel()])
    errs = []
    for mr in (0, 8):
        sx = torch.zeros_like(rx)
        sc = torch.zeros_like(rcd)
        info = prob.kkt_solve(rx, rcd, sx, sc, max_refine=mr, refine_tol=1e-12)
        gz_, gd_ = prob.from_soa(host(sx))
        gl_, _ = prob.from_soa(host(sc))
        xg = np.concatenate([[gd_], gz_.ravel(), gl_.ravel()])
        errs.append((np.linalg.norm(xg - xo) / np.linalg.norm(xo), info.refine_steps, info.residual))
    assert errs[0][0] <= 5e-2, errs
    assert errs[1][0] <= 1e-9 and errs[1][1] <= 4, errs


def _gpu_solve(B, F, prec=0, **opt):
    import torch
    prob = B.Problem(P, F)
    o = B.default_options(precision=prec, max_refine=(0 if prec == 0 else 8), **opt)
    x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    y = torch.zeros(prob.n_row, dtype=torch.float64, device="cuda")
    res = prob.ipm_solve(o, x_out=x, y_out=y)
    Z, d = prob.from_soa(host(x))
    lam, _ = prob.from_soa(host(y))
    return prob, res, Z, d, lam


@pytest.fixture(scope="module")
def oracle_s10():
    F = ai.make_feeds(10, 0)
    return F, ipm.solve(P, F)


def test_ipm_solve_matches_oracle_s10(B, oracle_s10):
    F, r = oracle_s10
    prob, res, Z, d, lam = _gpu_solve(B, F)
    assert res.status == 0 and r.status == "ok"
    assert res.E0 <= 1e-8
    assert abs(res.d - r.d) <= 1e-6 * r.d
    assert abs(d - res.d) == 0.0
    dmin, _ = checks.minimum_diameter(P, F, Z)
    assert abs(d - dmin) <= 1e-8 * dmin
    scale = np.maximum(1.0, np.abs(r.Z))
    assert np.max(np.abs(Z - r.Z) / scale) <= 1e-5
    assert abs(res.iters - r.iters) <= 3


def test_ipm_solve_fp32_mixed_matches_fp64(B, oracle_s10):
    F, r = oracle_s10
    prob, res, Z, d, lam = _gpu_solve(B, F, prec=1)
    assert res.status == 0 and res.E0 <= 1e-8
    assert abs(res.d - r.d) <= 1e-6 * r.d


def test_ipm_solve_s500_properties(B):
    F = ai.make_feeds(500, 1)
    prob, res, Z, d, lam = _gpu_solve(B, F)
    assert res.status == 0 and res.E0 <= 1e-8
    dmin, vol = checks.minimum_diameter(P, F, Z)
    assert abs(d - dmin) <= 1e-8 * dmin
    # sampled scenarios (including the one that sets d*): the GPU states are the root of
    # each scenario's own square MESH system, found by the oracle's independent Newton
    arg = int(np.unravel_index(np.argmax(vol), vol.shape)[0])
    rng = np.random.default_rng(9)
    sample = np.unique(np.concatenate([[arg, 0, 499], rng.choice(500, 5, replace=False)]))
    Zn, hist = checks.mesh_newton(P, F[:, sample], Z[sample], d, iters=5)
    assert hist[-1] <= 1e-12
    keep = np.ones(model.NS, dtype=bool)
    keep[model.NV - 1::model.NV] = False
    assert np.max(np.abs(Zn[:, keep] - Z[sample][:, keep]) / np.maximum(1, np.abs(Zn[:, keep]))) <= 1e-6
    el_in, el_out, h_in, h_out = checks.column_balances(P, F, Z)
    np.testing.assert_allclose(el_out, el_in, rtol=0, atol=1e-8 * np.abs(el_in).max())


def test_error_paths(B):
    import torch
    F = ai.make_feeds(4, 0)
    bad = dict(P)
    bad["d_lo"], bad["d_hi"] = 2.0, 1.0
    with pytest.raises(B.AbsorberError) as e:
        B.Problem(bad, F)
    assert e.value.status == -9
    Fn = F.copy()
    Fn[0, 1] = np.nan
    with pytest.raises(B.AbsorberError) as e:
        B.Problem(P, Fn)
    assert e.value.status == -7
    prob = B.Problem(P, F)
    v = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    r = torch.zeros(prob.n_row, dtype=torch.float64, device="cuda")
    with pytest.raises(B.AbsorberError):
        prob.kkt_solve(v, r, v.clone(), r.clone())          # no factorization yet
    with pytest.raises(B.AbsorberError):
        prob.kkt_factor(v, r, r, v, delta_c=1e-8)            # delta_c must be 0
    o = B.default_options(max_iter=3)
    res = prob.ipm_solve(o)
    assert res.status == -6 and res.iters == 3               # iteration limit is reported
    o = B.default_options(tol=-1.0)
    assert prob.ipm_solve(o).status == -1
    o = B.default_options(precision=1, max_refine=8, factor_tile=3)   # not a launch shape
    assert prob.ipm_solve(o).status == -1


def test_full_size_s5000_mixed_precision_properties(B):
    # the bench workload (5000 scenarios, truncated-normal feeds) with FP32 factors and
    # FP64 refinement: properties that fix the optimum at any size
    F = ai.workload_feeds("absorber-S5000-tn5-seed2")
    prob, res, Z, d, lam = _gpu_solve(B, F, prec=1)
    assert res.status == 0 and res.E0 <= 1e-8
    dmin, vol = checks.minimum_diameter(P, F, Z)
    assert abs(d - dmin) <= 1e-8 * dmin
    arg = int(np.unravel_index(np.argmax(vol), vol.shape)[0])
    rng = np.random.default_rng(17)
    sample = np.unique(np.concatenate([[arg, 0, 4999], rng.choice(5000, 5, replace=False)]))
    Zn, hist = checks.mesh_newton(P, F[:, sample], Z[sample], d, iters=5)
    assert hist[-1] <= 1e-12
    keep = np.ones(model.NS, dtype=bool)
    keep[model.NV - 1::model.NV] = False
    assert np.max(np.abs(Zn[:, keep] - Z[sample][:, keep]) / np.maximum(1, np.abs(Zn[:, keep]))) <= 1e-6
    el_in, el_out, h_in, h_out = checks.column_balances(P, F, Z)
    np.testing.assert_allclose(el_out, el_in, rtol=0, atol=1e-8 * np.abs(el_in).max())
    # one active hydraulic row: the binding scenario's multiplier carries the objective
    lh = lam.reshape(5000, model.N, model.NV)[:, :, model.NV - 1]
    assert abs(lh.sum() * P["u_max"] * math.pi * d / 2.0 - 1.0) <= 1e-6


def test_paper_layout_and_scenario_status(B):
    # the paper's 300-entry layout, bit for bit the oracle's restatement of it; the fixed
    # entries exactly zero; every scenario's factorization healthy after a solve
    import torch
    F = ai.make_feeds(37, 5)
    prob, res, Z, d, lam = _gpu_solve(B, F)
    assert res.status == 0
    x = dev(prob.to_soa(Z, d))
    out = torch.zeros(1 + 300 * 37, dtype=torch.float64, device="cuda")
    prob.paper_layout(x, out)
    o = host(out)
    assert o[0] == d
    ref = model.full_layout(P, Z)
    assert np.array_equal(o[1:].reshape(37, model.N, 30), ref)
    fixed = np.zeros(30, dtype=bool)
    fixed[9:11] = True            # x of N2, O2
    fixed[11:18] = True           # y of the 7 non-volatile species
    assert np.all(o[1:].reshape(37, model.N, 30)[:, :, fixed] == 0.0)
    assert np.all(prob.scenario_status() == 0)
