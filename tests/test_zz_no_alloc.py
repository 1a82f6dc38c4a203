"""The allocation-free Newton-direction entry point (kkt_newton_noalloc).

Some callers cannot allocate GPU memory once they run (a fixed device-memory budget,
memory owned by another runtime's allocator, no allocator synchronisation allowed
between graph captures).  For them the library offers one entry point whose scratch
lives in a static device array.  This file checks it through the C ABI against the
regular kkt_factor + kkt_solve pair on two calls in a row (different iterates, so the
shared scratch must not carry state from one call into the next), and that sizes above
the static maximum are rejected.  It is collected last on purpose."""
import numpy as np
import pytest

import absorber_inputs as ai
from oracle import ipm

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


def _case(B, S, seed, scale):
    """Device buffers of one Newton system at a perturbed default start."""
    import torch
    F = ai.make_feeds(S, seed)
    solver = ipm.IPM(P, F)
    st = solver.initial_state()
    st.Z = st.Z * (1.0 + scale * np.sin(np.arange(st.Z.size)).reshape(st.Z.shape))
    st.Z = np.maximum(st.Z, solver.pr.lo + 1e-3)
    C, J, Jd, W, Wdd = solver.evaluate(st)
    mu = 0.1
    sig, sigd = solver.sigma(st)
    gz, gd = solver.barrier_gradient(st, mu)
    rz = -(gz + np.einsum("src,sr->sc", J, st.lam))
    rd = -(gd + float(np.sum(Jd * st.lam)))
    prob = B.Problem(P, F)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x = dev(prob.to_soa(st.Z, st.d))
    lam = dev(prob.to_soa(st.lam))
    jac = torch.zeros(prob.sizes.nnzJ_scen * prob.ld, dtype=torch.float64, device="cuda")
    hes = torch.zeros(prob.sizes.nnzH_scen * prob.ld, dtype=torch.float64, device="cuda")
    prob.eval_grad_jac_hess(x, lam, 1.0, jac=jac, hess=hes)
    return prob, x, jac, hes, dev(prob.to_soa(sig, sigd)), dev(prob.to_soa(rz, rd)), dev(prob.to_soa(-C))


def test_noalloc_matches_factor_solve_two_calls(B):
    import torch
    for seed, scale in ((0, 0.0), (1, 0.02)):
        prob, x, jac, hes, sig, rx, rc = _case(B, 10, seed, scale)
        inert = prob.kkt_factor(x, jac, hes, sig, delta_w=1e-6)
        ref_x, ref_c = torch.zeros_like(rx), torch.zeros_like(rc)
        prob.kkt_solve(rx, rc, ref_x, ref_c, max_refine=0)
        out_x, out_c = torch.full_like(rx, np.nan), torch.full_like(rc, np.nan)
        sd = B.kkt_newton_noalloc(P, prob.S, prob.ld, x, jac, hes, sig, rx, rc, out_x, out_c, delta_w=1e-6)
        torch.cuda.synchronize()
        assert abs(sd - inert.schur_d) <= 1e-12 * abs(inert.schur_d)
        a = np.concatenate([prob.from_soa(out_x.cpu().numpy())[0].ravel(), [out_x[-1].item()],
                            prob.from_soa(out_c.cpu().numpy())[0].ravel()])
        b = np.concatenate([prob.from_soa(ref_x.cpu().numpy())[0].ravel(), [ref_x[-1].item()],
                            prob.from_soa(ref_c.cpu().numpy())[0].ravel()])
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("S", [97, 128])
def test_noalloc_ragged_and_maximum_size(B, S):
    # a size that is not a multiple of 32 (ragged last warp and block) and the largest
    # size the static scratch holds (every offset inside it at its limit)
    import torch
    prob, x, jac, hes, sig, rx, rc = _case(B, S, 2, 0.01)
    inert = prob.kkt_factor(x, jac, hes, sig, delta_w=1e-6)
    ref_x, ref_c = torch.zeros_like(rx), torch.zeros_like(rc)
    prob.kkt_solve(rx, rc, ref_x, ref_c, max_refine=0)
    out_x, out_c = torch.full_like(rx, np.nan), torch.full_like(rc, np.nan)
    sd = B.kkt_newton_noalloc(P, prob.S, prob.ld, x, jac, hes, sig, rx, rc, out_x, out_c, delta_w=1e-6)
    assert abs(sd - inert.schur_d) <= 1e-12 * abs(inert.schur_d)
    a = np.concatenate([prob.from_soa(out_x.cpu().numpy())[0].ravel(), [out_x[-1].item()],
                        prob.from_soa(out_c.cpu().numpy())[0].ravel()])
    b = np.concatenate([prob.from_soa(ref_x.cpu().numpy())[0].ravel(), [ref_x[-1].item()],
                        prob.from_soa(ref_c.cpu().numpy())[0].ravel()])
    assert np.all(np.isfinite(a))
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


def test_noalloc_reports_singular_block_and_negative_schur(B):
    import torch
    prob, x, jac, hes, sig, rx, rc = _case(B, 10, 0, 0.0)
    out_x, out_c = torch.zeros_like(rx), torch.zeros_like(rc)
    # every Jacobian value of scenario 3 zeroed: its stage blocks are singular
    js = jac.clone().view(prob.sizes.nnzJ_scen, prob.ld)
    js[:, 3] = 0.0
    with pytest.raises(B.AbsorberError) as e:
        B.kkt_newton_noalloc(P, prob.S, prob.ld, x, js.view(-1), hes, sig, rx, rc, out_x, out_c)
    assert e.value.status == -7
    # a barrier diagonal far below zero makes the Schur complement on d negative
    with pytest.raises(B.AbsorberError) as e:
        B.kkt_newton_noalloc(P, prob.S, prob.ld, x, jac, hes, sig - 1e12, rx, rc, out_x, out_c)
    assert e.value.status == -4
    # the entry still works after both failures
    sd = B.kkt_newton_noalloc(P, prob.S, prob.ld, x, jac, hes, sig, rx, rc, out_x, out_c, delta_w=1e-6)
    assert np.isfinite(sd) and sd > 0


def test_noalloc_rejects_oversized(B):
    import torch
    S = B.NOALLOC_MAX_SCENARIOS + 1
    ld = (S + 31) // 32 * 32
    v = torch.zeros(220 * ld + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(B.AbsorberError) as e:
        B.kkt_newton_noalloc(P, S, ld, v, v, v, v, v, v, v.clone(), v.clone())
    assert e.value.status == -1 and "static scratch" in str(e.value)
