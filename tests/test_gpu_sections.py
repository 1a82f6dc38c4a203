"""A design vector with two entries on the GPU (the general Eq. (8) with dim theta = 2): a
column of two sections of five stages, each with its own diameter used by its stages'
hydraulic rows (abs_params.n_sections = 2), the objective their stage-weighted sum.  The
scenario blocks are eliminated onto the two diameters by a 2 x 2 Schur complement
(q_k = J_s^-1 b_k for the border column of each section), Algorithm IC tests it for
positive definiteness, and every scalar of the method carries two design entries.

Checked against the oracle (oracle/ with P["n_sections"] = 2, pinned on the CPU): the
section diameters of the oracle's solve, the closed form of each section's diameter from
the GPU's states (checks.section_diameters), E_0 <= 1e-8 recomputed by the oracle at the
GPU's returned point with its bound multipliers, the largest section diameter equal to
the one-section optimum; the mixed-precision path and batches against the FP64 single
solves; entry points without two-section support refuse it."""
import numpy as np
import pytest

import absorber_inputs as ai
from oracle import checks, ipm

pytestmark = pytest.mark.gpu
P1 = ai.PARAMS
P2 = dict(ai.PARAMS, n_sections=2)


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
    K = prob.K
    return res, (Z, d, lam, ZL, ZU, zd[:K], zd[K:])


def test_two_sections_match_the_oracle_s4(B):
    F = ai.make_feeds(4, 0)
    ro = ipm.solve(P2, F)
    assert ro.status == "ok"
    prob = B.Problem(P2, F)
    assert prob.K == 2
    res, (Z, d, lam, ZL, ZU, zld, zud) = _solve_point(B, prob, B.default_options())
    assert res.status == 0 and res.E0 <= 1e-8, (res.status, res.E0)
    dsec = np.array(res.d_sec)
    assert np.allclose(d, dsec, rtol=0, atol=0) and res.d == dsec[0]
    assert np.all(np.abs(dsec - ro.d) <= 1e-6 * ro.d), (dsec, ro.d)
    assert abs(res.iters - ro.iters) <= 3, (res.iters, ro.iters)
    assert abs(res.obj - 0.5 * (dsec[0] + dsec[1])) <= 1e-15 * res.obj
    # each section's diameter is the smallest its own stages' hydraulic rows allow
    dk = checks.section_diameters(P2, F, Z, 2)
    assert np.all(np.abs(dsec - dk) <= 1e-8 * dk), (dsec, dk)
    # E_0 from the definitions at the returned point (complex-step Jacobian, both entries)
    assert checks.kkt_error(P2, F, dsec, Z, lam, ZL, ZU, zld, zud) <= 1e-8
    # the one-section optimum is the larger section diameter
    r1 = B.Problem(P1, F).ipm_solve(B.default_options())
    assert r1.status == 0 and abs(max(dsec) - r1.d) <= 1e-8 * r1.d


def test_two_sections_mixed_precision_and_full_size_s600(B):
    F = ai.make_feeds(600, 1)
    prob = B.Problem(P2, F)
    r64, pt = _solve_point(B, prob, B.default_options())
    r32 = prob.ipm_solve(B.default_options(precision=1, max_refine=8))
    assert r64.status == 0 and r32.status == 0 and r32.E0 <= 1e-8
    d64, d32 = np.array(r64.d_sec), np.array(r32.d_sec)
    assert np.all(np.abs(d32 - d64) <= 1e-6 * d64), (d32, d64)
    dk = checks.section_diameters(P2, F, pt[0], 2)
    assert np.all(np.abs(d64 - dk) <= 1e-8 * dk), (d64, dk)


def test_two_sections_batched_equal_single_and_graph_replay(B):
    sizes = [7, 1, 33, 12]
    feeds = ai.batched_feeds(sizes, seed=21)
    rb = B.Batch(P2, feeds).ipm_solve(B.default_options())
    for F, r in zip(feeds, rb):
        rs = B.Problem(P2, F).ipm_solve(B.default_options())
        assert r.status == rs.status == 0, (r.status, rs.status)
        assert r.iters == rs.iters and list(r.d_sec) == list(rs.d_sec)
    prob = B.Problem(P2, feeds[2])
    runs = [prob.ipm_solve(B.default_options(graphs=g)) for g in (0, 1, 1, 1)]
    assert runs[-1].graph_replays >= 1
    for r in runs[1:]:
        assert r.status == 0 and r.iters == runs[0].iters and list(r.d_sec) == list(runs[0].d_sec)


def test_entry_points_without_sections_refuse_them(B):
    import torch
    F = ai.make_feeds(3, 0)
    prob = B.Problem(P2, F)
    assert prob.ipm_solve(B.default_options(kkt=1)).status == -1
    x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    jac = torch.zeros(prob.sizes.nnzJ_scen * prob.ld, dtype=torch.float64, device="cuda")
    hes = torch.zeros(prob.sizes.nnzH_scen * prob.ld, dtype=torch.float64, device="cuda")
    with pytest.raises(B.AbsorberError) as e:
        prob.kkt_factor(x, jac, hes, torch.ones_like(x))
    assert e.value.status == -1
    with pytest.raises(B.AbsorberError):
        B.Problem(dict(ai.PARAMS, n_sections=3), F)
