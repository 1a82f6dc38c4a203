"""The pressure relation (7) with a specified drop per stage on the GPU
(abs_params.dp_stage: stage n at P + (9 - n) dP): the evaluation, the start and the
solve use each stage's pressure.  Checked against the oracle (P["dp_stage"], pinned on
the CPU): the diameter of its solve, the closed form from the GPU's states with the
stage pressures, E_0 <= 1e-8 recomputed by the oracle at the GPU's point; and with two
column sections at once."""
import numpy as np
import pytest

import absorber_inputs as ai
from oracle import checks, ipm

pytestmark = pytest.mark.gpu
PD = dict(ai.PARAMS, dp_stage=0.005)   # 5 mbar per stage


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


def _point(B, prob, opt):
    import torch
    x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    y = torch.zeros(prob.n_row, dtype=torch.float64, device="cuda")
    res = prob.ipm_solve(opt, x_out=x, y_out=y)
    zl, zu = torch.zeros_like(x), torch.zeros_like(x)
    zd = prob.bound_multipliers(zl, zu)
    Z, d = prob.from_soa(host(x))
    lam, _ = prob.from_soa(host(y))
    K = prob.K
    return res, Z, d, lam, prob.from_soa(host(zl))[0], prob.from_soa(host(zu))[0], zd[:K], zd[K:]


def test_pressure_drop_matches_the_oracle_s10(B):
    F = ai.make_feeds(10, 0)
    ro = ipm.solve(PD, F)
    assert ro.status == "ok"
    prob = B.Problem(PD, F)
    res, Z, d, lam, ZL, ZU, zld, zud = _point(B, prob, B.default_options())
    assert res.status == 0 and abs(res.d - ro.d) <= 1e-6 * ro.d, (res.d, ro.d)
    dmin, _ = checks.minimum_diameter(PD, F, Z)
    assert abs(res.d - dmin) <= 1e-8 * dmin
    assert checks.kkt_error(PD, F, d, Z, lam, ZL, ZU, float(zld[0]), float(zud[0])) <= 1e-8
    r0 = B.Problem(ai.PARAMS, F).ipm_solve(B.default_options())
    assert r0.status == 0 and r0.d != res.d


def test_pressure_drop_with_two_sections(B):
    P2 = dict(PD, n_sections=2)
    F = ai.make_feeds(4, 0)
    ro = ipm.solve(P2, F)
    prob = B.Problem(P2, F)
    res, Z, d, lam, ZL, ZU, zld, zud = _point(B, prob, B.default_options(precision=1, max_refine=8))
    assert ro.status == "ok" and res.status == 0
    dsec = np.array(res.d_sec)
    assert np.all(np.abs(dsec - ro.d) <= 1e-6 * ro.d), (dsec, ro.d)
    dk = checks.section_diameters(P2, F, Z, 2)
    assert np.all(np.abs(dsec - dk) <= 1e-8 * dk)
    assert checks.kkt_error(P2, F, dsec, Z, lam, ZL, ZU, zld, zud) <= 1e-8
