"""Oracle pins for the pressure relation (7) with a specified drop per stage,
P_n = P_top + (N - 1 - n) dP (the top stage at the scenario's absorber pressure).

Pressure is data here, so the MESH blocks stay square and the states at the optimum fix
the diameter: d* = max over scenarios and stages of sqrt(4 V R T / (pi u_max P_n)) with
each stage's own pressure; dP = 0 is the case study."""
import math

import numpy as np

import absorber_inputs as ai
from oracle import checks, ipm, model

P0 = ai.PARAMS
PD = dict(ai.PARAMS, dp_stage=0.01)


def test_stage_pressures_follow_relation_7():
    F = ai.make_feeds(3, 0)
    pr = model.stage_pressures(PD, F)
    assert pr.shape == (3, model.N)
    assert np.allclose(pr[:, model.N - 1], F[model.FEED["P"]])
    assert np.allclose(pr[:, :-1] - pr[:, 1:], 0.01)
    assert np.array_equal(model.stage_pressures(P0, F), np.repeat(F[model.FEED["P"]][:, None], model.N, axis=1))


def test_pressure_drop_optimum_is_the_closed_form():
    F = ai.make_feeds(3, 0)
    r = ipm.solve(PD, F)
    assert r.status == "ok"
    dmin, vol = checks.minimum_diameter(PD, F, r.Z)
    assert abs(r.d - dmin) <= 1e-8 * dmin
    # the volumes use each stage's pressure (relation (7)), not the absorber pressure
    Zs = r.Z.reshape(3, model.N, model.NV)
    v_abs = Zs[:, :, model.IV] * PD["R"] * PD["sT"] * Zs[:, :, model.IT] / F[model.FEED["P"]][:, None]
    assert np.all(vol[:, :-1] < v_abs[:, :-1]) and np.allclose(vol[:, -1], v_abs[:, -1])
    assert checks.kkt_error(PD, F, r.d, r.Z, r.lam, r.zL, r.zU, r.zLd, r.zUd) <= 1e-8
    r0 = ipm.solve(P0, F)
    assert r0.status == "ok" and r.d != r0.d
