"""Planted mistakes in the oracle (on the CPU only) must be caught by its pins: a wrong
stoichiometric coefficient breaks conservation, a wrong derivative rule breaks the
complex-step comparison, a wrong stage index breaks the element balance."""
import numpy as np
import pytest

import absorber_inputs as ai
from oracle import ad, checks, ipm, model

P = ai.PARAMS


def _solution_balances_ok(F, r):
    if r.status != "ok":
        return False
    el_in, el_out, h_in, h_out = checks.column_balances(P, F, r.Z)
    return np.allclose(el_out, el_in, rtol=0, atol=1e-8 * np.abs(el_in).max())


def test_wrong_stoichiometry_is_caught(monkeypatch):
    F = ai.make_feeds(1, 0)
    nu = model.NU.copy()
    nu[8, 3] = 0.0          # drop H2O from R4 (carbamate reversion)
    monkeypatch.setattr(model, "NU", nu)
    r = ipm.solve(P, F, ipm.Options(max_iter=80))
    assert not _solution_balances_ok(F, r)


def test_wrong_product_rule_is_caught(monkeypatch):
    def bad_mul(self, o):
        if isinstance(o, ad.Jet):
            v = self.v * o.v
            g = self.g * o.v[:, None]          # forgot the o.g * self.v term
            h = self.h * o.v[:, None, None]
            return ad.Jet(v, g, h)
        return ad.Jet(self.v * o, self.g * np.asarray(o)[..., None] if np.ndim(o) else self.g * o,
                      self.h * (np.asarray(o)[..., None, None] if np.ndim(o) else o))
    F = ai.make_feeds(1, 1)
    Z, d = model.initial_point(P, F)
    Z = np.abs(Z) + 0.1
    monkeypatch.setattr(ad.Jet, "__mul__", bad_mul)
    monkeypatch.setattr(ad.Jet, "__rmul__", bad_mul)
    _, J, _, _, _ = model.derivatives(P, F, Z, d, np.ones_like(Z), rows_only=True)
    monkeypatch.undo()
    Jc, _ = checks.jacobian_complex_step(P, F, Z, d)
    assert np.abs(J - Jc).max() > 1e-6 * np.abs(Jc).max()


def test_wrong_neighbour_index_is_caught(monkeypatch):
    F = ai.make_feeds(1, 2)
    orig = model.local_to_scenario

    def shifted(n):
        m = orig(n)
        if n + 1 < model.N:                      # liquid from above read two stages up
            m[model.A_L] = model.NV * min(n + 2, model.N - 1) + model.IL
        return m
    monkeypatch.setattr(model, "local_to_scenario", shifted)
    Z, d = model.initial_point(P, F)
    Z = np.abs(Z) + 0.1
    _, J, _, _, _ = model.derivatives(P, F, Z, d, np.ones_like(Z), rows_only=True)
    monkeypatch.undo()
    Jc, _ = checks.jacobian_complex_step(P, F, Z, d)
    assert np.abs(J - Jc).max() > 1e-6 * np.abs(Jc).max()
