"""Second-order AD (oracle/ad.py) against closed-form derivatives."""
import numpy as np

from oracle.ad import Jet, jexp, jlog


def test_jet_closed_forms():
    rng = np.random.default_rng(0)
    a = rng.uniform(0.5, 2.0, 50)
    b = rng.uniform(0.5, 2.0, 50)
    x = Jet.variable(a, 0, 2)
    y = Jet.variable(b, 1, 2)
    # f = x^2 y / log(1 + y) + exp(x y) - 3 / x
    f = x * x * y / jlog(1.0 + y) + jexp(x * y) - 3.0 / x
    lg = np.log(1 + b)
    e = np.exp(a * b)
    fx = 2 * a * b / lg + b * e + 3 / a ** 2
    fy = a * a * (1 / lg - b / ((1 + b) * lg ** 2)) + a * e
    fxx = 2 * b / lg + b * b * e - 6 / a ** 3
    fxy = 2 * a * (1 / lg - b / ((1 + b) * lg ** 2)) + e + a * b * e
    # d/dy [1/lg - b/((1+b) lg^2)]
    g1 = -1 / ((1 + b) * lg ** 2)
    g2 = -(1 / ((1 + b) * lg ** 2)) + b / ((1 + b) ** 2 * lg ** 2) + 2 * b / ((1 + b) ** 2 * lg ** 3)
    fyy = a * a * (g1 + g2) + a * a * e
    np.testing.assert_allclose(f.v, a * a * b / lg + e - 3 / a, rtol=1e-14)
    np.testing.assert_allclose(f.g[:, 0], fx, rtol=1e-13)
    np.testing.assert_allclose(f.g[:, 1], fy, rtol=1e-13)
    np.testing.assert_allclose(f.h[:, 0, 0], fxx, rtol=1e-12)
    np.testing.assert_allclose(f.h[:, 0, 1], fxy, rtol=1e-12)
    np.testing.assert_allclose(f.h[:, 1, 0], fxy, rtol=1e-12)
    np.testing.assert_allclose(f.h[:, 1, 1], fyy, rtol=1e-12)


def test_jet_inactive_seed_is_constant():
    x = Jet.variable(np.array([1.0, 2.0]), 0, 1, active=np.array([True, False]))
    f = jexp(x) * x
    assert f.g[1, 0] == 0.0 and f.h[1, 0, 0] == 0.0
    np.testing.assert_allclose(f.h[0, 0, 0], 3 * np.e, rtol=1e-14)
