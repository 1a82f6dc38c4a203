"""Oracle model (oracle/model.py): structure pinned to the paper's printed problem size,
derivatives pinned to complex step, structural properties the equations fix."""
import math
import os

import numpy as np
import pytest

import absorber_inputs as ai
from oracle import checks, model

P = ai.PARAMS
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_problem_size.txt")


def _random_interior(S, seed):
    rng = np.random.default_rng(seed)
    F = ai.make_feeds(S, seed)
    Z, d = model.initial_point(P, F)
    Z = Z.reshape(S, model.N, model.NV)
    Z[:, :, :13] = Z[:, :, :13] * rng.uniform(0.5, 1.5, Z[:, :, :13].shape) + 0.05
    Z[:, :, model.IL] *= rng.uniform(0.9, 1.1, (S, model.N))
    Z[:, :, model.IV] *= rng.uniform(0.9, 1.1, (S, model.N))
    Z[:, :, model.IT] = rng.uniform(3.1, 3.5, (S, model.N))
    Z[:, :, model.IE:model.IE + 5] = rng.normal(0, 1e-3, (S, model.N, 5))
    Z[:, :, model.IS] = rng.uniform(0.1, 2.0, (S, model.N))
    return F, Z.reshape(S, model.NS), 1.3 + 0.1 * seed, rng.standard_normal((S, model.NS))


def test_problem_size_matches_paper():
    vals = [int(v) for v in open(GOLDEN).read().split("\n")[-2].split()]
    S, nvar, nmesh, nfix, nhyd = vals
    assert model.problem_size(S) == (nvar, nmesh, nfix, nhyd)
    # after eliminating the fixings and adding one slack per hydraulic row, each scenario
    # block is square: 220 unknowns, 220 rows
    per = model.problem_size(1)
    assert (per[0] - 1) - per[2] + per[3] == model.NS
    assert per[1] + per[3] == model.NS


def test_jacobian_matches_complex_step():
    F, Z, d, lam = _random_interior(2, 1)
    C, J, Jd, W, Wdd = model.derivatives(P, F, Z, d, lam)
    Jc, Jdc = checks.jacobian_complex_step(P, F, Z, d)
    scale = np.abs(Jc).max()
    assert np.abs(J - Jc).max() <= 1e-13 * scale
    assert np.abs(Jd - Jdc).max() <= 1e-13 * np.abs(Jdc).max()
    np.testing.assert_allclose(C, model.residuals(P, F, Z, d), rtol=0, atol=1e-13)


def test_hessian_matches_fd_of_complex_step_gradient():
    F, Z, d, lam = _random_interior(1, 2)
    _, _, _, W, Wdd = model.derivatives(P, F, Z, d, lam)
    h = 1e-6
    rng = np.random.default_rng(3)
    cols = rng.choice(model.NS, 30, replace=False)
    for j in cols:
        hj = h * max(1.0, abs(Z[0, j]))
        Zp, Zm = Z.copy(), Z.copy()
        Zp[0, j] += hj
        Zm[0, j] -= hj
        fd = (checks.lagrangian_gradient_cs(P, F, Zp, d, lam)
              - checks.lagrangian_gradient_cs(P, F, Zm, d, lam)) / (2 * hj)
        assert np.abs(fd[0] - W[0, :, j]).max() <= 1e-6 * (1 + np.abs(W[0, :, j]).max())
    # d-d entry: -u_max pi / 2 times the hydraulic multipliers
    hyd = np.arange(model.NV - 1, model.NS, model.NV)
    assert abs(Wdd[0] - (-P["u_max"] * math.pi / 2) * lam[0, hyd].sum()) <= 1e-12 * abs(Wdd[0])


def test_structure_stage_local_hessian_and_d_column():
    F, Z, d, lam = _random_interior(1, 4)
    _, J, Jd, W, _ = model.derivatives(P, F, Z, d, lam)
    blocks = np.arange(model.NS) // model.NV
    # Lagrangian Hessian is block diagonal by stage
    cross = blocks[:, None] != blocks[None, :]
    assert np.all(W[0][cross] == 0.0)
    assert np.abs(W[0] - W[0].T).max() <= 1e-12 * np.abs(W[0]).max()
    # the Jacobian is block tridiagonal by stage
    far = np.abs(blocks[:, None] - blocks[None, :]) > 1
    assert np.all(J[0][far] == 0.0)
    # d enters only the hydraulic rows, with dc/dd = -u_max pi d / 2
    hyd = np.arange(model.NV - 1, model.NS, model.NV)
    nz = np.nonzero(Jd[0])[0]
    np.testing.assert_array_equal(nz, hyd)
    np.testing.assert_allclose(Jd[0, hyd], -P["u_max"] * math.pi * d / 2, rtol=1e-15)


def test_pattern_invariant_under_scenario_permutation():
    F, Z, d, lam = _random_interior(3, 5)
    _, J, _, W, _ = model.derivatives(P, F, Z, d, lam)
    perm = [2, 0, 1]
    _, J2, _, W2, _ = model.derivatives(P, F[:, perm], Z[perm], d, lam[perm])
    for s in range(3):
        np.testing.assert_array_equal(J[perm[s]] != 0, J2[s] != 0)
        np.testing.assert_array_equal(W[perm[s]] != 0, W2[s] != 0)
        np.testing.assert_array_equal(J[s] != 0, J[0] != 0)


def test_mesh_block_square_and_nonsingular():
    F, Z, d, lam = _random_interior(1, 6)
    _, J, _, _, _ = model.derivatives(P, F, Z, d, lam, rows_only=True)
    keep = np.ones(model.NS, dtype=bool)
    keep[model.NV - 1::model.NV] = False
    A = J[0][np.ix_(keep, keep)]
    assert A.shape == (210, 210)
    assert np.linalg.matrix_rank(A) == 210
