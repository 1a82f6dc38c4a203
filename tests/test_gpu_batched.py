"""Batched solves (many independent design problems in one engine run) on the GPU.

A problem solved inside a batch runs the same method as when solved alone: every
per-problem quantity (sums, maxima, the Schur scalar on d, the filter, mu) is reduced
over that problem's own scenarios only, in the same order.  So the batched result of
each problem must equal its single-problem solve (which the parity tests pin to the
oracle); the uneven 64-problem batch is checked by properties that fix the optimum:
d* equals the largest hydraulic volume over the problem's scenarios, and the states
solve each scenario's square MESH system."""
import numpy as np
import pytest

import absorber_inputs as ai
from oracle import checks, model

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


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _solve_batch(B, feeds, prec=0, **kw):
    import torch
    probs = [B.Problem(P, F) for F in feeds]
    xs = [torch.zeros(p.n_primal, dtype=torch.float64, device="cuda") for p in probs]
    o = B.default_options(precision=prec, max_refine=(0 if prec == 0 else 8), **kw)
    res = B.ipm_solve_batched(probs, o, x_out=xs)
    return probs, res, [p.from_soa(_host(x)) for p, x in zip(probs, xs)]


def _solve_single(B, F, prec=0):
    import torch
    prob = B.Problem(P, F)
    x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    o = B.default_options(precision=prec, max_refine=(0 if prec == 0 else 8))
    res = prob.ipm_solve(o, x_out=x)
    return res, prob.from_soa(_host(x))


def test_batched_equals_single_fp64(B):
    # ragged sizes: a one-scenario problem, sizes below and across a 32-slot tile
    sizes = [7, 1, 33, 12, 64]
    feeds = ai.batched_feeds(sizes, seed=21)
    probs, res, sol = _solve_batch(B, feeds)
    for p, F in enumerate(feeds):
        rs, (Zs, ds) = _solve_single(B, F)
        rb = res[p]
        Zb, db = sol[p]
        assert rs.status == 0 and rb.status == 0, (p, rs.status, rb.status)
        assert rb.iters == rs.iters and rb.base_iters == rs.base_iters, (p, rb.iters, rs.iters)
        assert abs(db - ds) <= 1e-12 * ds and abs(rb.d - db) == 0.0
        assert np.max(np.abs(Zb - Zs) / np.maximum(1.0, np.abs(Zs))) <= 1e-10
        assert rb.E0 <= 1e-8


def test_batched_fp32_mixed(B):
    sizes = [20, 45, 3]
    feeds = ai.batched_feeds(sizes, seed=22)
    probs, res, sol = _solve_batch(B, feeds, prec=1)
    for p, F in enumerate(feeds):
        rs, (Zs, ds) = _solve_single(B, F, prec=0)
        assert res[p].status == 0 and res[p].E0 <= 1e-8
        assert abs(res[p].d - ds) <= 1e-6 * ds


def test_batched_one_problem_is_ipm_solve(B):
    F = ai.make_feeds(10, 0)
    probs, res, sol = _solve_batch(B, [F])
    rs, (Zs, ds) = _solve_single(B, F)
    assert res[0].status == 0 and res[0].iters == rs.iters
    assert abs(res[0].d - rs.d) <= 1e-12 * rs.d


def test_batched_status_per_problem(B):
    # an iteration limit that stops the larger problem only: each problem keeps its own
    # outcome and the finished one its solution
    sizes = [1, 40]
    feeds = ai.batched_feeds(sizes, seed=23)
    r1, _ = _solve_single(B, feeds[0])
    probs, res, sol = _solve_batch(B, feeds, max_iter=r1.iters)
    assert res[0].status == 0 and res[0].iters == r1.iters
    assert res[1].status == -6


def test_batched_64_uneven_problems(B):
    sizes = ai.batched_sizes()
    feeds = ai.batched_feeds(sizes, seed=3)
    probs, res, sol = _solve_batch(B, feeds, prec=1)
    assert [r.status for r in res] == [0] * len(sizes)
    assert max(r.E0 for r in res) <= 1e-8
    rng = np.random.default_rng(5)
    for p, F in enumerate(feeds):
        Z, d = sol[p]
        dmin, vol = checks.minimum_diameter(P, F, Z)
        assert abs(d - dmin) <= 1e-8 * dmin, p
    # sampled scenarios of a few problems are roots of their square MESH systems
    keep = np.ones(model.NS, dtype=bool)
    keep[model.NV - 1::model.NV] = False
    for p in rng.choice(len(sizes), 3, replace=False):
        Z, d = sol[p]
        F = feeds[p]
        pick = rng.choice(F.shape[1], min(4, F.shape[1]), replace=False)
        Zn, hist = checks.mesh_newton(P, F[:, pick], Z[pick], d, iters=5)
        assert hist[-1] <= 1e-12
        assert np.max(np.abs(Zn[:, keep] - Z[pick][:, keep]) / np.maximum(1, np.abs(Zn[:, keep]))) <= 1e-6


def test_autotuned_tiles_give_identical_results(B):
    # the tile autotuner only regroups warps (one scenario per warp): the solve is the
    # same bit for bit with the tuned shapes and with the default shape
    import torch
    F = ai.make_feeds(600, 1)
    prob = B.Problem(P, F)
    outs = []
    for tune in (0, 1, 1):
        x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
        o = B.default_options(precision=1, max_refine=8, autotune=tune)
        r = prob.ipm_solve(o, x_out=x)
        assert r.status == 0, (tune, r.status, prob.last_error())
        outs.append((r.iters, r.d, _host(x), list(r.tiles)))
    assert outs[0][0] == outs[1][0] == outs[2][0]
    assert outs[0][1] == outs[1][1] == outs[2][1]
    assert np.array_equal(outs[0][2], outs[1][2]) and np.array_equal(outs[1][2], outs[2][2])
    assert outs[0][3] == [4, 4, 4, 4]
    assert all(w in (1, 2, 4, 8) for w in outs[2][3][1:])
    assert outs[2][3][0] in (1, 2, 4, 8)


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_gives_identical_results(B, prec):
    # a whole solve replayed from its captured CUDA graph (conditional nodes for the
    # iteration, refinement and line-search loops; the decisions taken by the control
    # kernels on the device) runs the same kernels with the same arguments as the eager
    # run, whose conditions the host reads back: the same solve bit for bit, the same
    # number of kernel launches, one graph launch per solve (the expected-value start's
    # run is a second one)
    import torch
    F = ai.make_feeds(300, 1)
    prob = B.Problem(P, F)
    outs = []
    for graphs in (0, 1, 1, 1):
        x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
        o = B.default_options(precision=prec, max_refine=(8 if prec else 0), graphs=graphs)
        r = prob.ipm_solve(o, x_out=x)
        assert r.status == 0
        outs.append((r.iters, r.d, _host(x), r.graph_replays, r.launches, r.base_iters))
    eager = outs[0]
    assert eager[3] == 0
    assert outs[1][3] == 0                       # the first run of a configuration is eager
    for o in outs[2:]:
        assert o[3] == 2                         # expected-value start + the solve
        assert o[0] == eager[0] and o[1] == eager[1] and o[5] == eager[5]
        assert np.array_equal(o[2], eager[2])
        # launches counted on the device equal the host's count of an eager run (the
        # very first solve also times the tile candidates: compare with the second)
        assert o[4] == outs[1][4], (o[4], outs[1][4])


@pytest.mark.parametrize("S", [37, 600])
def test_every_fp32_factor_shape_gives_identical_results(B, S):
    # the FP32 factor runs one scenario per warp: every launch shape gives the same solve
    # bit for bit
    import torch
    F = ai.make_feeds(S, 2)
    prob = B.Problem(P, F)
    outs = []
    for tile in (4, 1, 2, 8):
        x = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
        o = B.default_options(precision=1, max_refine=8, factor_tile=tile)
        r = prob.ipm_solve(o, x_out=x)
        assert r.status == 0, (tile, r.status)
        assert r.tiles[0] == tile
        outs.append((r.iters, r.d, _host(x)))
    for t, o in zip((1, 2, 8), outs[1:]):
        assert o[0] == outs[0][0] and o[1] == outs[0][1], t
        assert np.array_equal(o[2], outs[0][2]), t
