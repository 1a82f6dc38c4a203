"""Scenario partition of one problem across ranks: the sharding the problem's structure
allows (only d couples the scenarios, Section "Replicated scenario structure").

k oracle instances each hold a contiguous slice of the scenarios.  Each factors its own
scenario blocks (oracle/kkt.py BlockLDL, dense Bunch-Kaufman) and contributes, to one
exchange in fixed rank order, the three coupling sums of its slice: sum_s bh_s^T u_s
(u_s = K_s^-1 bh_s, the Schur scalar's part), sum_s bh_s^T v_s (v_s = K_s^-1 r_s, the d
row's right-hand side) and its inertia counts.  Every rank then forms the same S_d and dd
and back-substitutes its own scenarios.  Checked against the unsplit oracle (SchurKKT):
S_d, dd and every slice's direction to 1e-12 relative (summation order only), the inertia
exactly; and the minimum diameter -- the max over the slices of each slice's largest
hydraulic volume -- equals the unsplit one at the oracle's solution.  Two and three gloo
ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import absorber_inputs as ai

P = ai.PARAMS
S_PROB, SEED = 7, 0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _system(iters):
    """The oracle's iterate after `iters` iterations of the 7-scenario problem and its
    Newton system (matrices per scenario, right-hand sides), deterministic on every rank."""
    from oracle import ipm
    F = ai.make_feeds(S_PROB, SEED)
    solver = ipm.IPM(P, F)
    r = ipm.IPM(P, F, ipm.Options(max_iter=iters)).solve()
    st, mu = solver.state_from_result(r), r.mu
    C, J, Jd, W, Wdd = solver.evaluate(st)
    sig, sigd = solver.sigma(st)
    gz, gd = solver.barrier_gradient(st, mu)
    rz = -(gz + np.einsum("src,sr->sc", J, st.lam))
    rd = -(gd + float(np.sum(Jd * st.lam)))
    Kdd = float(np.sum(Wdd)) + sigd
    return F, W, sig, J, Jd, Kdd, rz, rd, -C


def _slice(rank, world):
    lo = (S_PROB * rank) // world
    hi = (S_PROB * (rank + 1)) // world
    return lo, hi


def _rank(rank, world, port, dw, dc, q):
    import torch
    import torch.distributed as dist
    from oracle import checks, ipm, kkt
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        F, W, sig, J, Jd, Kdd, rz, rd, rc = _system(4)
        lo, hi = _slice(rank, world)
        n = W.shape[1]
        U, V = [], []
        sbu = sbv = 0.0
        cnt = np.zeros(3)
        for s in range(lo, hi):
            f = kkt.BlockLDL(kkt.scenario_matrix(W[s], sig[s], J[s], dw, dc))
            cnt += f.inertia()
            bh = np.concatenate([np.zeros(n), Jd[s]])
            u = f.solve(bh)
            v = f.solve(np.concatenate([rz[s], rc[s]]))
            U.append(u)
            V.append(v)
            sbu += float(bh @ u)
            sbv += float(bh @ v)
        # one exchange: every rank's three sums, combined in rank order on every rank
        mine = torch.tensor([sbu, sbv, *cnt], dtype=torch.float64)
        allv = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(allv, mine)
        tot = allv[0].clone()
        for t in allv[1:]:
            tot += t
        Sd = (Kdd + dw) - float(tot[0])
        dd = (rd - float(tot[1])) / Sd
        X = np.array(V) - np.array(U) * dd
        inert = [int(tot[2]), int(tot[3]), int(tot[4])]
        inert[0 if Sd > 0 else (1 if Sd < 0 else 2)] += 1
        # the minimum diameter at the oracle's solution: max over the slices
        sol = ipm.solve(P, F)
        _, vol = checks.minimum_diameter(P, F[:, lo:hi], sol.Z[lo:hi])
        vmax = torch.tensor([float(vol.max())], dtype=torch.float64)
        dist.all_reduce(vmax, op=dist.ReduceOp.MAX)
        q.put((rank, lo, hi, Sd, dd, X, tuple(inert), float(vmax[0])))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,dw,dc", [(2, 0.0, 0.0), (3, 1e-4, 1e-8)])
def test_partitioned_newton_direction_equals_unsplit(world, dw, dc):
    import math
    from oracle import checks, ipm, kkt
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, dw, dc, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=600) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    F, W, sig, J, Jd, Kdd, rz, rd, rc = _system(4)
    fac = kkt.SchurKKT(W, sig, J, Jd, Kdd, dw, dc)
    dz, dd, dl = fac.solve(rz, rd, rc)
    n = W.shape[1]
    sol = ipm.solve(P, F)
    assert sol.status == "ok"
    dmin, _ = checks.minimum_diameter(P, F, sol.Z)
    assert abs(dmin - sol.d) <= 1e-8 * sol.d
    for rank, lo, hi, Sd, dd_r, X, inert, vmax in out:
        assert abs(Sd - fac.Sd) <= 1e-12 * abs(fac.Sd)
        assert abs(dd_r - dd) <= 1e-12 * abs(dd)
        ref = np.concatenate([dz[lo:hi], dl[lo:hi]], axis=1)
        got = np.concatenate([X[:, :n], X[:, n:]], axis=1)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        assert inert == fac.inertia()
        assert math.sqrt(4.0 * vmax / (math.pi * P["u_max"])) == dmin
