#!/usr/bin/env python
"""Benchmark: Newton steps/s and solve time of the interior-point solve of the
5000-scenario absorber design problem (seeded truncated-normal feeds, sigma 5 %, cut at
+-15 %, seed 2) on the GB300 path at KKT tolerance E_0 <= 1e-8, against the FP64 GPU
path.

One "step" is one full interior-point solve to E_0 <= 1e-8: every Newton iteration runs
the whole hot path (fused evaluation, block-LU factorization, Schur complement on d,
block solves, refinement, line search).  The timed form (--form) defaults to FP32 block
factors with FP64 refinement from the learned warm start (the network is trained once
in the run, untimed, on 20,000 single-scenario solves); the other forms -- the plain FP64
path from the default start among them -- are timed alongside under "forms".
value = Newton iterations of the K timed solves / their device time.  Prints one JSON
line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--form learned-fp32|learned-fp64|fp32|fp64] [--workload NAME]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Newton steps/s & solve time, 5000-scenario absorber, vs FP64 GPU path at 1e-8"
UNIT = "Newton steps/s"
DEFAULT_WORKLOAD = "absorber-S5000-tn5-seed2"
# Algorithmic work per scenario and launch.  Bytes: the values a launch must read and
# write once (Jacobian 1497 and Hessian 661 entries, 220-entry vectors, factors of 10
# stage blocks: 22 x 22 LU or inverse, 22 x 11 G for 9 stages, 44 bytes of row order).
# Flops: FP64 factor = block LU (7183 per stage) + G = At^-1 B (10406 per stage with B);
# FP32 factor = Gauss-Jordan exchanges (22 steps x 21 rows x 32 columns x 2 + the pivot
# row's 33 products, 22 columns without B on the last stage); a block solve applies a
# 22 x 22 factor (968), the coupling (28) and G (484) per stage and right-hand side.
EVAL_BYTES_PER_SCEN = 8 * (220 + 220 + 18 + 220 + 1497 + 661)    # read x, lambda, feed; write c, J, H
# FP64 flops of one evaluation, per scenario, from the kernels' executed FP64 instructions
# (one ncu capture at 5000 scenarios: DFMA 26.875e6, DMUL 28.27e6, DADD 12.775e6 thread
# instructions for the full evaluation; DFMA 16.59e6, DMUL 7.775e6, DADD 8.6e6 for the
# trial evaluation), a fused multiply-add counted as two
EVAL_FP64_FLOPS_PER_SCEN = (2 * 26.875e6 + 28.27e6 + 12.775e6) / 5000
TRIAL_FP64_FLOPS_PER_SCEN = (2 * 16.59e6 + 7.775e6 + 8.6e6) / 5000
TRIAL_BYTES_PER_SCEN = 8 * (2 * 220 + 18)                         # read x, dx, feed
FACTOR_FLOPS_PER_SCEN = {8: 10 * 7183 + 9 * 10406,                # FP64: stage LUs + G
                         4: 9 * 22 * (21 * 32 * 2 + 33) + 22 * (21 * 21 * 2 + 22)}   # FP32: Gauss-Jordan
SOLVE_FLOPS_PER_SCEN_RHS = 10 * (28 + 968 + 484)                  # coupling + block apply + G product
SOLVE_T_FLOPS_PER_SCEN = 10 * (484 + 968 + 28)                    # G^T product + transposed apply + coupling
PIV_BYTES_PER_SCEN = 10 * 44
# Algorithmic bytes per scenario and launch of every other kernel kind (abs_result.kind_launches,
# binding.KINDS): the vectors (220 doubles per scenario), Jacobian (1497) and Hessian (661)
# values each reads and writes once.  Reductions count planes (10 stage partials each).
V220 = 8 * 220
KIND_BYTES = {
    "eval_trial": 8 * (2 * 220 + 18) + V220,          # x, dx, feed; c
    "residual": 8 * 1497 + 7 * V220,                  # J; g, dl', dz, r_z, r_c; rho_z, rho_c
    "schur": 8 * 661 + 4.5 * V220,                    # H; sigma, q, p, r (half the launches); t or Hq
    "dual": 8 * 1497 + 5 * V220,                      # J; lambda, x, zL, zU; J^T lambda
    "reduce_planes": 8 * 10,                          # one stage partial per scenario and plane
    "rhs": 10 * V220,                                 # x, zL, zU, J^T l, c; Sigma, r_z, r_c, 1/s_L, 1/s_U
    "dz": 6 * V220,                                   # p, q, t, Hq; dz, g
    "step": 8 * V220,                                 # x, dz, zL, zU, 1/s_L, 1/s_U; dzL, dzU
    "accept": 12 * V220,                              # x, dz, lambda, dl, zL, dzL, zU, dzU; x, lambda, zL, zU
    "vector": 3 * V220,                               # axpby-like: two vectors in, one out
    "control": 0,
    "eval_jac": 8 * (2 * 220 + 18) + V220 + 8 * 1497, # x, lambda, feed; c, J
}


# DRAM bytes (read + write) per launch of the timed form's largest kernel, from one ncu
# capture of the 5000-scenario workload (summarised with the profiles), keyed by (kernel,
# element size) with the sha256 of the kernel source at capture: reported only while the
# source is unchanged
CAPTURED_TRAFFIC = {
    ("factor", 4): (146.073088e6, "8d0df1be6db130255886ce9808ab33651ac880e48082b1634cac8a808c94f246"),
}


def captured_traffic(kernel, es, S):
    import hashlib
    ent = CAPTURED_TRAFFIC.get((kernel, es))
    if ent is None or S != 5000:
        return None
    src = os.path.join(ROOT, "paper_2607_15420_gb300", "csrc", "kernels_warp.cuh")
    with open(src, "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != ent[1]:
            return None
    return ent[0]


def factor_bytes(es):
    return es * (4840 + 9 * 242) + 8 * 1497 + PIV_BYTES_PER_SCEN


def solve_bytes(es, nrhs):
    return es * (4840 + 9 * 242) + PIV_BYTES_PER_SCEN + 8 * 300 + nrhs * 8 * 2 * 220


def solve_t_bytes(es):
    return es * (4840 + 9 * 242) + PIV_BYTES_PER_SCEN + 8 * 300 + 8 * 2 * 220


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(workload, sample_scen, iters, timeout=600):
    """The oracle as it stands on the host cores: `iters` interior-point iterations on the
    first `sample_scen` scenarios of the workload, one thread, in a fresh process."""
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import absorber_inputs as ai
from oracle import ipm
F = ai.workload_feeds({workload!r})[:, :{sample_scen}]
opt = ipm.Options(max_iter={iters}, init="inlet")
t = time.perf_counter()
r = ipm.solve(ai.PARAMS, F, opt)
el = time.perf_counter() - t
print(json.dumps(dict(iters=r.iters, seconds=el)))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def visible_cores():
    """(nproc as the OS reports it, CPUs this process may run on)."""
    n = os.cpu_count() or 1
    try:
        a = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        a = n
    return n, a


def cpu_baseline_all_cores(workload, per_proc, iters, nproc, timeout=600):
    """The oracle on every visible core: nproc single-threaded processes at once, process
    k running `iters` interior-point iterations on its own block of `per_proc` scenarios
    (scenarios k*per_proc ...) as an independent problem -- the scenario-parallel part
    of an iteration; the scalar reductions that join the blocks are not timed."""
    code = """
import json, sys, time
sys.path.insert(0, {root!r})
import absorber_inputs as ai
from oracle import ipm
k = int(sys.argv[1])
F = ai.workload_feeds({wl!r})[:, k * {pp}:(k + 1) * {pp}]
opt = ipm.Options(max_iter={it}, init="inlet")
t = time.perf_counter()
r = ipm.solve(ai.PARAMS, F, opt)
print(json.dumps(dict(iters=r.iters, seconds=time.perf_counter() - t)))
""".format(root=ROOT, wl=workload, pp=per_proc, it=iters)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    t0 = time.perf_counter()
    procs = [subprocess.Popen([sys.executable, "-c", code, str(k)], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, env=env) for k in range(nproc)]
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=timeout)
        if p.returncode != 0:
            raise RuntimeError(e[-2000:])
        outs.append(json.loads(o.strip().splitlines()[-1]))
    wall = time.perf_counter() - t0
    return {"iters": min(o["iters"] for o in outs), "wall_s": wall,
            "per_process_s": [o["seconds"] for o in outs]}


def run_reference(args, S_full):
    """Reference arm: the CPU oracle, timed on the host cores, one bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sample, iters = 10, 2
    times, its = [], []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(args.workload, sample, iters)
        if k >= args.warmup:
            times.append(r["seconds"])
            its.append(r["iters"])
    tot = sum(times)
    value = sum(its) / tot * (sample / S_full)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / max(1, len(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded feeds)",
        "config": {"workload": args.workload, "scenarios": S_full, "tol": 1e-8,
                   "step": f"{iters} oracle IPM iterations on a {sample}-scenario sample, scaled by {sample}/{S_full}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "visible_cores": dict(zip(("nproc", "affinity"), visible_cores())),
                         "sample": f"{iters} IPM iterations on the first {sample} scenarios per step, "
                                   f"per-iteration cost scaled linearly to {S_full} scenarios"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def job_totals(t_local, iters_local, world, device):
    """Whole-job time and work of N replicas: the slowest rank's time, every rank's
    iterations (one all-reduce each; no collective on the data path)."""
    import torch
    if world <= 1:
        return t_local, iters_local
    import torch.distributed as dist
    t = torch.tensor([t_local, iters_local], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    isum = t.clone()
    dist.all_reduce(isum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(isum[1])


def timed(fn, reps):
    """Device time (CUDA events on the current stream) of reps calls of fn; returns
    (seconds per call, results)."""
    import torch
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    out = [fn() for _ in range(reps)]
    b.record(st)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / reps, out


FORMS = {"fp64": (0, False), "fp32": (1, False), "learned-fp64": (0, True), "learned-fp32": (1, True)}


def train_network(B, ai, n_train=20000, epochs=100):
    """The warm-start network, trained on n_train single-scenario solves (one batched
    solve from a shared expected-value start) by the library's own kernels."""
    import torch
    P = ai.PARAMS
    t0 = time.perf_counter()
    Ftr = ai.make_feeds(n_train, 7, stream=3)
    batch = B.Batch(P, [Ftr[:, i:i + 1] for i in range(n_train)])
    x = torch.zeros(batch.n_primal, dtype=torch.float64, device="cuda")
    y = torch.zeros(220 * batch.ld, dtype=torch.float64, device="cuda")
    res = batch.ipm_solve(B.default_options(init=2, obj_scaling=100.0), x_out=x, y_out=y)
    keep = [r.status == 0 for r in res]
    t_data = time.perf_counter() - t0
    X, Y = B.make_dataset(batch, x, y, keep=keep, n_aug=4, d_spread=0.15)
    net = B.MLP(seed=11)
    net.fit_normalization(X, Y)
    t1 = time.perf_counter()
    hist = net.train(X, Y, B.train_options(epochs=epochs, batch=256, lr=2e-3, lr_final=2e-5, seed=5))
    t_train = time.perf_counter() - t1
    info = {"single_scenario_solves": n_train, "converged": int(sum(keep)), "rows": int(X.shape[0]),
            "solve_s": t_data, "epochs": epochs, "train_s": t_train,
            "loss_first_last": [float(hist[0]), float(hist[-1])]}
    return net, info


FACTOR_TILE = 0   # --factor-tile: a fixed FP32 factor launch shape (0: autotuned)


def options(B, prec, profile=0, graphs=1):
    return B.default_options(precision=prec, max_refine=(8 if prec == B.PREC_FP32 else 0), profile=profile,
                             graphs=graphs, factor_tile=FACTOR_TILE)


def solve_form(B, prob, net, form, profile=0, graphs=1, x_out=None):
    prec, learned = FORMS[form]
    o = options(B, prec, profile, graphs)
    if learned:
        return B.ipm_solve_learned(prob, net, o, x_out=x_out)
    return prob.ipm_solve(o, x_out=x_out)


def compare_forms(B, prob, net, reps):
    """Every form on one problem, each after one untimed solve; solve time from CUDA
    events around reps solves."""
    out = {"scenarios": prob.S}
    for form in ("fp64", "fp32", "learned-fp64", "learned-fp32"):
        solve_form(B, prob, net, form)
        sec, rs = timed(lambda: solve_form(B, prob, net, form), reps)
        r = rs[0]
        out[form] = {"solve_time_s": sec, "iters": r.iters, "base_iters": r.base_iters, "status": r.status,
                     "E0": r.E0, "d": r.d, "fp64_fallbacks": r.fp64_fallbacks,
                     "learned_start_used": bool(r.warm_status) if FORMS[form][1] else None}
    base = out["fp64"]["solve_time_s"]
    for form in ("fp32", "learned-fp64", "learned-fp32"):
        out[form]["speedup_vs_fp64"] = base / out[form]["solve_time_s"]
    return out


def two_section_form(B, ai, P, reps):
    """The same 5000-scenario workload with a two-section column (a design vector of two
    diameters, 2 x 2 Schur complement): FP64 and FP32 + refinement from the default start,
    against the one-section solve of the same form."""
    F = ai.workload_feeds("absorber-S5000-tn5-seed2")
    out = {"scenarios": int(F.shape[1]), "n_sections": 2}
    for nsec in (1, 2):
        prob = B.Problem(dict(P, n_sections=nsec), F)
        for form, prec in (("fp64", B.PREC_FP64), ("fp32", B.PREC_FP32)):
            prob.ipm_solve(options(B, prec))
            sec, rs = timed(lambda: prob.ipm_solve(options(B, prec)), reps)
            r = rs[0]
            out[f"{form}-{nsec}-section"] = {"solve_time_s": sec, "iters": r.iters, "base_iters": r.base_iters,
                                            "status": r.status, "E0": r.E0,
                                            "d_sections": list(r.d_sec)[:nsec]}
        del prob
    return out


def batched_form(B, ai, reps):
    """64 independent design problems, scenario counts log-uniform in [50, 2000], solved
    as one batch (FP32 factors + FP64 refinement) against one-by-one solves."""
    P = ai.PARAMS
    sizes = ai.batched_sizes()
    feeds = ai.batched_feeds(sizes, seed=3)
    batch = B.Batch(P, feeds)
    o = B.default_options(precision=B.PREC_FP32, max_refine=8)
    batch.ipm_solve(o)
    sec, rs = timed(lambda: batch.ipm_solve(o), reps)
    res = rs[0]
    # every problem solved alone, one after the other (each after one untimed solve)
    probs = [B.Problem(P, F) for F in feeds]
    for p in probs:
        p.ipm_solve(o)
    sec1, rs1 = timed(lambda: [p.ipm_solve(o) for p in probs], 1)
    return {"problems": len(sizes), "scenarios": int(sizes.sum()), "solve_time_s": sec,
            "newton_steps_per_s": sum(r.iters for r in res) / sec,
            "status": sorted(set(r.status for r in res)), "iters_max": max(r.iters for r in res),
            "graph_replays": res[0].graph_replays,
            "one_by_one_s": sec1, "speedup_vs_one_by_one": sec1 / sec,
            "one_by_one_iters_equal": all(a.iters == b.iters for a, b in zip(res, rs1[0]))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="learned-fp32", choices=list(FORMS))
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the learned / batched form comparisons")
    ap.add_argument("--capture-iters", type=int, default=0,
                    help="profiling case: only N interior-point iterations of the workload from the inlet "
                         "start (no expected-value solve), then exit without a JSON line")
    ap.add_argument("--graphs", type=int, default=1,
                    help="1: each solve replays its captured CUDA graph; 0: eager launches (a profiler then sees "
                         "every kernel launch of the timed solves)")
    ap.add_argument("--factor-kernel", type=int, default=0,
                    help="FP32 factor kernel of the capture case: 0 Gauss-Jordan on the FP32 pipes, 1 tensor-core "
                         "panels")
    ap.add_argument("--factor-tile", type=int, default=0,
                    help="fixed FP32 factor launch shape (1/2/4/8 warps per block; 0: autotuned) -- for "
                         "profiling one shape")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    global FACTOR_TILE
    FACTOR_TILE = args.factor_tile

    import absorber_inputs as ai
    S_full = ai.WORKLOADS[args.workload]["S"]
    if args.impl == "reference":
        run_reference(args, S_full)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_15420_gb300 import binding as B

    P = ai.PARAMS
    # replicas: every rank solves its own instance of the workload (independent problems)
    F = ai.workload_feeds(args.workload)
    prob = B.Problem(P, F)
    st = torch.cuda.current_stream()
    prec, learned = FORMS[args.form]

    if args.capture_iters > 0:
        r = prob.ipm_solve(B.default_options(precision=prec, max_refine=(8 if prec == B.PREC_FP32 else 0),
                                             max_iter=args.capture_iters, init=1, factor_tile=FACTOR_TILE,
                                             factor_kernel=args.factor_kernel, graphs=0))
        torch.cuda.synchronize()
        print(f"capture case: {r.iters} iterations, status {B.STATUS.get(r.status)}", flush=True)
        return

    net, train_info = (None, None)
    if learned or not args.no_forms:
        net, train_info = train_network(B, ai)

    def step(profile=0, graphs=args.graphs, x_out=None):
        return solve_form(B, prob, net, args.form, profile, graphs, x_out)

    for _ in range(args.warmup):
        r = step()
        assert r.status == 0, f"warm-up solve failed: {B.STATUS.get(r.status)}"

    # ---- timed region: K full solves --------------------------------------------------
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")      # lets a profiler select the timed solves
    e0.record(st)
    results = [step() for _ in range(args.steps)]
    e1.record(st)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    for r in results:
        assert r.status == 0 and r.E0 <= 1e-8, (r.status, r.E0)
    iters = sum(r.iters for r in results)
    t_local = ms / 1e3
    t_job, it_job = job_totals(t_local, float(iters), world, "cuda")
    value = it_job / t_job

    # ---- per-kernel roofline: CUDA events around each hot launch in profiled solves of
    # the same form (profiling disables graph replay; these solves are not the timed ones)
    prof = [step(profile=1) for _ in range(2)]
    es = 4 if prec == B.PREC_FP32 else 8
    hbm, hbm_src = load_peaks()
    kms = [sum(r.kernel_ms[k] for r in prof) for k in range(5)]
    kn = [sum(r.kernel_launches[k] for r in prof) for k in range(5)]
    prof_ms = sum(r.solve_ms for r in prof)
    Sx = prob.S
    fma64 = B.measure_fma_peak(0)
    fma32 = B.measure_fma_peak(1)
    work = {  # (flops, bytes) per launch
        "eval": (EVAL_FP64_FLOPS_PER_SCEN * Sx, EVAL_BYTES_PER_SCEN * Sx),
        "eval_trial": (TRIAL_FP64_FLOPS_PER_SCEN * Sx, TRIAL_BYTES_PER_SCEN * Sx),
        "factor": (FACTOR_FLOPS_PER_SCEN[es] * Sx, factor_bytes(es) * Sx),
        "solve": (SOLVE_FLOPS_PER_SCEN_RHS * Sx * 1.5, solve_bytes(es, 1.5) * Sx),
        "solve_t": (SOLVE_T_FLOPS_PER_SCEN * Sx, solve_t_bytes(es) * Sx),
    }

    alu_peak = fma32 if es == 4 else fma64     # GFLOP/s: the measured FMA throughput of the dtype
    kern = {}
    for k, name in enumerate(B.KERNELS):
        if kn[k] == 0:
            continue
        avg_s = kms[k] / kn[k] / 1e3
        fl, by = work[name]
        kern[name] = {"launches": kn[k], "avg_us": 1e6 * avg_s, "share_of_solve": kms[k] / prof_ms,
                      "GB_s": by / avg_s / 1e9, "GFLOP_s": (fl / avg_s / 1e9) if fl else None}
        if name in ("eval", "eval_trial"):
            # FP64-bound: the achieved FP64 rate against the measured FP64 FMA throughput
            kern[name]["FP64_frac_of_measured"] = fl / avg_s / 1e9 / fma64
    dom = max(kern, key=lambda n: kms[B.KERNELS.index(n)])
    dk = kern[dom]
    fl, by = work[dom]
    intensity = (fl / by) if fl else 0.0
    balance = alu_peak / hbm
    if dom in ("eval", "eval_trial"):
        roof = {"bound": "alu", "achieved": dk["GFLOP_s"] / 1e3, "peak": fma64 / 1e3, "unit": "TFLOP/s",
                "frac": dk["GFLOP_s"] / fma64, "peak_source": "measured FP64 FMA throughput (abs_measure_fma_peak)"}
    elif fl and intensity > balance:
        roof = {"bound": "alu", "achieved": dk["GFLOP_s"] / 1e3, "peak": alu_peak / 1e3, "unit": "TFLOP/s",
                "frac": dk["GFLOP_s"] / alu_peak,
                "peak_source": ("measured FP32 FMA throughput" if es == 4 else
                                "measured FP64 FMA throughput") + " (abs_measure_fma_peak)"}
    else:
        roof = {"bound": "hbm", "achieved": dk["GB_s"], "peak": hbm, "unit": "GB/s", "frac": dk["GB_s"] / hbm,
                "peak_source": ("measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), of measured"
                                if hbm_src == "measured" else
                                "fallback copy bandwidth 6.8 TB/s (MEASURED_PEAKS.json absent), of fallback")}
    roof.update({"kernel": dom, "traffic": captured_traffic(dom, es, Sx), "algorithmic_bytes_per_launch": by,
                 "algorithmic_flops_per_launch": fl})
    # the whole solve: every kernel kind's launches (counted by the library in the profiled
    # solves, the same launch sequence as the timed ones) times its algorithmic bytes, over
    # the timed solve's device time
    kinds = {n: sum(r.kind_launches[k] for r in prof) / len(prof) for k, n in enumerate(B.KINDS)}
    kb = dict(KIND_BYTES)
    kb["eval"] = EVAL_BYTES_PER_SCEN
    kb["factor"] = factor_bytes(es)
    kb["solve"] = solve_bytes(es, 1.5)
    kb["solve_t"] = solve_t_bytes(es)
    solve_bytes_alg = sum(kinds[n] * kb[n] * Sx for n in kinds)
    whole = {"algorithmic_bytes_per_solve": solve_bytes_alg, "solve_time_s": ms / 1e3 / args.steps,
             "achieved_GB_s": solve_bytes_alg / (ms / 1e3 / args.steps) / 1e9,
             "peak": hbm, "frac": solve_bytes_alg / (ms / 1e3 / args.steps) / 1e9 / hbm,
             "launches_per_solve_by_kind": kinds}

    # ---- end to end through the C ABI: pinned host feeds in, solution out ------------
    e2e = None
    if not args.no_e2e:
        hf = torch.from_numpy(np.ascontiguousarray(F)).pin_memory()
        xo = torch.empty(prob.n_primal, dtype=torch.float64, device="cuda")
        xh = torch.empty(prob.n_primal, dtype=torch.float64).pin_memory()
        dfe = torch.empty(F.shape, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eit = 0
        for _ in range(args.steps):
            dfe.copy_(hf, non_blocking=True)          # H2D of the step's inputs
            prob.set_feeds(dfe)
            r = step(x_out=xo)
            xh.copy_(xo, non_blocking=True)           # D2H of the step's result
            torch.cuda.synchronize()
            assert r.status == 0
            eit += r.iters
        te = time.perf_counter() - t0
        e2e = {"value": eit / te, "unit": UNIT, "h2d_bytes_per_step": int(F.nbytes),
               "d2h_bytes_per_step": int(prob.n_primal * 8), "solve_time_s": te / args.steps}

    forms = None
    if rank == 0 and not args.no_forms:
        forms = {"training": train_info, "headline_workload": compare_forms(B, prob, net, reps=3)}
        # graph replay on / off for the timed form
        sec_off, _ = timed(lambda: step(graphs=0), 3)
        forms["graphs"] = {"form": args.form, "solve_time_s_graphs_on": t_job / args.steps,
                           "solve_time_s_graphs_off": sec_off}
        p20 = B.Problem(P, ai.workload_feeds("absorber-S20000-u10-seed4"))
        forms["absorber-S20000-u10-seed4"] = compare_forms(B, p20, net, reps=2)
        del p20
        forms["batched"] = batched_form(B, ai, reps=2)
        forms["two-section"] = two_section_form(B, ai, P, reps=2)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample, its = 50, 6
        nproc, naff = visible_cores()
        rb = cpu_baseline(args.workload, sample, its)
        cpu = {"value": rb["iters"] / rb["seconds"] * (sample / Sx), "unit": UNIT, "cores": 1, "kind": "oracle",
               "visible_cores": {"nproc": nproc, "affinity": naff},
               "sample": f"{rb['iters']} IPM iterations of the oracle on the first {sample} of the {Sx} "
                         f"scenarios ({rb['seconds']:.1f} s), one thread, per-iteration cost scaled linearly "
                         f"to {Sx} (extrapolated)"}
        per = 25
        ra = cpu_baseline_all_cores(args.workload, per, its, naff)
        cpu["all_cores"] = {
            "value": ra["iters"] / ra["wall_s"] * (naff * per / Sx), "unit": UNIT, "cores": naff, "kind": "oracle",
            "sample": f"{naff} single-threaded oracle processes at once, each {ra['iters']} IPM iterations on its "
                      f"own block of {per} scenarios ({ra['wall_s']:.1f} s wall for {naff * per} scenarios), "
                      f"per-iteration cost scaled linearly to {Sx} (extrapolated; the blocks' scalar "
                      f"reductions are not timed)"}

    if rank == 0:
        r0 = results[0]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == B.PREC_FP32 else "f64",
            "data": "synthetic (seeded feeds; the paper's measured cases are not published)",
            "config": {"workload": args.workload, "scenarios": Sx, "variables": int(prob.sizes.n_var_paper),
                       "tol": 1e-8, "form": args.form,
                       "step": ("one full interior-point solve to E_0 <= 1e-8 from the "
                                + ("learned warm start (network trained in the run, untimed)" if learned
                                   else "default start")),
                       "parallelism": f"replicas x{world}",
                       "l2": "working set > L2 (factors + Jacobian values ~ 0.3-0.6 GB per iteration)"},
            "solve_time_s": ms / 1e3 / args.steps,
            "iters_per_solve": [r.iters for r in results],
            "learned_start_used": [bool(r.warm_status) for r in results] if learned else None,
            "d_opt": r0.d, "E0": max(r.E0 for r in results),
            "tiles": list(r0.tiles), "graph_replays_per_solve": r0.graph_replays,
            "phase_ms_per_solve": {n: sum(r.phase_ms[i] for r in prof) / len(prof)
                                   for i, n in enumerate(B.PHASES)},
            "kernels": kern, "roofline": roof, "whole_solve_roofline": whole,
            "fma_peaks_gflops": {"fp64": fma64, "fp32": fma32},
            "forms": forms,
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": int(sum(r.launches for r in results)),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
