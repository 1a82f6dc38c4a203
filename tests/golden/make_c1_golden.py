"""Write the stored expected values of the 500-scenario workload (uniform +-10 % feeds,
seed 1) from the CPU oracle alone: the plain FP64 interior-point solve of problem (10)
(oracle/ipm.py, expected-value start), its optimal diameter, iteration counts, E_0
recomputed from the definitions (oracle/checks.kkt_error), and the stage states of a
few scenarios, among them the one whose hydraulic row sets d*.

    python tests/golden/make_c1_golden.py      (about 20 minutes on one core)

Nothing here calls the CUDA library.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import absorber_inputs as ai  # noqa: E402
from oracle import checks, ipm, model  # noqa: E402

OUT = os.path.join(HERE, "c1_s500_seed1.json")


def main():
    P = ai.PARAMS
    S, seed = 500, 1
    F = ai.make_feeds(S, seed)
    t0 = time.perf_counter()
    r = ipm.solve(P, F)
    el = time.perf_counter() - t0
    assert r.status == "ok", r.status
    E0 = checks.kkt_error(P, F, r.d, r.Z, r.lam, r.zL, r.zU, r.zLd, r.zUd, chunk=100)
    dmin, vol = checks.minimum_diameter(P, F, r.Z)
    arg = int(np.unravel_index(np.argmax(vol), vol.shape)[0])
    sample = sorted({0, 1, 250, S - 1, arg})
    out = {
        "what": "CPU oracle solve of problem (10), 500 scenarios, uniform +-10 % feeds from seed 1, "
                "expected-value start, objective scaled by S, E_0 <= 1e-8 (oracle/ipm.py)",
        "script": "tests/golden/make_c1_golden.py",
        "S": S, "seed": seed, "dist": "uniform",
        "status": r.status, "iters": int(r.iters), "base_iters": int(r.base_iters),
        "d": float(r.d), "E0_solver": float(r.E0), "E0_recomputed": float(E0),
        "d_from_states": float(dmin), "binding_scenario": arg,
        "sample": sample,
        "Z": {str(s): [float(v) for v in r.Z[s]] for s in sample},
        "lam_hydraulic_sum": float(r.lam.reshape(S, model.N, model.NV)[:, :, model.NV - 1].sum()),
        "oracle_seconds": el,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(f"wrote {OUT}: d* = {r.d:.12f}, {r.iters} iterations (+{r.base_iters} base), E0 {E0:.2e}, {el:.0f} s")


if __name__ == "__main__":
    main()
