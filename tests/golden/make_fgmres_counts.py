"""Write fgmres_counts.json: the FP64 oracle's FGMRES iteration counts on the
full-size workloads, for the GPU test that compares the library's counts with
them (within one iteration).

Each case: the oracle's own set-up of the workload, its low-rank term built
by its Arnoldi process (Algorithm 1, steps 6-8; SplitMix64 start vector, seed
0), and right-preconditioned FGMRES(restart) from x0 = 0 to a relative
residual of 1e-8 on b = A x*, x* ~ U[-1, 1] (seed 0), stopped after maxit
iterations (the Section 4 stopping rule).  A second run on b perturbed by
1e-15 relative (seeded) records how far the count itself moves under
rounding-level changes of the input.

Only oracle/ and pslr_inputs/ are used.  Run from the repository root:

    python tests/golden/make_fgmres_counts.py [workload ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from pslr_inputs import configs as C  # noqa: E402
from pslr_inputs import generators as G  # noqa: E402

CASES = [
    ("lap3d_64_4x4x2_ilu0", 120, 1500),
    ("lap3d_64_4x4x2_ilu0", 40, 500),
    ("kappa3d_48_3x3x3", 40, 500),
    ("kappa3d_48_3x3x3", 120, 1500),
    ("cd3d_128_8x8x4_ilu0", 40, 500),
    ("cd3d_128_8x8x4_ilu0_noshift", 40, 500),
]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fgmres_counts.json")


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name, restart, maxit in CASES:
        if names and name not in names:
            continue
        t0 = time.time()
        w = C.WORKLOADS[name]()
        orc = O.from_workload(w)
        rank, _ = orc.build_lowrank(w["m"], w["rank"], seed=0)
        b, _ = G.uniform_rhs(w["A"], 0)
        _, its, rel, st = orc.fgmres(b, rtol=1e-8, restart=restart, maxit=maxit)
        bp = b * (1.0 + 1e-15 * np.random.default_rng(9).uniform(-1, 1, b.size))
        _, its_p, rel_p, _ = orc.fgmres(bp, rtol=1e-8, restart=restart, maxit=maxit)
        data[f"{name}/restart{restart}"] = {
            "workload": name, "restart": restart, "maxit": maxit, "rtol": 1e-8, "m": w["m"], "rank": rank,
            "sigma": w["sigma"], "iters": int(its), "relres": float(rel), "converged": int(st) == 0,
            "iters_b_perturbed_1e-15": int(its_p), "relres_b_perturbed_1e-15": float(rel_p),
            "oracle_seconds": round(time.time() - t0, 1)}
        print(name, restart, data[f"{name}/restart{restart}"], flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
