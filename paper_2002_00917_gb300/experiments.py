"""The studies of Section 4.1 (the 50^3 shifted Laplacian and the meshes of
Table 6), ILUT(1e-2) local factors, m = 3, through the library:

* ``s``    - the number of subdomains (Table 1; r = 15, shift .05).  The
  geometric split stands in for METIS: 2x2x2, 4x2x2, 3x3x3, 3x3x4, 3x3x5 and
  3x3x6 for the paper's s = 5, 15, 25, 35, 45, 55 (five parts of a 50^3 cube
  do not fit one CTA each).
* ``m``    - the series order 0..5 (Table 2; 3x3x4, r = 15, shift .05).
* ``rank`` - the rank 0, 15, ..., 75 (Tables 3 and 4; 3x3x4; shift .05 and
  .14 with ``--shift``).
* ``lap``  - the meshes of Table 6 (32^3, 64^3, 128^3 at shifts .16, .08,
  .03; m = 3, r = 15): 3x3x4 for the paper's s = 35 on the two smaller
  meshes, 8x8x4 on 128^3 (35 parts of 128^3 do not fit one CTA each).
* ``neumann`` - the classical Neumann polynomial of Section 1 (the foil the
  paper contrasts PSLR with; pslr_set_neumann) for omega = 0.5 .. 1.5 at
  m = 3, next to PSLR with r = 0, 15 and 45 (3x3x4, shift .05 and .14).

Each run prints one JSON line: partition size, fill factors (Section 4's
definitions), levels per sweep, and, unless ``--dry-run``, the FGMRES(127)
iterations to 1e-8 with the FP64 preconditioner, the set-up, low-rank and
solve times on the current GPU.  ``--dry-run`` needs no GPU: it runs the
host set-up only (``pslr.plan``) and reports the partition, fills and levels.

    python -m paper_2002_00917_gb300.experiments rank --shift 0.14
    python -m paper_2002_00917_gb300.experiments lap --dry-run
"""
from __future__ import annotations

import argparse
import json
import time

from . import pslr

DIMS = (50, 50, 50)
LAP_MESHES = [(32, 0.16, (3, 3, 4)), (64, 0.08, (3, 3, 4)), (128, 0.03, (8, 8, 4))]
S_SPLITS = [(2, 2, 2), (4, 2, 2), (3, 3, 3), (3, 3, 4), (3, 3, 5), (3, 3, 6)]
PAPER_S = [5, 15, 25, 35, 45, 55]
OMEGAS = [0.5, 0.75, 1.0, 1.25, 1.5]


def runs(sweep, shift=None):
    """(shift, splits, m, r) of every run of a sweep, in order; the ``lap``
    runs add their mesh dimensions (the others use the 50^3 mesh)."""
    if sweep == "s":
        return [(0.05 if shift is None else shift, sp, 3, 15) for sp in S_SPLITS]
    if sweep == "m":
        return [(0.05 if shift is None else shift, (3, 3, 4), m, 15) for m in range(6)]
    if sweep == "rank":
        return [(0.05 if shift is None else shift, (3, 3, 4), 3, r) for r in range(0, 76, 15)]
    if sweep == "lap":
        return [(sh, sp, 3, 15, (N, N, N)) for N, sh, sp in LAP_MESHES]
    if sweep == "neumann":
        out = []
        for sh in ((0.05, 0.14) if shift is None else (shift,)):
            out += [(sh, (3, 3, 4), 3, 0, DIMS, om) for om in OMEGAS]
            out += [(sh, (3, 3, 4), 3, r) for r in (0, 15, 45)]
        return out
    raise ValueError(f"unknown sweep {sweep!r}")


def one(A, shift, splits, m, r, drop_tol=1e-2, restart=127, maxit=1500, dry_run=False, rhs_seed=0, dims=DIMS,
        omega=None):
    """One run; returns its JSON record.  omega: the Section 1 Neumann
    polynomial with that scaling instead of PSLR (r is then 0)."""
    rec = {"shift": shift, "dims": list(dims), "splits": list(splits), "s": splits[0] * splits[1] * splits[2],
           "m": m, "r": r}
    if omega is not None:
        rec["preconditioner"] = f"neumann(omega={omega})"
    if dry_run:
        info = pslr.plan(A, dims, splits, factor=2, m=m, rank=r, drop_tol=drop_tol)[0]
        rec.update(q=info["q"], fill_ilu=round(info["fill_ilu"], 4), fill_lr=round(info["fill_lr"], 4),
                   fill_total=round(info["fill_total"], 4), levels_B=info["levels_B"], levels_C0=info["levels_C0"])
        return rec
    import torch

    from pslr_inputs import generators as G

    b, _ = G.uniform_rhs(A, rhs_seed)
    bd = torch.tensor(b, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = pslr.Pslr(A, dims=dims, splits=splits, factor=2, drop_tol=drop_tol)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    try:
        t0 = time.perf_counter()
        if omega is not None:
            ctx.set_neumann(m, omega)
        elif r:
            ctx.build_lowrank(m, r)
        else:
            ctx.set_lowrank(m)
        torch.cuda.synchronize()
        t_lr = time.perf_counter() - t0
        x = torch.empty_like(bd)
        ctx.solve(bd, x, rtol=1e-8, restart=restart, maxit=restart, check=False)  # captures the cycle
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, rel, st = ctx.solve(bd, x, rtol=1e-8, restart=restart, maxit=maxit, check=False)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        info = ctx.info
        full = ctx.get_info()
        rec.update(q=info["q"], fill_ilu=round(info["fill_ilu"], 4), fill_lr=round(full["fill_lr"], 4),
                   fill_total=round(full["fill_total"], 4), levels_B=info["levels_B"], levels_C0=info["levels_C0"],
                   its=its, relres=rel,
                   converged=st == pslr.PSLR_OK, setup_s=round(t_setup, 4), lowrank_s=round(t_lr, 4),
                   solve_ms=round(1e3 * t_solve, 2))
    finally:
        ctx.close()
    return rec


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("sweep", choices=["s", "m", "rank", "lap", "neumann"])
    ap.add_argument("--shift", type=float, default=None, help="shift of the Laplacian (default .05)")
    ap.add_argument("--drop-tol", type=float, default=1e-2)
    ap.add_argument("--restart", type=int, default=127)
    ap.add_argument("--dry-run", action="store_true", help="host set-up only: partition, fills, levels")
    a = ap.parse_args(argv)
    from pslr_inputs import generators as G

    out = []
    A, key = None, None
    for run in runs(a.sweep, a.shift):
        shift, splits, m, r = run[:4]
        dims = run[4] if len(run) > 4 else DIMS
        omega = run[5] if len(run) > 5 else None
        if key != (dims, shift):
            A, key = G.shifted_laplacian(dims, shift), (dims, shift)
        rec = one(A, shift, splits, m, r, drop_tol=a.drop_tol, restart=a.restart, dry_run=a.dry_run, dims=dims,
                  omega=omega)
        print(json.dumps(rec), flush=True)
        out.append(rec)
    return out


if __name__ == "__main__":
    main()
