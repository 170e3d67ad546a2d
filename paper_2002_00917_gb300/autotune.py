"""Autotuner of the batch's launch shape (pslr_batch_opts).

The batched kernel sweeps a group of subdomains of one system in lockstep
(their levels merged), and how many to group trades steps per CTA against
shared memory (vectors of every grouped subdomain and right-hand side) and
ring depth.  ``tune_group`` builds the batch for each candidate group size,
times the batched apply with CUDA events (L2 flushed between launches, as the
bench does) and returns the fastest.  ``tune_batch`` searches every knob of
pslr_batch_opts: group size and ring depth per precision, the FP64 thread
mapping of the right-hand sides ((row, rhs) pairs or rows), and the chunk
length of the batched Krylov kernels (timed on a batched FGMRES solve).
Every candidate computes the same result; only the speed differs.  The
number of consumer warps per CTA is not a knob: the level-sweep barriers,
the ring protocol and the shared-memory layout are built for eight.
"""
from __future__ import annotations

import torch

from . import pslr


def _time_apply(bt, prec, steps, warmup, flush):
    dtype = torch.float64 if prec == pslr.PSLR_FP64 else torch.float32
    b = torch.rand(bt.info["n_total"], dtype=dtype, device="cuda")
    z = torch.empty_like(b)
    for _ in range(warmup):
        bt.apply(b, z)
    bt.sync()
    st = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        bt.apply(b, z)
        e1.record(st)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    bt.sync()
    ms.sort()
    return ms[len(ms) // 2]


def tune_group(systems, nrhs, prec=pslr.PSLR_FP32, candidates=(1, 2, 4, 6, 8), steps=5, warmup=2,
               flush_bytes=512 << 20):
    """Time the batched apply of ``systems`` (set-up :class:`pslr.Pslr`
    contexts with their low-rank terms) for each requested group size and
    return ``(best_group, table)``; ``table`` maps each request to
    ``(effective group, ms per apply)`` (a request larger than shared memory
    allows is reduced by the library)."""
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device="cuda")
    k = 0 if prec == pslr.PSLR_FP64 else 1
    table = {}
    for g in candidates:
        bt = pslr.Batch(systems, nrhs, group=g)
        try:
            table[g] = (bt.info["group"][k], _time_apply(bt, prec, steps, warmup, flush))
        finally:
            bt.close()
    best = min(table, key=lambda g: table[g][1])
    return best, table


def _time_solve(bt, b, restart, prec, rtol, maxit):
    x = torch.zeros_like(b)
    bt.solve(b, x, rtol=rtol, restart=restart, maxit=1, prec=prec, check=False)  # workspace, cycle graph
    torch.cuda.synchronize()
    x.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    bt.solve(b, x, rtol=rtol, restart=restart, maxit=maxit, prec=prec, check=False)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def tune_batch(systems, nrhs, groups=((0, 2, 3), (0, 2, 4, 6)), rings=(0, 3), pairs=(1, 0),
               chunks=(512, 1024, 2048), restart=127, rtol=1e-8, maxit=2000, steps=3, warmup=2,
               flush_bytes=512 << 20):
    """Search the launch-shape knobs of a batch over ``systems`` (set-up
    :class:`pslr.Pslr` contexts with their low-rank terms), ``nrhs``
    right-hand sides each.  The applies are timed per precision over
    ``groups[prec]`` x ``rings`` (x ``pairs`` in FP64, where it applies);
    then, with the best FP32 apply, a batched FGMRES(``restart``) solve of
    the FP32 form to ``rtol`` (a seeded random right-hand side; the late
    cycles, with few problems left, favour other chunk lengths than the
    first) per Krylov chunk length.  Returns ``(best, table)``: ``best``
    holds the keyword arguments of :class:`pslr.Batch` (group and ring_max
    per precision, pair_rhs, krylov_chunk); ``table`` is one dict per timed
    candidate: the request, what the library made of it (effective group,
    ring slots) and the milliseconds."""
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device="cuda")
    table = []
    best_apply = {}
    for k, prec in ((0, pslr.PSLR_FP64), (1, pslr.PSLR_FP32)):
        tag = "fp64" if k == 0 else "fp32"
        for g in groups[k]:
            for ring in rings:
                for pair in (pairs if k == 0 and nrhs > 1 else (1,)):
                    rm = [0, 0]
                    rm[k] = ring
                    gg = [0, 0]
                    gg[k] = g
                    bt = pslr.Batch(systems, nrhs, group=tuple(gg), ring_max=tuple(rm), pair_rhs=pair)
                    try:
                        ms = _time_apply(bt, prec, steps, warmup, flush)
                        row = {"what": "apply_" + tag, "group": g, "ring_max": ring, "pair_rhs": pair,
                               "effective_group": bt.info["group"][k], "ring": bt.info["ring"][k], "ms": ms}
                    finally:
                        bt.close()
                    table.append(row)
                    if tag not in best_apply or ms < best_apply[tag]["ms"]:
                        best_apply[tag] = row
    b64, b32 = best_apply["fp64"], best_apply["fp32"]
    best = {"group": (b64["group"], b32["group"]), "ring_max": (b64["ring_max"], b32["ring_max"]),
            "pair_rhs": b64["pair_rhs"], "krylov_chunk": 0}
    best_ms = None
    for ch in chunks:
        bt = pslr.Batch(systems, nrhs, group=best["group"], ring_max=best["ring_max"], pair_rhs=best["pair_rhs"],
                        krylov_chunk=ch)
        try:
            gen = torch.Generator(device="cuda")
            gen.manual_seed(7)
            b = torch.rand(bt.info["n_total"], dtype=torch.float64, device="cuda", generator=gen)
            ms = _time_solve(bt, b, restart, pslr.PSLR_FP32, rtol, maxit)
        finally:
            bt.close()
        table.append({"what": f"fgmres{restart}_solve_fp32", "krylov_chunk": ch, "ms": ms})
        if best_ms is None or ms < best_ms:
            best_ms, best["krylov_chunk"] = ms, ch
    return best, table
