"""Run monitor: step a context in chunks and append one JSON line per chunk
with the FP64 totals, the per-star totals of a batch and the library's
counters (a time series of conserved quantities, yield and damage counts,
neighbour numbers and centre of mass for a run).

Every number comes from the library's own reductions (sph_totals,
sph_totals_per_star, sph_stats); this module only schedules the calls and
writes the lines.
"""
from __future__ import annotations

import json
import time

from . import sph

TOTAL_NAMES = ("mass", "px", "py", "pz", "kinetic", "internal", "energy", "Lx", "Ly", "Lz",
               "yielded", "broken", "mean_neighbours", "cx", "cy", "cz")


def totals_record(tot) -> dict:
    """The 16 totals of sph_totals (or one row of sph_totals_per_star) by name."""
    return {k: float(v) for k, v in zip(TOTAL_NAMES, tot)}


def run_logged(ctx, dt: float, nsteps: int, every: int, path: str, nstars: int = 1,
               t0: float = 0.0) -> int:
    """Advance `nsteps` steps of size dt in chunks of `every` steps; after the
    initial state and after each chunk append a line to the JSONL file `path`:
    step, time, wall seconds since the call, the totals, the per-star totals
    (when nstars > 1), candidate-list builds and pairs of the last
    right-hand side.  Returns the number of lines written."""
    if every < 1 or nsteps < 0:
        raise ValueError("every must be >= 1 and nsteps >= 0")
    start = time.perf_counter()
    lines = 0
    with open(path, "a") as f:
        done = 0
        while True:
            sph.sph_sync(ctx)
            stats = sph.sph_stats(ctx)
            rec = {"step": int(stats[9]), "t": t0 + done * dt,
                   "wall_s": time.perf_counter() - start,
                   "totals": totals_record(sph.sph_totals(ctx)),
                   "pairs_last_rhs": int(stats[0]), "candidate_builds": int(stats[18])}
            if nstars > 1:
                rec["stars"] = [totals_record(r) for r in sph.sph_totals_per_star(ctx, nstars)]
            f.write(json.dumps(rec) + "\n")
            lines += 1
            if done >= nsteps:
                break
            k = min(every, nsteps - done)
            sph.sph_step(ctx, dt, k)
            done += k
    return lines
