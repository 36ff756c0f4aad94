"""Parameter autotuner for a resident chain (or batch of chains).

The threshold schedules have knobs the paper leaves open: the multiplier and
the exponent r of theta_t(r) (Sec. 6), and here also the fraction of the
edges at which a move pulls over the in-links instead of pushing over the
out-links, and, for a batch of chains solved in one persistent launch, the
threads per block of that launch (block size). Which setting reaches a tolerance first depends on the chain
(degree spread, mixing) and on the device. The tuner runs the same solve
(step 0, then the schedule to the tolerance) once per candidate on the
chain itself, measures its wall time around the library call (which
synchronises), keeps the fastest setting that converged, and leaves it set
on the chain. Every candidate restarts from step 0, so the chain's state
after tuning is that of the winning solve.
"""
from __future__ import annotations

import itertools
import time
from typing import Dict, Iterable, List, Optional

DEFAULT_GRID = {
    "theta_scale": (0.25, 0.5, 1.0, 2.0),
    "r": (1, 2),
    "pull_crossover": (0.1, 0.25, 0.5),
}

# A batch adds the block size of its persistent launch.
DEFAULT_BATCH_GRID = dict(DEFAULT_GRID, batch_block=(128, 256, 512))


def default_grid(chain) -> Dict[str, Iterable]:
    """The default search grid for `chain`: with the block size for a batch
    of several chains."""
    return DEFAULT_BATCH_GRID if getattr(chain, "nchains", 1) > 1 else DEFAULT_GRID


def candidates(grid: Optional[Dict[str, Iterable]] = None) -> List[dict]:
    """The cartesian product of the grid's values, as parameter dicts."""
    grid = DEFAULT_GRID if grid is None else grid
    keys = sorted(grid)
    return [dict(zip(keys, vals)) for vals in itertools.product(*(tuple(grid[k]) for k in keys))]


def autotune(chain, schedule: str = "link_threshold", tol: float = 1e-6,
             grid: Optional[Dict[str, Iterable]] = None, m0=None, max_steps: int = 100000,
             repeats: int = 1, clock=time.perf_counter) -> dict:
    """Tries every candidate of `grid` on `chain` (a rlgl.Chain) and sets the
    fastest one that reached `tol`. Returns {"best": params, "seconds": s,
    "moves": m, "trials": [(params, seconds or None, moves, status)]}.
    Raises RuntimeError when no candidate converged."""
    trials = []
    best = None
    if grid is None:
        grid = default_grid(chain)
    for cand in candidates(grid):
        chain.set_params(**cand)
        secs = []
        info = None
        for _ in range(max(1, repeats)):
            chain.reset(m0)
            t0 = clock()
            info = chain.solve(schedule, tol=tol, max_steps=max_steps, raise_on_noconv=False)
            secs.append(clock() - t0)
        ok = info["status"] == "RLGL_OK"
        s = min(secs) if ok else None
        trials.append((cand, s, info["moves"], info["status"]))
        if ok and (best is None or s < best[1]):
            best = (cand, s, info["moves"])
    if best is None:
        raise RuntimeError(f"no candidate reached tol {tol} within {max_steps} moves")
    chain.set_params(**best[0])
    chain.reset(m0)
    chain.solve(schedule, tol=tol, max_steps=max_steps, raise_on_noconv=False)
    return {"best": best[0], "seconds": best[1], "moves": best[2], "trials": trials}
