"""Autotuner of the fused step kernel's block shape.

Candidates are (ty, cz): ty rows of 32 nodes per CTA (4, 8 or 16) and cz
z-planes marched per CTA.  Each candidate is timed with CUDA events around
the fused kernel over a few steps of the real boxes (the simulation
advances while tuning, so run it as part of the warm-up), and the fastest
is kept.  Results are cached per (box sizes, precision) in memory.
"""
_CACHE = {}

DEFAULT_CANDIDATES = ((4, 16), (4, 32), (4, 64), (8, 16), (8, 32), (8, 64), (16, 16), (16, 32))


def _key(sim):
    return (tuple(sim.dims), tuple(p.precision for p in sim._params))


def autotune(sim, candidates=DEFAULT_CANDIDATES, steps=4, use_cache=True):
    """Pick the fastest (ty, cz) for this simulation's boxes; returns
    (best, {candidate: ms per fused launch})."""
    key = _key(sim)
    if use_cache and key in _CACHE:
        best, table = _CACHE[key]
        sim.set_tiling(*best)
        return best, table
    maxnz = max(d[2] for d in sim.dims)
    table = {}
    for ty, cz in candidates:
        if cz > maxnz and cz != candidates[0][1]:
            continue
        sim.set_tiling(ty, cz)
        sim.step(2)  # settle
        sim.sync()
        sim.set_profiling(True)
        sim.step(steps)
        ms, n, _ = sim.kernel_time()
        sim.set_profiling(False)
        table[(ty, cz)] = ms / max(n, 1)
    best = min(table, key=table.get)
    sim.set_tiling(*best)
    _CACHE[key] = (best, table)
    return best, table
