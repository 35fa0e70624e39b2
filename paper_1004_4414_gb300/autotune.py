"""Autotuner of the fused step kernel's block shape.

Candidates are (ty, cz, split): split 0 runs one thread per node with ty
rows of 32 nodes per CTA (4, 8 or 16); split 1 runs one thread per node and
component with ty rows of 16 nodes (8 or 16); cz z-planes are marched per
CTA.  Each candidate is timed with CUDA events around
the fused kernel over a few steps of the real boxes (the simulation
advances while tuning, so run it as part of the warm-up), and the fastest
is kept.  Results are cached per (box sizes, precision, tau) in memory.
"""
_CACHE = {}

DEFAULT_CANDIDATES = ((4, 16, 0), (4, 32, 0), (4, 64, 0), (8, 16, 0), (8, 32, 0), (8, 64, 0), (16, 16, 0), (16, 32, 0),
                      (8, 16, 1), (8, 32, 1), (16, 16, 1), (16, 32, 1))


def _key(sim):
    # box sizes, storage and relaxation times (tau = 1 selects a specialised kernel)
    return (tuple(sim.dims), tuple(p.precision for p in sim._params),
            tuple((p.tau[0], p.tau[1]) for p in sim._params))


def autotune(sim, candidates=DEFAULT_CANDIDATES, steps=4, use_cache=True):
    """Pick the fastest (ty, cz, split) for this simulation's boxes; returns
    (best, {candidate: ms per fused launch})."""
    key = _key(sim)
    if use_cache and key in _CACHE:
        best, table = _CACHE[key]
        sim.set_tiling(*best)
        return best, table
    maxnz = max(d[2] for d in sim.dims)
    table = {}
    for cand in candidates:
        ty, cz, split = tuple(cand) + (0,) * (3 - len(cand))
        if cz > maxnz and cz != candidates[0][1]:
            continue
        sim.set_tiling(ty, cz, split)
        sim.step(2)  # settle
        sim.sync()
        sim.set_profiling(True)
        sim.step(steps)
        ms, n, _ = sim.kernel_time()
        sim.set_profiling(False)
        table[(ty, cz, split)] = ms / max(n, 1)
    best = min(table, key=table.get)
    sim.set_tiling(*best)
    _CACHE[key] = (best, table)
    return best, table
