"""Write tests/golden/lt_layers112.json: domain size (Eq. eq:domsize) and
interface coverage of the FP64 oracle on a 112^3 box of alternating red
and blue layers (period 56 along z, densities 0.6 / 0.1 with node noise
0.01, seed 7) holding 402 spheres (R = 5, about 15 % of the volume, placed
at random by lbinputs.spheres with seed 8, at rest), g = 0.08, neutral
wetting, particle density 3, every 250 steps up to 2500.  Spheres inside a
layer see one phase, spheres on an interface both, so the coverage lies
well below 1 and changes as particles reach the interfaces.

Only oracle/ and lbinputs are used.  Run from the repository root:
    python tests/golden/make_lt_layers_golden.py [threads]
(about 40 minutes with 8 threads)."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import lbinputs  # noqa: E402
from oracle import analysis, ref  # noqa: E402

SHAPE = (112, 112, 112)
PARAMS = dict(nx=112, ny=112, nz=112, n_particles=402, tau=(1.0, 1.0), g_br=0.08, rho0=1.0, sc_weight=(2.0, 1.0),
              rho_init=(0.35, 0.35), noise_amp=0.0, radius=5.0, particle_density=3.0, color=0.0, k_hertz=100.0)
LAYERS = dict(period=56, rho_major=0.6, rho_minor=0.1, amp=0.01, seed=7)
SPHERES = dict(radius=5.0, n=402, seed=8, min_gap=0.5)
EVERY, STEPS = 250, 2500


def inputs():
    rho = lbinputs.layers(SHAPE, **LAYERS)
    parts = lbinputs.spheres(SHAPE, **SPHERES)
    return rho, parts


def observe(o):
    st = o.get_state()
    rho = o.rho()
    shape = (PARAMS["nz"], PARAMS["ny"], PARAMS["nx"])
    phi = (rho[0] - rho[1]).reshape(shape)  # 0 on solid nodes
    L = analysis.domain_size(phi)
    cov = analysis.coverage(phi, st["owner"].reshape(shape), o.np)
    return [float(v) for v in L], float(cov)


def main():
    ref.set_threads(int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count() or 1)
    o = ref.Oracle(**PARAMS)
    rho, parts = inputs()
    o.init_fields(rho, particles=parts)
    out = {"params": {k: list(v) if isinstance(v, tuple) else v for k, v in PARAMS.items()},
           "layers": LAYERS, "spheres": SPHERES, "steps": [], "L": [], "coverage": [],
           "source": "oracle/ (FP64), tests/golden/make_lt_layers_golden.py"}
    L, cov = observe(o)
    out["steps"].append(0)
    out["L"].append(L)
    out["coverage"].append(cov)
    t0 = time.time()
    for k in range(STEPS // EVERY):
        o.step(EVERY)
        L, cov = observe(o)
        out["steps"].append((k + 1) * EVERY)
        out["L"].append(L)
        out["coverage"].append(cov)
        print((k + 1) * EVERY, L, cov, "%.0f s" % (time.time() - t0), flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "lt_layers112.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
