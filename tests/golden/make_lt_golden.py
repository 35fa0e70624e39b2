"""Write tests/golden/lt_c128.json: domain size L(t) (Eq. eq:domsize) and
interface coverage of the FP64 oracle on the 128^3 configuration (50:50 of
total density 0.7, alpha = 0.15, R = 5, contact angle 90 deg, g = 0.08,
particle density 3, seed 2), every 100 steps up to 1000.

Only oracle/ is used.  Run from the repository root:
    python tests/golden/make_lt_golden.py [threads]
(about 25 minutes with 8 threads)."""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import analysis, ref  # noqa: E402

PARAMS = dict(nx=128, ny=128, nz=128, n_particles=-1, tau=(1.0, 1.0), g_br=0.08, rho0=1.0, sc_weight=(2.0, 1.0),
              rho_init=(0.35, 0.35), noise_amp=0.01, volume_fraction=0.15, radius=5.0, particle_density=3.0,
              color=0.0, k_hertz=100.0)
SEED = 2
EVERY, STEPS = 100, 1000


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
    o.init_from_seed(SEED)
    out = {"params": {k: list(v) if isinstance(v, tuple) else v for k, v in PARAMS.items()}, "seed": SEED,
           "steps": [], "L": [], "coverage": [], "n_particles": o.np,
           "source": "oracle/ (FP64), tests/golden/make_lt_golden.py"}
    t0 = time.time()
    for k in range(STEPS // EVERY):
        o.step(EVERY)
        L, cov = observe(o)
        out["steps"].append((k + 1) * EVERY)
        out["L"].append(L)
        out["coverage"].append(cov)
        print((k + 1) * EVERY, L, cov, "%.0f s" % (time.time() - t0), flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "lt_c128.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
