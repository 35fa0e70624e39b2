"""Write tests/golden/lt_c128_long.json: domain size L(t) (Eq. eq:domsize) and
interface coverage of the FP64 oracle on the 128^3 configuration of
lt_c128.json (50:50 of total density 0.7, alpha = 0.15, R = 5, contact
angle 90 deg, g = 0.08, particle density 3, seed 2), every 500 steps up to
STEPS, for the late-time comparison (coarsening, coverage below 1).

Only oracle/ is used.  Run from the repository root:
    python tests/golden/make_lt_long_golden.py [threads] [steps]
(about 25 minutes per 1000 steps with 8 threads).  The file is rewritten
after every checkpoint, so an interrupted run leaves the checkpoints it
reached."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from oracle import ref  # noqa: E402
from make_lt_golden import PARAMS, SEED, observe  # noqa: E402

EVERY = 500


def main():
    ref.set_threads(int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count() or 1)
    steps = int(sys.argv[2]) if len(sys.argv) > 2 else 6000
    o = ref.Oracle(**PARAMS)
    o.init_from_seed(SEED)
    out = {"params": {k: list(v) if isinstance(v, tuple) else v for k, v in PARAMS.items()}, "seed": SEED,
           "steps": [], "L": [], "coverage": [], "n_particles": o.np,
           "source": "oracle/ (FP64), tests/golden/make_lt_long_golden.py"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lt_c128_long.json")
    t0 = time.time()
    for k in range(steps // EVERY):
        o.step(EVERY)
        L, cov = observe(o)
        out["steps"].append((k + 1) * EVERY)
        out["L"].append(L)
        out["coverage"].append(cov)
        with open(path + ".tmp", "w") as fh:
            json.dump(out, fh, indent=1)
        os.replace(path + ".tmp", path)
        print((k + 1) * EVERY, L, cov, "%.0f s" % (time.time() - t0), flush=True)


if __name__ == "__main__":
    main()
