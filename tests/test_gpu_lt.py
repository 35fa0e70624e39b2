"""Long-run statistics where trajectories diverge: domain size L(t)
(Eq. eq:domsize) and interface coverage of the CUDA path against the FP64
oracle on the 128^3 configuration (50:50 of total density 0.7,
alpha = 0.15, R = 5, contact angle 90 deg, particle density 3, seed 2),
every 100 steps up to 1000, read through lb_observables.  The oracle's
values are stored in
tests/golden/lt_c128.json, written by tests/golden/make_lt_golden.py (which
uses only oracle/).  Tolerance: 2 % of the oracle's value."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lt_c128.json")


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_domain_size_and_coverage_follow_the_oracle(precision):
    from paper_1004_4414_gb300 import Simulation, build

    build.build()
    g = json.load(open(GOLDEN))
    p = dict(g["params"])
    p["tau"], p["sc_weight"], p["rho_init"] = tuple(p["tau"]), tuple(p["sc_weight"]), tuple(p["rho_init"])
    sim = Simulation(dict(p, precision=precision))
    sim.init_from_seed(g["seed"])
    assert sim.n_particles[0] == g["n_particles"]
    step = 0
    for k, target in enumerate(g["steps"]):
        sim.step(target - step)
        step = target
        ob = sim.observables(0)  # domain size and coverage computed by the library
        L, cov = np.array(ob["L"]), ob["coverage"]
        Lo = np.array(g["L"][k])
        assert np.all(np.abs(L - Lo) <= 0.02 * Lo), (precision, target, L, Lo)
        assert abs(cov - g["coverage"][k]) <= 0.02 * g["coverage"][k], (precision, target, cov, g["coverage"][k])
    assert sim.observables()["error"] == 0
    sim.close()
