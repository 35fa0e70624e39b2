"""Late-time domain size L(t) (Eq. eq:domsize) and interface coverage of the
CUDA path against the FP64 oracle on the 128^3 configuration of
test_gpu_lt.py (50:50 of total density 0.7, alpha = 0.15, R = 5, contact
angle 90 deg, particle density 3, seed 2), every 500 steps through the
coarsening, read through lb_observables.  The oracle's values are stored in
tests/golden/lt_c128_long.json, written by
tests/golden/make_lt_long_golden.py (which uses only oracle/).  The
trajectories of the FP32 / 16-bit runs and of the FP64 oracle diverge in
detail (the flow is chaotic); the box averages must not.  Tolerance: 2 %
of the oracle's value for FP32; for 16-bit deviation storage, whose error
of each observable is stated rather than bound to FP32's, 2 % in L and 3 %
in the coverage.  Measured on GB300s, the largest deviation over the 12
checkpoints: FP32 0.4 % (L) and 1.0 % (coverage); FP16 1.0 % and 2.1 %
(1.9 % in another run: single runs differ, the float reductions being
unordered); BF16 1.0 % and 0.5 %."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lt_c128_long.json")
TOL = {"fp32": (0.02, 0.02), "fp16": (0.02, 0.03), "bf16": (0.02, 0.03)}


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_late_domain_size_and_coverage_follow_the_oracle(precision):
    from paper_1004_4414_gb300 import Simulation, build

    build.build()
    g = json.load(open(GOLDEN))
    p = dict(g["params"])
    p["tau"], p["sc_weight"], p["rho_init"] = tuple(p["tau"]), tuple(p["sc_weight"]), tuple(p["rho_init"])
    sim = Simulation(dict(p, precision=precision))
    sim.init_from_seed(g["seed"])
    assert sim.n_particles[0] == g["n_particles"]
    step = 0
    dL, dc = [], []
    for k, target in enumerate(g["steps"]):
        sim.step(target - step)
        step = target
        ob = sim.observables(0)
        assert ob["error"] == 0
        Lo = np.array(g["L"][k])
        dL.append(np.max(np.abs(np.array(ob["L"]) - Lo) / Lo))
        dc.append(abs(ob["coverage"] - g["coverage"][k]) / g["coverage"][k])
    sim.close()
    tL, tc = TOL[precision]
    assert max(dL) <= tL and max(dc) <= tc, (precision, np.round(dL, 4), np.round(dc, 4))
