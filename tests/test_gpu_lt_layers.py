"""Domain size (Eq. eq:domsize) and interface coverage through the C ABI
(lb_observables) against the FP64 oracle, on a case where the coverage is
well below 1 and changes: an 80^3 box of alternating red and blue layers
(period 40 along z) holding 147 spheres (R = 5, about 15 % of the volume,
particle density 3, neutral wetting, g = 0.08), every 250 steps up to 2500.
Spheres inside a layer see one phase, spheres on an interface both.  The
oracle's values are stored in tests/golden/lt_layers80.json, written by
tests/golden/make_lt_layers_golden.py (oracle/ and lbinputs only).
Tolerance: 2 % of the oracle's value, for FP32 and for FP16 / BF16
deviation storage."""
import json
import os

import numpy as np
import pytest

import lbinputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lt_layers80.json")


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_layers_domain_size_and_coverage_follow_the_oracle(precision):
    from paper_1004_4414_gb300 import Simulation, build

    build.build()
    g = json.load(open(GOLDEN))
    p = dict(g["params"])
    p["tau"], p["sc_weight"], p["rho_init"] = tuple(p["tau"]), tuple(p["sc_weight"]), tuple(p["rho_init"])
    shape = (p["nx"], p["ny"], p["nz"])
    rho = lbinputs.layers(shape, **g["layers"])
    parts = lbinputs.spheres(shape, **g["spheres"])
    sim = Simulation(dict(p, precision=precision))
    sim.init_fields(0, rho, particles=parts)
    step = 0
    for k, target in enumerate(g["steps"]):
        sim.step(target - step)
        step = target
        ob = sim.observables()
        L, cov = ob["L"], ob["coverage"]
        Lo = np.array(g["L"][k])
        assert np.all(np.abs(L - Lo) <= 0.02 * Lo), (precision, target, L, Lo)
        assert abs(cov - g["coverage"][k]) <= 0.02 * g["coverage"][k], (precision, target, cov, g["coverage"][k])
        assert ob["error"] == 0
    sim.close()
