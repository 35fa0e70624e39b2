"""The stored oracle values (tests/golden/) have the properties their GPU
tests rely on; CPU only."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_layers_golden_coverage_is_informative():
    """On the layered 112^3 case the interface coverage stays well inside
    (0, 1) and changes over the run, so comparing it tests something."""
    g = json.load(open(os.path.join(GOLDEN, "lt_layers112.json")))
    cov = np.array(g["coverage"])
    assert len(cov) == len(g["steps"]) == len(g["L"])
    assert np.all(cov < 0.95) and np.all(cov > 0.05)
    assert cov.max() - cov.min() > 0.05
    assert g["source"].startswith("oracle/")


def test_c128_golden_shape():
    g = json.load(open(os.path.join(GOLDEN, "lt_c128.json")))
    assert len(g["steps"]) == len(g["L"]) == len(g["coverage"]) == 10
    assert np.all(np.array(g["L"]) > 0)
