"""Host-side logic that needs no GPU: the autotuner's candidate filtering,
selection and cache, run against a stand-in for the simulation whose fused
kernel times are given."""
from types import SimpleNamespace

import pytest

from paper_1004_4414_gb300 import autotune as at


class FakeSim:
    """Records the calls the autotuner makes; kernel_time returns the time
    assigned to the tiling that was set last."""

    def __init__(self, dims, times, precision=1, tau=(1.0, 1.0)):
        self.dims = list(dims)
        self._params = [SimpleNamespace(precision=precision, tau=tau) for _ in dims]
        self.times = times
        self.tiling = None
        self.steps = 0
        self.profiling = False
        self.timed = []

    def set_tiling(self, ty, cz, split=0):
        self.tiling = (ty, cz, split)

    def step(self, n=1):
        self.steps += n

    def sync(self):
        pass

    def set_profiling(self, on):
        self.profiling = on

    def kernel_time(self):
        self.timed.append(self.tiling)
        return self.times.get(self.tiling, 9.0) * 4, 4, 60


@pytest.fixture(autouse=True)
def clear_cache():
    at._CACHE.clear()
    yield
    at._CACHE.clear()


def test_picks_the_fastest_candidate_and_leaves_it_set():
    times = {c: 2.0 for c in at.DEFAULT_CANDIDATES}
    times[(16, 32, 1)] = 1.1
    sim = FakeSim([(256, 256, 256)], times)
    best, table = at.autotune(sim)
    assert best == (16, 32, 1) and sim.tiling == best
    assert table[best] == pytest.approx(1.1)
    assert set(table) == set(at.DEFAULT_CANDIDATES)
    assert not sim.profiling


def test_candidates_deeper_than_the_box_are_skipped():
    sim = FakeSim([(64, 64, 20)], {})
    _, table = at.autotune(sim)
    assert all(cz <= 20 or cz == at.DEFAULT_CANDIDATES[0][1] for _, cz, _ in table)
    assert (8, 32, 0) not in table and (4, 16, 0) in table


def test_cache_is_keyed_by_sizes_precision_and_tau():
    times = {c: 2.0 for c in at.DEFAULT_CANDIDATES}
    times[(8, 16, 1)] = 1.0
    a = FakeSim([(128, 128, 128)], times)
    at.autotune(a)
    b = FakeSim([(128, 128, 128)], {})
    best, _ = at.autotune(b)
    assert best == (8, 16, 1) and b.timed == [] and b.tiling == best
    c = FakeSim([(128, 128, 128)], {}, tau=(1.0, 0.8))
    at.autotune(c)
    assert c.timed  # a different tau is tuned again
    d = FakeSim([(128, 128, 128)], {}, precision=2)
    at.autotune(d)
    assert d.timed


def test_two_element_candidates_default_to_one_thread_per_node():
    sim = FakeSim([(64, 64, 64)], {(8, 16, 0): 1.0, (4, 16, 0): 2.0})
    best, _ = at.autotune(sim, candidates=((4, 16), (8, 16)))
    assert best == (8, 16, 0)


def test_traffic_is_used_only_for_the_same_kernel_and_sources(tmp_path, monkeypatch):
    import json

    import bench

    entry = {"kernel_hash": bench.kernel_hash(), "dram_bytes_per_launch": 123.0}
    (tmp_path / "traffic.json").write_text(json.dumps({"c256_fp32_k_step_split": entry}))
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    assert bench.ncu_traffic("c256", "fp32", 1) == 123.0
    assert bench.ncu_traffic("c256", "fp32", 0) is None  # the other fused kernel
    assert bench.ncu_traffic("c256", "fp16", 1) is None
    stale = dict(entry, kernel_hash="0" * 16)
    (tmp_path / "traffic.json").write_text(json.dumps({"c256_fp32_k_step_split": stale}))
    assert bench.ncu_traffic("c256", "fp32", 1) is None


def test_reference_arm_times_a_bounded_sample():
    import bench

    r = bench.oracle_steps("c32", steps=2, warmup=1, edge=16)
    assert r["steps"] == 2 and r["N"] == 16 ** 3 and r["value"] > 0
    assert "16x16x16" in r["sample"] and "32x32x32" in r["sample"]


class _ObsSim:
    """Boxes with given node and fluid-node counts (bench.fused_bytes reads
    nb, n_nodes and observables(b)["n_fluid"])."""

    def __init__(self, boxes):
        self.nb = len(boxes)
        self.n_nodes = [n for n, _ in boxes]
        self._fluid = [f for _, f in boxes]

    def observables(self, b):
        return {"n_fluid": self._fluid[b]}


@pytest.mark.parametrize("prec,per_fluid,per_node", [("fp32", 288, 17), ("fp16", 144, 17), ("bf16", 144, 17),
                                                     ("fp64", 576, 33)])
def test_algorithmic_bytes_count_18_stored_populations(prec, per_fluid, per_node):
    """The roofline numerator: a fluid node reads and writes its 2 x 18 moving
    populations (the rest population is the density minus them and is never
    stored); every node reads one and writes one density per component and
    reads a flag byte."""
    import bench

    sim = _ObsSim([(1000, 800), (64, 0), (27, 27)])
    assert bench.fused_bytes(sim, prec) == (800 + 27) * per_fluid + (1000 + 64 + 27) * per_node
