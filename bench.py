"""Throughput of the particle-laden two-component Shan-Chen LB step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload c256|c128|c512|c32|batch|...] [--precision fp32|fp16|bf16]

One "step" is one time step of the whole hot path over the workload: particle
remap with cover/uncover, shell virtual fluid, fused stream-collide with the
Shan-Chen force and moving bounce-back, particle force reduction and MD.
The metric is MLUPS (lattice node updates per second, both components,
every node of the box counted once per step), for FP32, for FP16 / BF16
deviation storage and for the batched sweep, on the same GPU.

With no --workload / --precision the run measures every leg of the metric
and prints one JSON line: the 256^3 FP32 leg is the headline (value, e2e,
roofline), and "legs" holds the 256^3 FP16-deviation, 256^3 BF16-deviation
and 64-box batch legs with the same fields (the batch also with
batch_vs_sequential).  Two roofline fractions are reported per leg:
  roofline.frac       the fused stream-collide kernel alone: its algorithmic
                      bytes per launch over its CUDA-event launch time, against
                      the measured HBM copy bandwidth (the 6800 GB/s
                      fallback when no measurement is available);
  roofline.step_frac  the whole step: MLUPS over the roofline MLUPS of the
                      ideal byte count per node (2 components x 19
                      populations read and written: 304 B in FP32, 152 B in
                      16-bit storage) at the measured HBM bandwidth.
The timed steps replay the CUDA graphs exactly as lb_step does; the fused
kernel's launch time comes from a separate pass of the same steps with
per-launch CUDA events.  End to end through the C ABI with host buffers:
  e2e             import of every box's storage-format state from pinned
                  host memory (lb_import_state_native), the K steps, export
                  into pinned host memory (lb_export_state_native);
  e2e_fp64_state  the same with the FP64 canonical state (lb_import_state /
                  lb_export_state): twice the population bytes of FP32
                  storage, four times those of 16-bit storage.

Workloads (seeded, synthetic; the paper's runs are synthetic as well):
  c256  256^3, fluid ratio 60:40 of total density 0.7, alpha = 0.20, R = 5,
        contact angle 77 deg (colour -0.0294), g = 0.08 (default)
  c256p the c256 parameters on a 128^3 box (small case for profiler captures)
  c256s 256^3 with 5007 prolate spheroids (semi-axes 4, 4, 6), alpha = 0.12
  c128  128^3, 50:50, alpha = 0.15, R = 5, 90 deg
  c512  512^3, 50:50, alpha = 0.20, R = 5, 90 deg
  c32   32^3, 0.7 / 0.7, 16 spheres R = 4 (parity configuration)
  batch 64 boxes with edges from {48, 64, 96, 128}, contact angle 60-120 deg,
        alpha 0.05-0.25, fluid ratio 50:50-70:30, one launch per phase

For N > 1 (torchrun) every rank runs its own copy of the workload on its
GPU (independent problems, no communication): weak scaling, value = all
ranks' node updates / max-over-ranks time.  --impl reference times the FP64
CPU oracle (the only other implementation of the method) on a bounded
sample of the same workload on the host cores.
"""
import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PROFILES = os.path.join(ROOT, "profiles")
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal
# ideal bytes per node and step: 2 components x 19 populations, read and written
IDEAL_BYTES = {"fp32": 2 * 19 * 4 * 2, "fp16": 2 * 19 * 2 * 2, "bf16": 2 * 19 * 2 * 2, "fp64": 2 * 19 * 8 * 2}
# the legs of the metric measured by a default run: (workload, precision)
DEFAULT_LEGS = (("c256", "fp32"), ("c256", "fp16"), ("c256", "bf16"), ("batch", "fp32"))
KERNEL_SOURCES = ("lb_step_kernel.cuh", "lb_step_split.cuh", "lb_common.cuh")


def workload_params(name, precision="fp32"):
    # particle density 3: with the explicit particle update, spheres of
    # density 1 in fluid of total density 0.7 that touch in clusters drive a
    # growing fluid mode after ~200 steps at 256^3 (the FP64 oracle does the
    # same); at 3 the workloads stay stable for thousands of steps
    base = dict(tau=(1.0, 1.0), g_br=0.08, rho0=1.0, sc_weight=(2.0, 1.0), noise_amp=0.01, radius=5.0,
                particle_density=3.0, k_hertz=100.0, precision=precision)
    if name == "c256":
        return [dict(base, nx=256, ny=256, nz=256, n_particles=-1, volume_fraction=0.20,
                     rho_init=(0.42, 0.28), contact_angle_deg=77.0)], 3
    if name == "c256p":
        # profiling case: the c256 parameters on a 128^3 box (state > L2, ~1 GB)
        return [dict(base, nx=128, ny=128, nz=128, n_particles=-1, volume_fraction=0.20,
                     rho_init=(0.42, 0.28), contact_angle_deg=77.0)], 3
    if name == "c256s":
        # the 256^3 fluid with prolate spheroids (semi-axes 4, 4, 6) at a
        # volume fraction their bounding spheres can be placed at (0.27)
        return [dict(base, nx=256, ny=256, nz=256, n_particles=-1, volume_fraction=0.12, radius=4.0, aspect=1.5,
                     rho_init=(0.42, 0.28), contact_angle_deg=77.0)], 3
    if name == "c128":
        return [dict(base, nx=128, ny=128, nz=128, n_particles=-1, volume_fraction=0.15,
                     rho_init=(0.35, 0.35), contact_angle_deg=90.0)], 2
    if name == "c512":
        return [dict(base, nx=512, ny=512, nz=512, n_particles=-1, volume_fraction=0.20,
                     rho_init=(0.35, 0.35), contact_angle_deg=90.0)], 5
    if name == "c32":
        return [dict(base, nx=32, ny=32, nz=32, n_particles=16, radius=4.0, rho_init=(0.7, 0.7),
                     particle_density=2.0, contact_angle_deg=90.0)], 1
    if name == "batch":
        import numpy as np

        rng = np.random.default_rng(4)
        boxes = []
        for b in range(64):
            L = int(rng.choice([48, 64, 96, 128]))
            theta = float(rng.uniform(60.0, 120.0))
            alpha = float(rng.uniform(0.05, 0.25))
            red = float(rng.uniform(0.5, 0.7))
            boxes.append(dict(base, nx=L, ny=L, nz=L, n_particles=-1, volume_fraction=alpha,
                              rho_init=(0.7 * red, 0.7 * (1.0 - red)), contact_angle_deg=theta))
        return boxes, 4
    raise ValueError(name)


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash():
    """Hash of the fused kernel's sources with comments and blank space
    removed, so that a comment edit does not invalidate the DRAM counters."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1004_4414_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def fused_kernel_name(split):
    return "k_step_split" if split else "k_step"


def ncu_traffic(workload, precision, split):
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary, if it was taken on the same kernel and its current source."""
    path = os.path.join(PROFILES, "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get("%s_%s_%s" % (workload, precision, fused_kernel_name(split)))
        if e and e.get("kernel_hash") == kernel_hash():
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks during the timed region (200 ms period)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = float(f[2])
                except ValueError:
                    continue
                for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                   f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id(device):
    """nvidia-smi addresses GPUs by UUID regardless of CUDA_VISIBLE_DEVICES."""
    import torch

    try:
        u = str(torch.cuda.get_device_properties(device).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(device.index or 0)


def fused_bytes(sim, precision):
    """Algorithmic bytes of one launch of the fused kernel: every fluid node
    reads and writes its 2 x 18 moving populations (FP32: 4 B each; 16-bit
    deviation storage: 2 B; the rest population is the density minus them
    and is not stored), every node reads and writes 2 densities (4 B each,
    8 B in FP64) and reads 1 flag byte."""
    pop = {"fp32": 2 * 18 * 4, "fp64": 2 * 18 * 8, "fp16": 2 * 18 * 2, "bf16": 2 * 18 * 2}[precision]
    rs = 8 if precision == "fp64" else 4
    total = 0
    for b in range(sim.nb):
        ob = sim.observables(b)
        total += ob["n_fluid"] * pop * 2 + sim.n_nodes[b] * (2 * rs * 2 + 1)
    return total


def job_throughput(node_updates, seconds, world, device):
    """Whole-job MLUPS over all ranks: the node updates of every rank divided
    by the slowest rank's time.  Returns (MLUPS, max-over-ranks ms)."""
    import torch

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    n = torch.tensor([float(node_updates)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(n, op=torch.distributed.ReduceOp.SUM)
    return float(n.item()) / float(t.item()) / 1e6, float(t.item()) * 1e3


def run_ours(args, rank, world, device):
    import numpy as np
    import torch

    from paper_1004_4414_gb300 import Simulation, build

    build.build()
    boxes, seed = workload_params(args.workload, args.precision)
    sim = Simulation(boxes, device=device)
    sim.init_from_seed(seed + 1000 * rank)
    nodes = sum(sim.n_nodes)
    stream = sim.stream
    # warm-up: the autotuner times candidate block shapes on these boxes,
    # then W plain steps
    from paper_1004_4414_gb300.autotune import autotune

    if args.tiling:
        tiling = tuple(int(v) for v in args.tiling.split(","))
        sim.set_tiling(*tiling)
    else:
        tiling, _ = autotune(sim)
    # the timed steps start from the seeded state again
    sim.init_from_seed(seed + 1000 * rank)
    sim.step(args.warmup)
    sim.sync()
    # host copy of the state after the warm-up, the input of the end-to-end leg
    def pinned_like(a):
        out = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True).numpy()
        out[...] = a
        return out

    states_in, outs, h2d = [], [], 0
    for b in range(sim.nb):
        st = sim.export_state(b)
        states_in.append(dict(st, f=pinned_like(st["f"]), owner=pinned_like(st["owner"])))
        outs.append((pinned_like(st["f"]), pinned_like(st["owner"])))
        h2d += st["f"].nbytes + st["owner"].nbytes + st["particles"].nbytes

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- device-timed region: inputs resident in HBM (the state is larger
    # than the 129 MB L2, so no flush is needed between steps).  The steps
    # replay the CUDA graphs exactly as lb_step does for a caller.
    barrier()
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_id(device)) as clk:
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize(device)
    barrier()
    ms = e0.elapsed_time(e1)
    sim.sync()
    clocks = clk.summary()
    value, ms_max = job_throughput(nodes * args.steps, ms * 1e-3, world, device)

    # ---- a separate pass of the same steps with per-launch CUDA events
    # around the fused kernel (kernel-by-kernel launches instead of graph
    # replays), for the fused kernel's launch time and the launch count
    prof_steps = min(args.steps, 20)
    sim.set_profiling(True)
    sim.step(prof_steps)
    fused_ms, fused_n, total_launches = sim.kernel_time()
    phases = {k: v / prof_steps for k, v in sim.phase_times().items()}
    sim.set_profiling(False)
    sim.sync()
    launches = int(round(total_launches / max(prof_steps, 1) * args.steps))

    # ---- roofline of the fused kernel
    bytes_launch = fused_bytes(sim, args.precision)
    avg_ms = fused_ms / max(fused_n, 1)
    achieved = bytes_launch / (avg_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()

    # ---- end to end through the C ABI with host buffers: import the
    # post-warm-up state from pinned host memory, K steps, export it back.
    # The boxes of one handle share the step counter, so the states are
    # imported as of the current step (the exported state is canonical).
    # One untimed import / export first (the warm-up of the copy path: the
    # first transfers through freshly pinned pages are slower).
    def stamp():
        cur = sim.observables(0)["step"]
        for st in states_in:
            st["meta"] = st["meta"].copy()
            st["meta"][0] = cur

    stamp()
    for b in range(sim.nb):
        sim.import_state(b, states_in[b])
        sim.export_state(b, f_out=outs[b][0], owner_out=outs[b][1])
    stamp()
    barrier()
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for b in range(sim.nb):
        sim.import_state(b, states_in[b])
    sim.step(args.steps)
    sim.sync()
    for b in range(sim.nb):
        sim.export_state(b, f_out=outs[b][0], owner_out=outs[b][1])
    t1 = time.perf_counter()
    barrier()
    e2e_value, _ = job_throughput(nodes * args.steps, t1 - t0, world, device)
    e2e_fp64 = {"value": e2e_value, "unit": "MLUPS",
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": h2d / args.steps,
                "what": "lb_import_state of every box (FP64 canonical state) from pinned host memory + lb_step(K) + "
                        "lb_export_state of every box into pinned host memory"}

    # ---- the same through the storage-format state (the checkpoint a run
    # restarts from: the device's own population bytes, no FP64 conversion).
    # Its bytes follow the step's parity, so the input is exported at the
    # current step, where the import puts it.
    nstates_in, nouts, nh2d = [], [], 0
    for b in range(sim.nb):
        st = sim.export_state_native(b)
        nstates_in.append(dict(st, state=pinned_like(st["state"]), owner=pinned_like(st["owner"])))
        nouts.append((pinned_like(st["state"]), pinned_like(st["owner"])))
        nh2d += st["state"].nbytes + st["owner"].nbytes + st["particles"].nbytes
    for b in range(sim.nb):
        sim.import_state_native(b, nstates_in[b])
        sim.export_state_native(b, state_out=nouts[b][0], owner_out=nouts[b][1])
    barrier()
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for b in range(sim.nb):
        sim.import_state_native(b, nstates_in[b])
    sim.step(args.steps)
    sim.sync()
    for b in range(sim.nb):
        sim.export_state_native(b, state_out=nouts[b][0], owner_out=nouts[b][1])
    t1 = time.perf_counter()
    barrier()
    e2e_value, _ = job_throughput(nodes * args.steps, t1 - t0, world, device)
    e2e = {"value": e2e_value, "unit": "MLUPS",
           "h2d_bytes_per_step": nh2d / args.steps, "d2h_bytes_per_step": nh2d / args.steps,
           "what": "lb_import_state_native of every box (storage-format state) from pinned host memory + "
                   "lb_step(K) + lb_export_state_native of every box into pinned host memory"}
    ob = sim.observables(0)
    n_fluid = sum(sim.observables(b)["n_fluid"] for b in range(sim.nb))
    seq = None
    if sim.nb > 1 and not args.no_sequential:
        seq_value, seq_ms = sequential_boxes(args, boxes, seed + 1000 * rank, device)
        seq = {"sequential_mlups": seq_value, "batched_mlups": value, "ratio": value / seq_value,
               "sequential_ms": seq_ms, "what": "the same boxes and states, one handle per box, run one after another"}
    return dict(value=value, ms=ms_max, fused_ms=avg_ms, fused_n=fused_n, bytes=bytes_launch, achieved=achieved,
                peak=peak, peak_kind=peak_kind, clocks=clocks, e2e=e2e, e2e_fp64=e2e_fp64, launches=launches,
                nodes=nodes, phases=phases,
                n_particles=sum(sim.n_particles), error=ob["error"], n_fluid=n_fluid, tiling=tiling, seq=seq)


def sequential_boxes(args, boxes, seed, device):
    """The boxes of a batch run one after another, each on its own handle
    (its own autotuned tiling), from the same seeded states (box b of a
    batch uses seed + b): MLUPS over the summed CUDA-event time of K steps."""
    import torch

    from paper_1004_4414_gb300 import Simulation
    from paper_1004_4414_gb300.autotune import autotune

    updates, ms = 0, 0.0
    for b, box in enumerate(boxes):
        sim = Simulation([box], device=device)
        sim.init_from_seed(seed + b)
        autotune(sim)
        sim.init_from_seed(seed + b)
        sim.step(args.warmup)
        sim.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(args.steps)
        e1.record(sim.stream)
        torch.cuda.synchronize(device)
        ms += e0.elapsed_time(e1)
        updates += sim.n_nodes[0] * args.steps
        sim.close()
    return updates / (ms * 1e-3) / 1e6, ms


def oracle_sample(workload, budget_s=12.0):
    """Time the FP64 oracle on the host cores on the first box of the
    workload: init, then steps until the budget is used (at least one)."""
    from oracle import ref

    boxes, seed = workload_params(workload, "fp64")
    p = {k: v for k, v in boxes[0].items() if k not in ("precision", "contact_angle_deg")}
    theta = boxes[0].get("contact_angle_deg", 90.0)
    p["color"] = (theta - 90.0) / 442.0 if theta is not None and not math.isnan(theta) else 0.0
    o = ref.Oracle(**p)
    o.init_from_seed(seed)
    N = p["nx"] * p["ny"] * p["nz"]
    steps, spent = 0, 0.0
    while steps == 0 or spent < budget_s:
        t0 = time.perf_counter()
        o.step(1)
        spent += time.perf_counter() - t0
        steps += 1
        if spent > 3 * budget_s:
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dict(value=N * steps / spent / 1e6, steps=steps, seconds=spent, cores=cores, N=N,
                sample="%d step(s) of box 0 of %s (%d^3 nodes, %d particles) after seeded init" %
                       (steps, workload, p["nx"], o.np))


def oracle_steps(workload, steps, warmup, edge=64):
    """Reference arm: the FP64 oracle on the host cores, W untimed and K
    timed steps, each step one oracle step of a bounded sample of the
    workload: a box of at most edge^3 nodes with the parameters of its first
    box (same volume fraction, radius, densities and wetting; the particle
    count scales with the volume)."""
    from oracle import ref

    boxes, seed = workload_params(workload, "fp64")
    p = {k: v for k, v in boxes[0].items() if k not in ("precision", "contact_angle_deg")}
    theta = boxes[0].get("contact_angle_deg", 90.0)
    p["color"] = (theta - 90.0) / 442.0 if theta is not None and not math.isnan(theta) else 0.0
    full = (p["nx"], p["ny"], p["nz"])
    for k in ("nx", "ny", "nz"):
        p[k] = min(p[k], edge)
    if p.get("n_particles", -1) >= 0:  # an explicit count scales with the volume
        frac = p["nx"] * p["ny"] * p["nz"] / float(full[0] * full[1] * full[2])
        p["n_particles"] = int(round(p["n_particles"] * frac))
    o = ref.Oracle(**p)
    o.init_from_seed(seed)
    o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    spent = time.perf_counter() - t0
    N = p["nx"] * p["ny"] * p["nz"]
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dict(value=N * steps / spent / 1e6, steps=steps, seconds=spent, cores=cores, N=N,
                sample="%d timed step(s) after %d warm-up step(s) of a %dx%dx%d box with the parameters of box 0 "
                       "of %s (%dx%dx%d; %d particles in the sample)" %
                       (steps, warmup, p["nx"], p["ny"], p["nz"], workload, full[0], full[1], full[2], o.np))


NAMES = {"c256": "256^3 60:40 alpha=0.20 R=5 theta=77deg", "c128": "128^3 50:50 alpha=0.15 R=5 theta=90deg",
         "c256p": "128^3 with the 256^3 parameters (profiling case)",
         "c256s": "256^3 60:40 alpha=0.12 prolate spheroids 4x4x6 theta=77deg",
         "c512": "512^3 50:50 alpha=0.20 R=5 theta=90deg", "c32": "32^3 16 spheres R=4",
         "batch": "64 boxes {48,64,96,128}^3 theta 60-120 alpha 0.05-0.25 ratio 50:50-70:30"}
DTYPES = {"fp32": "f32", "fp16": "f16-dev/f32", "bf16": "bf16-dev/f32"}


def leg_fields(args, r):
    """The fields of one measured leg (workload, precision)."""
    traffic = ncu_traffic(args.workload, args.precision, r["tiling"][2])
    ideal = IDEAL_BYTES[args.precision]
    roof_mlups = r["peak"] * 1e3 / ideal  # GB/s / (B/node) -> MLUPS
    return {
        "value": r["value"], "unit": "MLUPS", "ms_per_step": r["ms"] / args.steps,
        "dtype": DTYPES[args.precision],
        "config": {"workload": NAMES[args.workload], "precision": args.precision, "nodes": r["nodes"],
                   "fluid_nodes": r["n_fluid"], "particles": r["n_particles"],
                   "l2": "state larger than L2 (no flush needed)",
                   "tiling": {"ty": r["tiling"][0], "cz": r["tiling"][1], "split": r["tiling"][2]}},
        "roofline": {"bound": "hbm", "achieved": r["achieved"], "peak": r["peak"], "unit": "GB/s",
                     "frac": r["achieved"] / r["peak"], "traffic": traffic,
                     "peak_kind": r["peak_kind"], "kernel": fused_kernel_name(r["tiling"][2]) + " (fused stream-collide)",
                     "bytes_per_launch": r["bytes"], "launch_ms": r["fused_ms"],
                     "frac_nominal": r["achieved"] / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                     "dram_gbs": traffic / (r["fused_ms"] * 1e6) if traffic else None,
                     "step_frac": r["value"] / roof_mlups, "step_roofline_mlups": roof_mlups,
                     "ideal_bytes_per_node": ideal},
        "fluid_mlups": r["value"] * r["n_fluid"] / r["nodes"],
        "phases_ms_per_step": r["phases"],
        "e2e": r["e2e"],
        "e2e_fp64_state": r["e2e_fp64"],
        "clocks": r["clocks"],
        "gpu_launches": r["launches"],
        "batch_vs_sequential": r["seq"],
        "device_error": r["error"],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None, choices=["c256", "c256p", "c256s", "c128", "c512", "c32", "batch"],
                    help="one workload only (default: every leg of the metric)")
    ap.add_argument("--precision", default=None, choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sequential", action="store_true", help="batch: skip the one-box-at-a-time comparison")
    ap.add_argument("--tiling", default=None, metavar="TY,CZ,SPLIT",
                    help="fixed block shape of the fused kernel instead of the autotuner's (for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload is None and args.precision is None and args.tiling is None:
        legs = list(DEFAULT_LEGS)
    else:
        legs = [(args.workload or "c256", args.precision or "fp32")]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    metric = "MLUPS and % of HBM roofline: FP32 vs BF16/FP16-storage vs batched, same GPU"

    if args.impl == "reference":
        if rank != 0:
            return
        workload = legs[0][0]
        r = oracle_steps(workload, args.steps, args.warmup)
        line = {"impl": "reference", "metric": metric, "value": r["value"], "unit": "MLUPS", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["seconds"] / r["steps"] * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": NAMES[workload], "precision": "fp64 (oracle)"},
                "cpu_baseline": {"value": r["value"], "unit": "MLUPS", "cores": r["cores"], "kind": "oracle",
                                 "sample": r["sample"]},
                "e2e": {"value": r["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch

    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    device = torch.device("cuda", local)
    results = []
    for workload, precision in legs:
        a = argparse.Namespace(**vars(args))
        a.workload, a.precision = workload, precision
        r = run_ours(a, rank, world, device)
        results.append((a, r))
        torch.cuda.empty_cache()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        c = oracle_sample(legs[0][0])
        cpu = {"value": c["value"], "unit": "MLUPS", "cores": c["cores"], "kind": "oracle", "sample": c["sample"]}
    head_args, head = results[0]
    f = leg_fields(head_args, head)
    line = {"metric": metric, "value": f["value"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": f["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": f["dtype"], "data": "synthetic"}
    line.update({k: v for k, v in f.items() if k not in line})
    line["cpu_baseline"] = cpu
    if len(results) > 1:
        line["legs"] = {}
        for a, r in results[1:]:
            name = "%s_%s" % (a.workload, a.precision)
            line["legs"][name] = leg_fields(a, r)
        fp32 = head["value"]
        line["legs_vs_fp32"] = {n: v["value"] / fp32 for n, v in line["legs"].items()}
        line["gpu_launches_all_legs"] = sum(r["launches"] for _, r in results)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
