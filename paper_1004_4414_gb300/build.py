"""Build the sm_103a shared library paper_1004_4414_gb300/_build/liblbpart.so.

Six translation units are compiled in parallel with nvcc for
compute_103a / sm_103a: the host C ABI (lb_api.cu), the allocation-free
field sums (lb_noalloc.cu) and one instantiation of
the precision-dependent kernels per population storage type
(lb_kern_inst.cu with LB_PREC = 0..3).  Host code is compiled without
floating-point contraction so the seeded sphere placement takes the same
decisions on x86 and Arm hosts.
"""
import os
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblbpart.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(HERE, "..", "include")]


def _sources():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(HERE, "..", "include", "lbpart.h"))
    units = [("lb_api", os.path.join(CSRC, "lb_api.cu"), []),
             ("lb_noalloc", os.path.join(CSRC, "lb_noalloc.cu"), [])]
    for k, name in enumerate(("fp64", "fp32", "fp16", "bf16")):
        units.append(("lb_kern_" + name, os.path.join(CSRC, "lb_kern_inst.cu"), ["-DLB_PREC=%d" % k]))
    return units, hdrs


def build(force=False, verbose=False, extra=()):
    units, hdrs = _sources()
    os.makedirs(OUT, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in hdrs + [u[1] for u in units] + [__file__])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    procs = []
    t0 = time.time()
    for name, src, defs in units:
        obj = os.path.join(OUT, name + ".o")
        cmd = [nvcc, "-c", src, "-o", obj] + ARCH + FLAGS + defs + list(extra)
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((name, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    objs, failed = [], []
    for name, obj, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(name)
        objs.append(obj)
    if failed:
        raise RuntimeError("nvcc failed for: %s" % ", ".join(failed))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc, "-shared", "-o", tmp] + objs + ARCH)
    os.replace(tmp, LIB)
    if verbose:
        sys.stderr.write("built %s in %.1f s\n" % (LIB, time.time() - t0))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
