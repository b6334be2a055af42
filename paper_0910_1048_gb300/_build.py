"""Build libovl.so (the C-ABI library) in-tree with nvcc for sm_103a.

Every translation unit under csrc/ is compiled in parallel into _build/ and linked into
paper_0910_1048_gb300/libovl.so with the CUDA runtime linked statically. The bench's
FMA-throughput probe (fp64_peak.cu beside bench.py, the measured FP64 peak of its roofline)
becomes libfp64_peak.so beside it; it is not part of the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "libovl.so")
PROBE_SRC = os.path.join(ROOT, "fp64_peak.cu")
PROBE_OUT = os.path.join(ROOT, "libfp64_peak.so")
BUILD = os.path.join(ROOT, "_build", "ovl-" + platform.machine())  # objects never cross architectures
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
         "--expt-relaxed-constexpr"]


def _nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libovl.so")
    return exe


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    deps = [src] + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "ovl.h")]
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        if _stale(o, s):
            cmd = [nvcc] + ARCH + FLAGS + (extra or []) + ["-c", s, "-o", o]
            if s.endswith(".cpp"):
                cmd = [nvcc] + FLAGS + (extra or []) + ["-x", "c++", "-c", s, "-o", o]
            jobs.append(cmd)
    probe_obj = os.path.join(BUILD, "fp64_peak.cu.o")
    if not os.path.exists(probe_obj) or os.path.getmtime(probe_obj) < os.path.getmtime(PROBE_SRC):
        jobs.append([nvcc] + ARCH + FLAGS + (extra or []) + ["-c", PROBE_SRC, "-o", probe_obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    stamp = os.path.join(BUILD, "libovl.machine")
    fresh = os.path.exists(stamp) and open(stamp).read() == platform.machine()
    if jobs or not os.path.exists(OUT) or not os.path.exists(PROBE_OUT) or not fresh:
        cmd = [nvcc] + ARCH + ["-shared", "-o", OUT] + objs + ["-lpthread", "-ldl", "-lrt"]
        run(cmd)
        run([nvcc] + ARCH + ["-shared", "-o", PROBE_OUT, probe_obj])
        with open(stamp, "w") as f:
            f.write(platform.machine())
    return OUT


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
