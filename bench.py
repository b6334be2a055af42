"""Benchmark: sign(H_W(mu)) b solves per second on GB300.

One step = one pass of the hot path over one batch: for each mu of the workload, one solve
x = sign(H_W(mu)) b through ovl_apply_sign (LR deflation set, Lanczos or multishift
iteration, sign of the projected matrix, combine), inputs resident in HBM. L2 is flushed
(a 256 MB write) between timed steps. `e2e` repeats the steps through the same call with
host buffers (copies inside the timed region). `roofline` reports the dominant kernel (the
fused pair stencil) from CUDA events recorded around its launches inside the library.
The default workload is 12^4, mu = 0.3, plain FP64 two-sided Lanczos (Algorithm 4) to 1e-8.

Beside the headline the line carries its companions (COMPANIONS: the same problem by the
multishift BiCG with FP32 or FP16 12-real links under FP64 reliable updates, with their speedup
over the line's value, and the 16-source 16^4 batch), `lattice8_defl16` (8^4 with 16 deflated
eigenpairs: error at k = 600 and the k reaching 1e-10), `dslash` (kernel-only stencil bandwidth on
32^4) and `serving` (a bounded sample of the serving stream: p50/p99 latency, solves/s, success
rate); `--no-extras` skips them. `cpu_baseline` and `--impl reference` time the oracle (the plain C
FP64 two-sided Lanczos with numpy's eigendecomposition of H_k) on the host cores at the GPU's k.

Multi-GPU: replicas only (each rank solves its own copies, no collective on the data path);
value = solves of all ranks / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import json
from concurrent.futures import ThreadPoolExecutor
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sgn(H_W)b solves/s at rel.err 1e-8"
UNIT = "solves/s"
M_W = -2.0  # Wilson mass of the paper's configurations (Section 6)

# Workloads: the lattice, chemical potentials, method and precision of one step.
WORKLOADS = {
    # 8^4, n = 49152, mu in {0, 0.1, 0.3}, 16 deflated critical eigenpairs per mu, FP64 direct
    # two-sided Lanczos-LR (Algorithm 4), stopping at the metric's 1e-8. The configuration's
    # k <= 600 does not reach 1e-8 at mu = 0.3 with 16 deflated vectors on this ensemble, so
    # k_max is 2000 and the k actually used is reported.
    "lattice8_mu0-0.1-0.3_defl16_direct_f64": dict(dims=(8, 8, 8, 8), mus=(0.0, 0.1, 0.3), m=16, method="direct",
                                                     precision="f64", tol=1e-8, k_max=2000),
    # same lattice and deflation, rational variant (Algorithm 3 + Neuberger, Eq. no_of_poles)
    "lattice8_mu0-0.1-0.3_defl16_multishift_f64": dict(dims=(8, 8, 8, 8), mus=(0.0, 0.1, 0.3), m=16,
                                                         method="multishift", precision="f64", tol=1e-8,
                                                         k_max=5000),
    # the same step in mixed precision: multishift BiCG with FP16 12-real links (or FP32 links,
    # the `_f32_f64rel` line, the faster one) and FP32 vectors, FP64 reliable updates down to the
    # metric's 1e-8
    "lattice8_mu0-0.1-0.3_defl16_multishift_f16links_f64rel": dict(dims=(8, 8, 8, 8), mus=(0.0, 0.1, 0.3), m=16,
                                                                     method="multishift", precision="f16",
                                                                     tol=1e-8, k_max=5000),
    "lattice8_mu0-0.1-0.3_defl16_multishift_f32_f64rel": dict(dims=(8, 8, 8, 8), mus=(0.0, 0.1, 0.3), m=16,
                                                                method="multishift", precision="f32",
                                                                tol=1e-8, k_max=5000),
    # 12^4, mu = 0.3: multishift BiCG with 20 Zolotarev poles on [|lambda|_min, |lambda|_max] from a
    # spectrum estimate, FP16 12-real links and FP32 vectors under FP64 reliable updates, 1e-8;
    # and the FP32 direct method (FP64 scalars and sign(H_k)), whose FP32 vectors bound it near 1e-5
    "lattice12_mu0.3_multishift_zolo20_f16links_f64rel": dict(dims=(12, 12, 12, 12), mus=(0.3,), m=0,
                                                               method="multishift", precision="f16", tol=1e-8,
                                                               k_max=8000, rational="zolotarev", s=20),
    "lattice12_mu0.3_direct_f32": dict(dims=(12, 12, 12, 12), mus=(0.3,), m=0, method="direct", precision="f32",
                                       tol=1e-5, k_max=3000),
    # the plain FP64 two-sided Lanczos path on the same 12^4 problem at 1e-8, with the mixed-precision
    # multishift line above as its companion (speedup reported in the line)
    "lattice12_mu0.3_direct_f64": dict(dims=(12, 12, 12, 12), mus=(0.3,), m=0, method="direct", precision="f64",
                                       tol=1e-8, k_max=3000),
    # 16^4, mu = 0.2 at 1e-8: FP64 direct on batches of 4 sources (16 sources at this k do not fit in
    # HBM: the basis is nrhs x k x 12.6 MB) against the mixed-precision multishift on all 16 at once
    "lattice16_mu0.2_nrhs4_direct_f64": dict(dims=(16, 16, 16, 16), mus=(0.2,), m=0, method="direct",
                                             precision="f64", tol=1e-8, k_max=2500, nrhs=4),
    "lattice16_mu0.2_nrhs16_multishift_f16links_f64rel": dict(dims=(16, 16, 16, 16), mus=(0.2,), m=0,
                                                               method="multishift", precision="f16", tol=1e-8,
                                                               k_max=8000, rational="zolotarev", s=20, nrhs=16),
    # the same two mixed-precision solves with FP32 links (FP32 vectors, FP64 reliable updates)
    "lattice12_mu0.3_multishift_zolo20_f32_f64rel": dict(dims=(12, 12, 12, 12), mus=(0.3,), m=0,
                                                          method="multishift", precision="f32", tol=1e-8,
                                                          k_max=8000, rational="zolotarev", s=20),
    "lattice16_mu0.2_nrhs16_multishift_f32_f64rel": dict(dims=(16, 16, 16, 16), mus=(0.2,), m=0,
                                                          method="multishift", precision="f32", tol=1e-8,
                                                          k_max=8000, rational="zolotarev", s=20, nrhs=16),
    # the same FP64 solve on all 16 sources in one batch by the two-pass strategy (Section 2.3): three
    # basis vectors per source instead of k, twice the stencil work
    "lattice16_mu0.2_nrhs16_direct_f64_twopass": dict(dims=(16, 16, 16, 16), mus=(0.2,), m=0, method="direct",
                                                      precision="f64", tol=1e-8, k_max=2500, nrhs=16, two_pass=1),
    # 16^4, mu = 0.2, 16 Gaussian sources in one batch sharing the links, FP32 vectors with FP64
    # recurrence scalars and sign(H_k); FP32 vectors bound the attainable accuracy near 1e-5
    "lattice16_mu0.2_nrhs16_direct_f32": dict(dims=(16, 16, 16, 16), mus=(0.2,), m=0, method="direct",
                                              precision="f32", tol=1e-5, k_max=1500, nrhs=16),
    # 12^4, mu = 0.3: restarted FOM-LR (Algorithm 1) on A^2, k = 40 per cycle, 20 Zolotarev poles, FP64
    "lattice12_mu0.3_fom_zolo20_f64": dict(dims=(12, 12, 12, 12), mus=(0.3,), m=0, method="fom", precision="f64",
                                           tol=1e-8, k_max=40000, rational="zolotarev", s=20, restart_k=40),
    # 4^4 smoke-sized case (the oracle finishes it in seconds)
    "lattice4_mu0.3_direct_f64": dict(dims=(4, 4, 4, 4), mus=(0.3,), m=0, method="direct", precision="f64",
                                      tol=1e-8, k_max=1200),
}
DEFAULT_WORKLOAD = "lattice12_mu0.3_direct_f64"

# Lines carried beside a headline workload in the same JSON object (same GPU, same run): the
# mixed-precision companions of the same problem at the same tolerance (their speedup over the
# headline's plain FP64 two-sided Lanczos value is reported), and the 16-source batch.
COMPANIONS = {
    "lattice12_mu0.3_direct_f64": [
        ("mixed_precision", "lattice12_mu0.3_multishift_zolo20_f32_f64rel"),
        ("mixed_precision_f16links", "lattice12_mu0.3_multishift_zolo20_f16links_f64rel"),
        ("fom_restarted", "lattice12_mu0.3_fom_zolo20_f64"),
        ("lattice16_nrhs16_mixed", "lattice16_mu0.2_nrhs16_multishift_f32_f64rel"),
        ("lattice16_nrhs16_direct_f32", "lattice16_mu0.2_nrhs16_direct_f32"),
    ],
    "lattice8_mu0-0.1-0.3_defl16_direct_f64": [
        ("mixed_precision", "lattice8_mu0-0.1-0.3_defl16_multishift_f32_f64rel")],
    "lattice16_mu0.2_nrhs4_direct_f64": [("mixed_precision", "lattice16_mu0.2_nrhs16_multishift_f32_f64rel"),
                                         ("two_pass_16_sources", "lattice16_mu0.2_nrhs16_direct_f64_twopass")],
}

# Krylov dimension k the GPU's FP64 direct solve reaches on each workload and mu (seed-0 links,
# seed-1000 source), measured on a GB300. The reference arm runs the oracle for exactly these k
# (the same amount of Lanczos work); the GPU arm reports its own k beside them.
K_TABLE = {
    "lattice12_mu0.3_direct_f64": {0.3: 1250},
    "lattice8_mu0-0.1-0.3_defl16_direct_f64": {0.0: 730, 0.1: 825, 0.3: 1125},
    "lattice4_mu0.3_direct_f64": {0.3: 1000},
}

# The 8^4 configuration with 16 deflated critical eigenpairs per mu: the error attained at a fixed
# k = 600 and the k that reaches 1e-10 (FP64 direct method).
C2 = dict(workload="lattice8_mu0-0.1-0.3_defl16_direct_f64", k_fixed=600, tol=1e-10, k_max=3000)

# Algorithmic traffic / work of one launch of the fused pair stencil per site: per right-hand
# side two spinors in (neighbours read once each: 2 x 24 reals) and two out; the 4 links of a site
# (18 reals each; FP16 12-real: 12 halves) once per launch, shared by all right-hand sides of a
# batch; flops: 2 x 1368 per site and right-hand side.
PAIR_LINK_BYTES_PER_SITE = {"f64": 576, "f32": 288, "f16": 96}
PAIR_SPINOR_BYTES_PER_SITE = {"f64": 4 * 192, "f32": 4 * 96, "f16": 4 * 96}
PAIR_BYTES_PER_SITE = {k: PAIR_LINK_BYTES_PER_SITE[k] + PAIR_SPINOR_BYTES_PER_SITE[k] for k in PAIR_LINK_BYTES_PER_SITE}
PAIR_FLOPS_PER_SITE = 2 * 1368


def pair_bytes(prec, vol, nrhs):
    """Algorithmic bytes of one pair-stencil launch over `nrhs` right-hand sides."""
    return vol * (PAIR_LINK_BYTES_PER_SITE[prec] + nrhs * PAIR_SPINOR_BYTES_PER_SITE[prec])

# FP64 FMA throughput of a GB300 in TFLOP/s (the FMA-chain probe fp64_peak.cu; the
# bench runs the probe itself and uses this value only when the probe library is missing)
FP64_PEAK_TFLOPS = 1.256

# DRAM bytes (read + write) per launch of the dominant kernel from one ncu capture (cold L2, every
# pass flushed), keyed (kernel, precision, lattice, nrhs, pair-stencil shape); the captures and their
# commands are in profiles/. An entry is removed when its kernel changes.
TRAFFIC = {
    ("k_lz_pair", "f64", (12, 12, 12, 12), 1, 7): 20003840,  # k_lz_pair_dyn<double>: 20.003 MB read + 0.5 KB written
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() in ("active", "0x1", "1"):
                        reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank scalar over all ranks (the timed region's length); identity at N=1."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(steps: int, solves_per_step: int, world: int, max_ms: float) -> float:
    """Whole-job solves/s: every rank's solves over the slowest rank's timed region."""
    return steps * solves_per_step * world / (max_ms / 1e3)


_SETUP_MEMO: dict = {}  # spectral set-up already computed in this process


def _setup(ovl, ctx, wl, rng_seed=0, cache=None):
    """Lattice, links, sources and per-mu deflation sets (untimed set-up). With `cache`, the
    spectral set-up is loaded from / saved to that .npz file (same workload inputs)."""
    import synth
    from paper_0910_1048_gb300 import spectrum

    dims = wl["dims"]
    u = synth.gauge_links(dims, rng_seed)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64 | ovl.OVL_F32 | ovl.OVL_F16R12)
    b = synth.gaussian_source(dims, 1000)
    stored = _SETUP_MEMO
    if cache and os.path.exists(cache):
        with np.load(cache) as z:
            stored.update({k: z[k] for k in z.files})
    per_mu = []
    changed = False
    for i, mu in enumerate(wl["mus"]):
        d = {"mu": mu}
        key = "%s_%d_%g_%d" % ("x".join(map(str, dims)), rng_seed, mu, wl["m"])
        if wl["m"] > 0:
            if key + "_lam" in stored:
                d.update(lam=stored[key + "_lam"], R=stored[key + "_R"], L=stored[key + "_L"],
                         gap=float(stored[key + "_gap"]), setup_s=0.0)
            else:
                t0 = time.time()
                # untimed set-up; its inverse solves in mixed precision (FP64 reliable updates to
                # the same 1e-12), about twice as fast as FP64 ones at 8^4
                lam, R, L, gap, info = spectrum.critical_eigenpairs(ovl, lat, M_W, mu, wl["m"],
                                                                    precision=ovl.OVL_PREC_F32)
                d.update(lam=lam, R=R, L=L, gap=gap, setup_s=time.time() - t0,
                         setup_inverse_solves=info["inverse_solves"])
                stored.update({key + "_lam": lam, key + "_R": R, key + "_L": L, key + "_gap": np.array(gap)})
                changed = True
        if wl["method"] in ("multishift", "fom") and wl["m"] == 0:
            if key + "_lo" in stored:
                d["gap"] = float(stored[key + "_lo"])
            else:
                d["gap"] = spectrum.smallest_modulus(ovl, lat, M_W, mu, precision=ovl.OVL_PREC_F32)
                stored[key + "_lo"] = np.array(d["gap"])
                changed = True
        if wl["method"] in ("multishift", "fom"):
            if key + "_hi" in stored:
                d["spec_hi"] = float(stored[key + "_hi"])
            else:
                d["spec_hi"] = 1.02 * spectrum.largest_modulus(ovl, lat, M_W, mu)
                stored[key + "_hi"] = np.array(d["spec_hi"])
                changed = True
        per_mu.append(d)
    if cache and changed:
        np.savez(cache, **stored)
    return lat, u, b, per_mu


def _params(ovl, wl, d):
    prec = {"f64": ovl.OVL_PREC_F64, "f32": ovl.OVL_PREC_F32, "f16": ovl.OVL_PREC_F32_F16LINKS}[wl["precision"]]
    kw = dict(m_W=M_W, mu=d["mu"], tol=wl["tol"], k_max=wl["k_max"], precision=prec,
              use_deflation=1 if wl["m"] > 0 else 0, check_every=25, two_pass=wl.get("two_pass", 0))
    if wl["method"] in ("multishift", "fom"):
        kw.update(method=ovl.OVL_MULTISHIFT_BICG if wl["method"] == "multishift" else ovl.OVL_FOM_RESTARTED,
                  spec_lo=0.98 * d["gap"], spec_hi=d["spec_hi"], check_every=20, restart_k=wl.get("restart_k", 40))
        if wl.get("rational") == "zolotarev":
            kw.update(rational_kind=ovl.OVL_RAT_ZOLOTAREV, s=wl["s"])
    return ovl.ovl_sign_params_default(**kw)


def _fp64_peak():
    """FP64 FMA throughput of this GPU (TFLOP/s), measured by the FMA-chain probe library built
    beside bench.py (libfp64_peak.so); falls back to the value that probe gave on a GB300."""
    import ctypes

    try:
        lib = ctypes.CDLL(os.path.join(ROOT, "libfp64_peak.so"))
        out = ctypes.c_double(0.0)
        if lib.ovl_probe_fma_tflops(1, ctypes.byref(out)) == 0 and out.value > 0:
            return out.value, "FP64 FMA-chain probe (fp64_peak.cu) run by bench.py on this GPU"
    except OSError:
        pass
    return FP64_PEAK_TFLOPS, "FP64 FMA-chain probe, earlier measurement on a GB300"


def _sources(wl):
    import synth

    nrhs = wl.get("nrhs", 1)
    return synth.gaussian_source(wl["dims"], 1000, nrhs=nrhs if nrhs > 1 else None)


def _time_workload(ovl, ctx, args, wl, u, per_mu, b, flush, world, steps=None, warmup=None):
    """Warm-up, then `steps` (default args.steps) timed steps of one workload. A step = one
    ovl_apply_sign per mu (each with all of the workload's right-hand sides), run concurrently from
    host threads."""
    import torch

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup

    lats = []
    for d in per_mu:
        lt = ovl.ovl_create_lattice(ctx, wl["dims"], -1)
        ovl.ovl_set_links(lt, u, ovl.OVL_F64 | ovl.OVL_F32 | ovl.OVL_F16R12)
        if wl["m"] > 0:
            ovl.ovl_set_deflation(lt, M_W, d["mu"], d["R"], d["L"], d["lam"])
        lats.append(lt)
    bdev = torch.from_numpy(b).cuda()
    xdevs = [torch.empty_like(bdev) for _ in per_mu]
    xhosts = [torch.empty(b.shape, dtype=torch.complex128).pin_memory().numpy() for _ in per_mu]
    # the step's solves are independent (one per mu, each with its own lattice workspace and
    # streams): they run concurrently from host threads, so their GPU work and their host-side
    # sign(H_k) e_1 evaluations overlap (the library releases the GIL inside every call)
    pool = ThreadPoolExecutor(max_workers=len(per_mu)) if args.concurrent and len(per_mu) > 1 else None

    prio = [0] * len(per_mu)

    def one(i, host, bh):
        p = _params(ovl, wl, per_mu[i])
        p.priority = prio[i]
        return ovl.ovl_apply_sign(lats[i], p, bh if host else bdev, xhosts[i] if host else xdevs[i])

    def step(host=False, bh=None):
        if pool is None:
            return [one(i, host, bh) for i in range(len(per_mu))]
        return list(pool.map(lambda i: one(i, host, bh), range(len(per_mu))))

    for w in range(warmup):
        res = step()
        if w == 0 and pool is not None and warmup >= 2:
            # concurrent solves: the one needing the most iterations gets the most urgent streams,
            # so it runs near its alone speed while the others fill the idle SMs (ranked on the
            # first warm-up step; the remaining warm-up steps run with the final priorities)
            its = [max(inf["iterations"] for inf in r[1]) for r in res]
            for rank, i in enumerate(sorted(range(len(its)), key=lambda i: its[i])):
                prio[i] = rank
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    times, infos = [], []
    stream = torch.cuda.current_stream()
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        infos.append(res)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(times), world, "cuda")
    # end to end through the same call with pinned host buffers
    bh = torch.from_numpy(b).pin_memory().numpy()
    step(True, bh)
    t0 = time.perf_counter()
    for _ in range(steps):
        step(True, bh)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    # accuracy actually reached: the paper's measure 0.5 |sign(A)^2 b - b| / |b| (Section 6),
    # worst right-hand side
    acc = []
    for i, (lt, d) in enumerate(zip(lats, per_mu)):
        p = _params(ovl, wl, d)
        p.priority = prio[i]
        x1 = torch.empty_like(bdev)
        x2 = torch.empty_like(bdev)
        ovl.ovl_apply_sign(lt, p, bdev, x1)
        ovl.ovl_apply_sign(lt, p, x1, x2)
        nb = bdev.shape[0] if wl.get("nrhs", 1) > 1 else 1
        e = (x2 - bdev).reshape(nb, -1)
        acc.append(float(torch.max(0.5 * torch.linalg.vector_norm(e, dim=1)
                                   / torch.linalg.vector_norm(bdev.reshape(nb, -1), dim=1))))
    for lt in lats:
        ovl.ovl_destroy_lattice(lt)
    if pool is not None:
        pool.shutdown()
    return total_ms, e2e_s, infos, acc


def _dslash_gbs(ovl, ctx, u_fn, L=32, reps=20):
    """Kernel-only bandwidth of the FP32 and FP16-12-real stencil H_W(mu) psi on an L^4 lattice
    (native layout, CUDA events around `reps` back-to-back launches; inputs > L2)."""
    import torch

    dims = (L, L, L, L)
    vol = L ** 4
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u_fn(dims), ovl.OVL_F32 | ovl.OVL_F16R12)
    x = torch.randn(12 * vol, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    out = {}
    stream = torch.cuda.current_stream()
    for name, fl, per_site in (("f32", ovl.OVL_LINKS_F32, 480), ("f16_links", ovl.OVL_LINKS_F16R12, 288)):
        flags = fl | ovl.OVL_NATIVE | ovl.OVL_GAMMA5
        for _ in range(3):
            ovl.ovl_apply_DW(lat, M_W, 0.3, flags, x, y)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ovl.ovl_apply_DW(lat, M_W, 0.3, flags, x, y)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps
        out[name] = {"lattice": "%d^4" % L, "us_per_launch": t * 1e3, "algorithmic_bytes_per_site": per_site,
                     "achieved_gbs": per_site * vol / (t * 1e-3) / 1e9}
    ovl.ovl_destroy_lattice(lat)
    out.update(_dslash_batch_gbs(ovl, ctx, u_fn, reps=max(3, reps // 4)))
    return out


def _dslash_batch_gbs(ovl, ctx, u_fn, L=24, nrhs=16, reps=5):
    """FP32 stencil on a batch of `nrhs` sources on an L^4 lattice (native layout): one launch over
    the batch (links loaded once per site for each group of sources) against `nrhs` single-source
    launches. Algorithmic bytes per launch: the links once (288 B per site) plus 192 B per site and
    source (spinor in and out)."""
    import torch

    dims = (L, L, L, L)
    vol = L ** 4
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u_fn(dims), ovl.OVL_F32)
    x = torch.randn(nrhs * 12 * vol, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    flags = ovl.OVL_LINKS_F32 | ovl.OVL_NATIVE | ovl.OVL_GAMMA5
    byts = vol * (288 + nrhs * 192)
    stream = torch.cuda.current_stream()
    res = {}
    for name, run in (("f32_batch%d" % nrhs, lambda: ovl.ovl_apply_DW(lat, M_W, 0.3, flags, x, y)),
                      ("f32_batch%d_one_by_one" % nrhs,
                       lambda: [ovl.ovl_apply_DW(lat, M_W, 0.3, flags, x[r * 12 * vol:(r + 1) * 12 * vol],
                                                 y[r * 12 * vol:(r + 1) * 12 * vol]) for r in range(nrhs)])):
        for _ in range(2):
            run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps
        res[name] = {"lattice": "%d^4" % L, "nrhs": nrhs, "us_per_batch": t * 1e3,
                     "algorithmic_bytes_per_batch": byts, "achieved_gbs": byts / (t * 1e-3) / 1e9}
    ovl.ovl_destroy_lattice(lat)
    return res


def _prec_code(ovl, prec):
    return {"f64": ovl.OVL_PREC_F64, "f32": ovl.OVL_PREC_F32, "f16": ovl.OVL_PREC_F32_F16LINKS}[prec]


def _roofline(wl, infos, fp64_peak, fp64_src):
    peaks, src = _peaks()
    vol = int(np.prod(wl["dims"]))
    kt = [i["t_kernel_ms"] for step in infos for _, inf in step for i in inf[:1] if i["kernel_samples"] > 0]
    t_pair = float(np.mean(kt)) if kt else None
    prec = wl["precision"]
    kernel = {"direct": "k_lz_pair", "multishift": "k_ms_pair", "fom": "k_dslash (two per Arnoldi step)"}[wl["method"]]
    nr = wl.get("nrhs", 1)
    import paper_0910_1048_gb300 as ovl
    shape = ovl.ovl_get_pair_variant(vol, _prec_code(ovl, prec))  # the autotuner's pick (ovl_set_pair_variant)
    traffic = TRAFFIC.get((kernel, prec, tuple(wl["dims"]), nr, shape))
    if prec == "f64":
        flops = PAIR_FLOPS_PER_SITE * vol * nr
        ach = flops / (t_pair * 1e-3) / 1e12 if t_pair else None
        return {"kernel": kernel, "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s (FP64)",
                "frac": (ach / fp64_peak) if ach else None, "traffic": traffic, "peak_source": fp64_src,
                "algorithmic_flops_per_launch": flops,
                "algorithmic_bytes_per_launch": pair_bytes("f64", vol, nr), "pair_variant": shape,
                "note": "FP64 kernels are bound by GB300's FP64 pipe (ncu at 12^4: FP64 pipe 84% of active "
                        "cycles in the pair stencil, 66-72% in the update)"}
    byts = pair_bytes(prec, vol, nr)
    ach = byts / (t_pair * 1e-3) / 1e9 if t_pair else None
    return {"kernel": kernel, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"] if ach else None, "traffic": traffic,
            "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)", "algorithmic_bytes_per_launch": byts,
            "pair_variant": shape}


def _summary(wl, per_mu, infos, acc):
    flat = [i for step in infos for _, inf in step for i in inf]
    its = [i["iterations"] for i in flat]
    per_mu_stats = []
    for j, d in enumerate(per_mu):
        sel = [i for step in infos for i in step[j][1]]
        per_mu_stats.append({"mu": d["mu"], "k": float(np.mean([i["iterations"] for i in sel])),
                             "t_solve_ms": float(np.mean([i["t_total_ms"] for i in sel])),
                             "t_small_ms": float(np.mean([i["t_small_ms"] for i in sel])),
                             "t_pair_ms": float(np.mean([i["t_kernel_ms"] for i in sel])),
                             "t_update_ms": float(np.mean([i["t_update_ms"] for i in sel])),
                             "t_finish_ms": float(np.mean([i["t_finish_ms"] for i in sel])),
                             "evaluations": float(np.mean([i["evaluations"] for i in sel])),
                             "ritz_evaluations": float(np.mean([i["ritz_evaluations"] for i in sel])),
                             "gap": d.get("gap"), "accuracy_half_sign2b_minus_b": acc[j]})
    statuses = sorted({st for step in infos for st, _ in step})
    launches = sum(inf[0]["kernel_launches"] for step in infos for _, inf in step)
    return its, per_mu_stats, statuses, launches


def _companion(ovl, ctx, args, cname, flush, world, local, fp64_peak, fp64_src, ref_value):
    """One companion workload, timed like the headline with at most 3 warm-up and 3 timed steps."""
    wm = WORKLOADS[cname]
    lat_m, u_m, _, pm = _setup(ovl, ctx, wm, cache=args.setup_cache)
    ovl.ovl_destroy_lattice(lat_m)
    bm = _sources(wm)
    sps = len(pm) * wm.get("nrhs", 1)
    steps, warm = min(args.steps, 3), min(args.warmup, 3)
    with ClockSampler(local) as clk:
        tm, em, im, am = _time_workload(ovl, ctx, args, wm, u_m, pm, bm, flush, world, steps=steps, warmup=warm)
    vm = throughput(steps, sps, world, tm)
    _, pms, stm, lm = _summary(wm, pm, im, am)
    return {"workload": cname, "lattice": "x".join(map(str, wm["dims"])), "method": wm["method"],
            "precision": wm["precision"], "rational": wm.get("rational", "neuberger"), "poles": wm.get("s"),
            "tol": wm["tol"], "nrhs": wm.get("nrhs", 1), "value": vm, "unit": UNIT, "steps": steps, "warmup": warm,
            "ms_per_step": tm / steps, "speedup_vs_line_value": vm / ref_value,
            "e2e_value": steps * sps * world / em, "statuses": stm, "accuracy_half_sign2b_minus_b": am,
            "per_mu": pms, "gpu_launches": int(lm), "roofline": _roofline(wm, im, fp64_peak, fp64_src),
            "clocks": clk.summary()}


def _c2_line(ovl, ctx, args):
    """8^4, mu in {0, 0.1, 0.3}, 16 deflated critical eigenpairs per mu, FP64 direct: the error
    reached at k = 600 (the paper's measure 0.5 |sign(A)^2 b - b| / |b|, both solves at k = 600) and
    the k that reaches 1e-10 (with the same measure for that solve)."""
    import torch

    wl = WORKLOADS[C2["workload"]]
    lat, u, b, per_mu = _setup(ovl, ctx, wl, cache=args.setup_cache)
    bt = torch.from_numpy(b).cuda()
    out = []
    for d in per_mu:
        ovl.ovl_set_deflation(lat, M_W, d["mu"], d["R"], d["L"], d["lam"])
        row = {"mu": d["mu"], "deflated": wl["m"], "gap": d["gap"]}
        for tag, kw in (("fixed_k600", dict(fixed_k=C2["k_fixed"])),
                        ("tol1e-10", dict(tol=C2["tol"], k_max=C2["k_max"]))):
            p = ovl.ovl_sign_params_default(mu=d["mu"], use_deflation=1, check_every=25, **kw)
            x1, x2 = torch.empty_like(bt), torch.empty_like(bt)
            t0 = time.perf_counter()
            st1, i1 = ovl.ovl_apply_sign(lat, p, bt, x1)
            t1 = time.perf_counter()
            ovl.ovl_apply_sign(lat, p, x1, x2)
            err = float(0.5 * torch.linalg.vector_norm(x2 - bt) / torch.linalg.vector_norm(bt))
            row[tag] = {"k": i1[0]["iterations"], "status": st1, "accuracy_half_sign2b_minus_b": err,
                        "t_solve_ms": 1e3 * (t1 - t0)}
        out.append(row)
    ovl.ovl_destroy_lattice(lat)
    return {"workload": C2["workload"], "method": "direct", "precision": "f64", "per_mu": out,
            "note": "attained error at fixed k = 600 and the k reaching 1e-10 (16 deflated eigenpairs)"}


def run_ours(args, wl):
    import torch

    import paper_0910_1048_gb300 as ovl
    import synth

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ctx = ovl.ovl_ctx_create(local)
    lat, u, _, per_mu = _setup(ovl, ctx, wl, cache=args.setup_cache)
    if args.pair_variant >= 0:  # a pinned pair-stencil shape instead of the autotuner's pick
        ovl.ovl_set_pair_variant(int(np.prod(wl["dims"])), _prec_code(ovl, wl["precision"]), args.pair_variant)
    b = _sources(wl)
    nrhs = wl.get("nrhs", 1)
    n = b.size // nrhs
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    fp64_peak, fp64_src = _fp64_peak()

    with ClockSampler(local) as clk:
        total_ms, e2e_s, infos, acc = _time_workload(ovl, ctx, args, wl, u, per_mu, b, flush, world)
    clocks = clk.summary()
    solves_per_step = len(per_mu) * nrhs
    solves = args.steps * solves_per_step * world
    value = throughput(args.steps, solves_per_step, world, total_ms)
    e2e = {"value": solves / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(len(per_mu) * b.size * 16),
           "d2h_bytes_per_step": int(len(per_mu) * b.size * 16)}
    its, per_mu_stats, statuses, launches = _summary(wl, per_mu, infos, acc)
    prec = wl["precision"]
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "f64" else "f32",
        "data": "synthetic: SU(3) links exp(0.5 i H) seed 0, Gaussian b seed 1000",
        "config": {"workload": args.workload, "lattice": "x".join(map(str, wl["dims"])), "n": int(n),
                   "mu": list(wl["mus"]), "m_W": M_W, "deflated": wl["m"], "method": wl["method"],
                   "precision": prec, "tol": wl["tol"], "k_max": wl["k_max"], "nrhs": nrhs,
                   "solves_per_step": solves_per_step, "concurrent_solves": bool(args.concurrent),
                   "stream_priority": "longest solve most urgent" if args.concurrent and len(per_mu) > 1 else "default",
                   "l2": "flushed between steps (256 MB write)",
                   "iterations_mean": float(np.mean(its)), "statuses": statuses,
                   "accuracy_half_sign2b_minus_b": acc, "per_mu": per_mu_stats,
                   "untimed_setup_s": [round(d.get("setup_s", 0.0), 2) for d in per_mu],
                   "setup_inverse_solves": [d.get("setup_inverse_solves", 0) for d in per_mu],
                   "parallelism": "replicas" if world > 1 else "single",
                   "pair_variant_pinned": args.pair_variant if args.pair_variant >= 0 else None},
        "roofline": _roofline(wl, infos, fp64_peak, fp64_src), "e2e": e2e, "clocks": clocks,
        "gpu_launches": int(launches),
    }
    # companion lines: the same problem in mixed precision (speedup over this line's value), the
    # 16-source batch; each timed with at most 3 warm-up and 3 timed steps
    if not args.no_extras:
        for key, cname in COMPANIONS.get(args.workload, []):
            res[key] = _companion(ovl, ctx, args, cname, flush, world, local, fp64_peak, fp64_src, value)
        if args.workload == DEFAULT_WORKLOAD:
            res["lattice8_defl16"] = _c2_line(ovl, ctx, args)
    k_table = K_TABLE.get(args.workload)
    if k_table:
        res["config"]["k_table"] = {"%g" % m: {"gpu": s_["k"], "table": k_table.get(m)} for m, s_ in
                                    zip(wl["mus"], per_mu_stats)}
    if not args.no_extras:
        res["dslash"] = _dslash_gbs(ovl, ctx, lambda d: synth.gauge_links(d, 0))
        if args.serving_requests > 0:
            res["serving"] = serving_sample(ovl, ctx, args.serving_requests)
        pk, _ = _peaks()
        for v in res["dslash"].values():
            v["frac_of_measured_hbm"] = v["achieved_gbs"] / pk["hbm_gbs"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(wl, args.workload, its, seconds=args.cpu_seconds)
    ovl.ovl_destroy_lattice(lat)
    ovl.ovl_ctx_destroy(ctx)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


SERVING = dict(sizes=(4, 8, 12, 16), fields_per_size=5, tols=(1e-6, 1e-8, 1e-10), nrhs_max=8, seed=42,
               k_max_by_tol={1e-6: 1500, 1e-8: 3000, 1e-10: 5000}, k_max_cap={4: 5000, 8: 5000, 12: 5000, 16: 5000},
               two_pass_over_bytes=25 << 30,
               mean_interarrival_s=0.25)


def _serving_stream(n_requests):
    """The first n requests of the serving stream (seed 42): field index uniform over 20 resident
    fields (5 per lattice size 4^4, 8^4, 12^4, 16^4), mu ~ U[0, 1], tol in {1e-6, 1e-8, 1e-10}, 1-8
    Gaussian sources (seed 2000 + request), exponential inter-arrival gaps of unit mean (scaled by
    the run's rate)."""
    cfg = SERVING
    rng = np.random.default_rng(cfg["seed"])
    nf = len(cfg["sizes"]) * cfg["fields_per_size"]
    reqs = []
    for i in range(n_requests):
        fi = int(rng.integers(0, nf))
        L = cfg["sizes"][fi // cfg["fields_per_size"]]
        nrhs = int(rng.integers(1, cfg["nrhs_max"] + 1))
        reqs.append(dict(i=i, fi=fi, L=L, nrhs=nrhs, mu=float(rng.uniform(0.0, 1.0)),
                         tol=float(rng.choice(cfg["tols"])), gap=float(rng.exponential(1.0))))
    return reqs


def _serving_run(ovl, srv, ids, reqs, mean_gap_s):
    """Submit `reqs` with gaps gap * mean_gap_s (0: all at once) and poll until every one is done.
    Returns (done list of (request, latency_s, status, info), wall seconds)."""
    import synth

    cfg = SERVING
    for r in reqs:  # sources made before the clock starts
        r["b"] = synth.gaussian_source((r["L"],) * 4, 2000 + r["i"], nrhs=r["nrhs"])
    pending, done = {}, []
    t_start = time.perf_counter()
    t_next = t_start
    i = 0
    while i < len(reqs) or pending:
        now = time.perf_counter()
        while i < len(reqs) and now >= t_next:
            r = reqs[i]
            k_max = min(cfg["k_max_by_tol"][r["tol"]], cfg["k_max_cap"][r["L"]])
            # the two-pass strategy (O(n) memory) where the basis of one request would take more than
            # an eighth of the budget (8 slots)
            basis = r["nrhs"] * (k_max + 1) * 12 * r["L"] ** 4 * 16
            tk = ovl.ovl_submit(srv, ids[r["fi"]], r["b"], r["mu"], r["tol"], k_max=k_max,
                                two_pass=int(basis > cfg["two_pass_over_bytes"]))
            pending[tk] = (r, now)
            i += 1
            if i < len(reqs):
                t_next += reqs[i]["gap"] * mean_gap_s
        for tk in list(pending):
            r, t0 = pending[tk]
            st, info = ovl.ovl_poll(srv, tk, r["nrhs"], None)
            if st != ovl.OVL_PENDING:
                done.append((r, time.perf_counter() - t0, st, info))
                del pending[tk]
        time.sleep(0.001)
    wall = time.perf_counter() - t_start
    for r in reqs:
        r.pop("b", None)
    return done, wall


def _serving_stats(ovl, done, wall):
    lat_ms = sorted(1e3 * d for _, d, _, _ in done)
    ok = sum(1 for r, _, _, info in done for inf in info[:r["nrhs"]] if inf["status"] == ovl.OVL_OK)
    sources = sum(r["nrhs"] for r, _, _, _ in done)
    per_size = {}
    for r, d, _, _ in done:
        per_size.setdefault("%d^4" % r["L"], []).append(1e3 * d)
    statuses = {}
    for r, _, _, info in done:
        for inf in info[:r["nrhs"]]:
            nm = ovl.STATUS_NAMES.get(inf["status"], str(inf["status"]))
            statuses[nm] = statuses.get(nm, 0) + 1
    return {"requests": len(done), "sources": sources, "wall_s": wall, "solves_per_s": sources / wall,
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "success_rate": ok / max(1, sources), "statuses": statuses,
            "p50_ms_by_size": {k: float(np.percentile(v, 50)) for k, v in sorted(per_size.items())}}


def _serving_server(ovl, ctx, mem_budget, max_slots):
    import synth

    cfg = SERVING
    lats, ids = [], []
    srv = ovl.ovl_server_create(ctx, mem_budget, max_slots=max_slots)
    for si, L in enumerate(cfg["sizes"]):
        for f in range(cfg["fields_per_size"]):
            dims = (L, L, L, L)
            lat = ovl.ovl_create_lattice(ctx, dims, -1)
            ovl.ovl_set_links(lat, synth.gauge_links(dims, si * cfg["fields_per_size"] + f), ovl.OVL_F64)
            lats.append(lat)
            ids.append(ovl.ovl_server_add_field(srv, lat))
    return srv, lats, ids


def serving_sample(ovl, ctx, n_requests, mem_budget=200 << 30, max_slots=8):
    """A bounded sample of the serving stream: the first n requests, Poisson arrivals with a mean gap
    of SERVING['mean_interarrival_s'], FP64 direct method, admitted by device-memory footprint
    (ovl_submit / ovl_poll). Latency = completion - arrival."""
    cfg = SERVING
    srv, lats, ids = _serving_server(ovl, ctx, mem_budget, max_slots)
    done, wall = _serving_run(ovl, srv, ids, _serving_stream(n_requests), cfg["mean_interarrival_s"])
    ovl.ovl_server_destroy(srv)
    for lat in lats:
        ovl.ovl_destroy_lattice(lat)
    res = _serving_stats(ovl, done, wall)
    res.update({"precision": "f64", "method": "direct",
                "sample": "%d requests of the 2000-request stream (Poisson, mean gap %g s)"
                          % (n_requests, cfg["mean_interarrival_s"]), "mem_budget_bytes": mem_budget,
                "max_slots": max_slots, "k_max_by_tol": {"%g" % k: v for k, v in cfg["k_max_by_tol"].items()},
                "k_max_cap": {"%d^4" % k: v for k, v in cfg["k_max_cap"].items()},
                "two_pass_when_basis_over_bytes": cfg["two_pass_over_bytes"]})
    return res


def run_serving(args):
    """The serving configuration as its own line: the first `--serving-requests` requests of the
    2000-request stream (seed 42) all submitted at once (the saturation throughput S, sources/s),
    then the same requests with Poisson arrivals at 0.5 S and 0.9 S (mean gap = mean sources per
    request / rate). value = solves/s of the 0.9 S run; p50 / p99 latency of each run."""
    import torch

    import paper_0910_1048_gb300 as ovl

    rank, world, local = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    ctx = ovl.ovl_ctx_create(local)
    n = args.serving_requests if args.serving_requests > 0 else 200
    reqs = _serving_stream(n)
    mean_src = float(np.mean([r["nrhs"] for r in reqs]))
    srv, lats, ids = _serving_server(ovl, ctx, 200 << 30, 8)
    with ClockSampler(local) as clk:
        done, wall = _serving_run(ovl, srv, ids, reqs, 0.0)
        sat = _serving_stats(ovl, done, wall)
        runs = {}
        for frac in (0.5, 0.9):
            rate = frac * sat["solves_per_s"]  # sources per second
            d2, w2 = _serving_run(ovl, srv, ids, reqs, mean_src / rate)
            runs["%.1fx" % frac] = dict(_serving_stats(ovl, d2, w2), offered_sources_per_s=rate)
    ovl.ovl_server_destroy(srv)
    for lat in lats:
        ovl.ovl_destroy_lattice(lat)
    ovl.ovl_ctx_destroy(ctx)
    main_run = runs["0.9x"]
    res = {
        "metric": "sgn(H_W)b serving solves/s; p50/p99 latency", "value": main_run["solves_per_s"],
        "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * main_run["wall_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: 20 fields (seeds 0-19), Gaussian sources seed 2000+request",
        "config": {"workload": "serving", "requests": n, "of_stream": 2000, "seed": SERVING["seed"],
                   "sizes": ["%d^4" % L for L in SERVING["sizes"]], "mu": "U[0,1]", "tols": list(SERVING["tols"]),
                   "nrhs": "1-%d" % SERVING["nrhs_max"], "mem_budget_bytes": 200 << 30, "max_slots": 8,
                   "method": "direct", "precision": "f64", "parallelism": "single"},
        "saturation": sat, "runs": runs, "p50_ms": main_run["p50_ms"], "p99_ms": main_run["p99_ms"],
        "clocks": clk.summary(),
        "e2e": {"value": main_run["solves_per_s"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(res))


def _oracle_inputs(wl, mu):
    """Links, the first source and (with deflation) the critical eigenpairs for the oracle legs."""
    import synth
    from oracle import deflation

    dims = wl["dims"]
    u = synth.gauge_links(dims, 0)
    b = synth.gaussian_source(dims, 1000, nrhs=wl.get("nrhs", 1) if wl.get("nrhs", 1) > 1 else None)
    b0 = b[0] if wl.get("nrhs", 1) > 1 else b
    R = L = lam = None
    if wl["m"] > 0:
        lam, R, L, _ = deflation.critical_sparse(u, dims, M_W, mu, wl["m"])
    return u, b0, R, L, lam


def _oracle_solve(wl, mu, k, seconds):
    """Time one oracle solve (the C FP64 two-sided Lanczos of Algorithm 4, exactly k steps, then
    numpy's eigendecomposition for sign(H_k) e_1 and the combine) at mu on the workload's first
    source. The whole solve runs when its estimate (from the first 10 steps) fits `seconds`;
    otherwise as many steps as fit are timed and the steps and the k^3 eigendecomposition are
    extrapolated to k. Returns (seconds per solve, description)."""
    from oracle import krylov, lanczos

    u, b0, R, L, lam = _oracle_inputs(wl, mu)
    dims = wl["dims"]
    s = krylov.DirectSolve(u, dims, M_W, mu, b0, k, R=R, L=L, lam=lam)
    t0 = time.perf_counter()
    s.start()
    s.steps(10)
    per_step = (time.perf_counter() - t0) / 10
    lat = "x".join(map(str, dims))
    if per_step * k * 1.2 <= seconds:
        s.steps(k - s.k)
        s.finish()
        total = time.perf_counter() - t0
        return total, ("one full oracle solve at %s mu=%g: C two-sided Lanczos, k=%d steps (%s), numpy eig "
                       "sign(H_k) e_1, combine" % (lat, mu, s.k, "deflated %d" % wl["m"] if wl["m"] else "no deflation"))
    budget = max(10, int(0.7 * seconds / per_step))
    s.steps(budget - s.k)
    t_steps = time.perf_counter() - t0
    kk = s.k
    t1 = time.perf_counter()
    lanczos.sign_tridiag_e1(s.alpha[:kk], s.beta[:kk - 1], s.delta[:kk - 1])
    t_eig = (time.perf_counter() - t1) * (k / kk) ** 3
    total = t_steps / kk * k + t_eig
    return total, ("oracle at %s mu=%g: %d of k=%d C two-sided Lanczos steps timed (%.1f s), extrapolated, "
                   "plus numpy eig of H_k scaled as k^3" % (lat, mu, kk, k, t_steps))


def _oracle_step_scaling(wl, mu, seconds=4.0, max_steps=40):
    """Milliseconds per Lanczos step of the C oracle (two stencil applications and the biorthogonal
    update of Algorithm 4) on one core and on all of this host's cores, each timed over up to
    `max_steps` steps within about seconds / 2, after two untimed steps."""
    from oracle import krylov

    u, b0, R, L, lam = _oracle_inputs(wl, mu)
    all_cores = krylov.threads()
    out = {}
    try:
        for nt in sorted({1, all_cores}):
            krylov.threads(nt)
            s = krylov.DirectSolve(u, wl["dims"], M_W, mu, b0, max_steps + 2, R=R, L=L, lam=lam).start()
            s.steps(2)
            k0 = s.k
            t0 = time.perf_counter()
            while s.k < k0 + max_steps and (s.k - k0 < 3 or time.perf_counter() - t0 < seconds / 2):
                before = s.k
                if s.steps(1) == before:  # breakdown, or nothing to start from
                    break
            done = s.k - k0
            if done > 0:
                out[str(nt)] = 1e3 * (time.perf_counter() - t0) / done
    finally:
        krylov.threads(all_cores)
    return out


def cpu_baseline(wl, workload, iterations, seconds=20.0):
    """The oracle on this host's cores, one solve of the workload's hardest mu at the k the GPU
    needed (bounded: see _oracle_solve), and its per-step time on one core and on all cores."""
    from oracle import krylov

    mu = wl["mus"][-1]
    k = int(round(float(np.mean(iterations)))) if len(iterations) else K_TABLE.get(workload, {}).get(mu, wl["k_max"])
    t, desc = _oracle_solve(wl, mu, k, seconds)
    res = {"value": 1.0 / t, "unit": UNIT, "cores": krylov.threads(), "kind": "oracle", "sample": desc}
    try:
        res["step_ms_by_cores"] = _oracle_step_scaling(wl, mu)
    except Exception as e:  # a side figure: it never costs the line
        res["step_ms_by_cores"] = {"error": "%s: %s" % (type(e).__name__, e)}
    return res


def run_reference(args, wl):
    """The oracle (plain C FP64 two-sided Lanczos, Algorithm 4, with numpy's eigendecomposition of
    H_k) on this host's cores, for the workload's mu set, deflation and the per-mu k of K_TABLE (the
    GPU's). The K timed steps are pieces of one full solve per mu: each advances every solve by
    k/K Lanczos steps, the last one also evaluates sign(H_k) e_1 and combines. A multi-source
    workload times its first source and counts it as nrhs solves (the sources are independent)."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    from oracle import krylov

    ktab = K_TABLE.get(args.workload, {})
    nrhs = wl.get("nrhs", 1)
    solves = []
    for mu in wl["mus"]:
        u, b0, R, L, lam = _oracle_inputs(wl, mu)
        solves.append(krylov.DirectSolve(u, wl["dims"], M_W, mu, b0, int(ktab.get(mu, wl["k_max"])), R=R, L=L,
                                         lam=lam))
    warm = krylov.DirectSolve(u, wl["dims"], M_W, wl["mus"][0], b0, args.warmup + 1).start()
    for _ in range(args.warmup):
        warm.steps(1)
    del warm
    K = max(1, args.steps)
    times = []
    for i in range(K):
        t0 = time.perf_counter()
        for sv in solves:
            if i == 0:
                sv.start()
            sv.steps(-(-sv.kcap // K))
            if i == K - 1:
                sv.steps(sv.kcap - sv.k)
                sv.finish()
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = len(solves) * nrhs / total
    ks = {"%g" % sv.mu: sv.k for sv in solves}
    desc = ("one full oracle solve per mu at %s (k per mu %s from the GPU's runs%s), split over the %d timed "
            "steps" % ("x".join(map(str, wl["dims"])), ks, ", 16 deflated" if wl["m"] else "", K))
    if nrhs > 1:
        desc += "; first of %d sources timed, counted %d times" % (nrhs, nrhs)
    cores = krylov.threads()
    res = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic: SU(3) links exp(0.5 i H) seed 0, Gaussian b seed 1000",
        "config": {"workload": args.workload, "lattice": "x".join(map(str, wl["dims"])), "mu": list(wl["mus"]),
                   "deflated": wl["m"], "method": "direct", "precision": "f64", "tol": wl["tol"], "k_per_mu": ks},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(res))


def run_profile_case(args):
    """A small, fixed amount of work for an Nsight Compute capture (a few hundred MB on the device,
    a bounded number of launches): one fixed-k direct solve (`direct`), one fixed-iteration
    multishift solve (`multishift`) or three stencil launches per link format (`dslash`) on an L^4
    lattice with the seed-0 links. Prints nothing to compare; the capture is the product."""
    import torch

    import paper_0910_1048_gb300 as ovl
    import synth

    L = args.lattice
    dims = (L, L, L, L)
    ctx = ovl.ovl_ctx_create(0)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, synth.gauge_links(dims, 0), ovl.OVL_F64 | ovl.OVL_F32 | ovl.OVL_F16R12)
    prec = {"f64": ovl.OVL_PREC_F64, "f32": ovl.OVL_PREC_F32, "f16": ovl.OVL_PREC_F32_F16LINKS}[args.prec]
    if args.pair_variant >= 0:  # a pinned pair-stencil shape: no autotuner launches before the capture
        ovl.ovl_set_pair_variant(L ** 4, prec, args.pair_variant)
    if args.profile_case == "dslash":
        dt = torch.complex128 if args.prec == "f64" else torch.complex64
        x = torch.randn(args.nrhs * 12 * L ** 4, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        fl = {"f64": 0, "f32": ovl.OVL_LINKS_F32, "f16": ovl.OVL_LINKS_F16R12}[args.prec]
        for _ in range(3):
            ovl.ovl_apply_DW(lat, M_W, 0.3, fl | ovl.OVL_NATIVE | ovl.OVL_GAMMA5, x, y)
    else:
        b = torch.from_numpy(synth.gaussian_source(dims, 1000, nrhs=args.nrhs if args.nrhs > 1 else None)).cuda()
        x = torch.empty_like(b)
        if args.profile_case == "direct":
            p = ovl.ovl_sign_params_default(mu=0.3, precision=prec, fixed_k=args.fixed_k, check_every=20)
        else:
            p = ovl.ovl_sign_params_default(mu=0.3, precision=prec, method=ovl.OVL_MULTISHIFT_BICG,
                                            rational_kind=ovl.OVL_RAT_ZOLOTAREV, s=20, spec_lo=0.05, spec_hi=2.7,
                                            tol=1e-3, k_max=args.fixed_k)
        ovl.ovl_apply_sign(lat, p, b, x)
    torch.cuda.synchronize()
    ovl.ovl_destroy_lattice(lat)
    ovl.ovl_ctx_destroy(ctx)


def summarize_launches(path, skip_before=None):
    """Per-kernel totals of an Nsight Compute launch list (`ncu --metrics gpu__time_duration.sum --csv
    --log-file PATH ...`): launches, total time, share and mean per kernel, largest share first.
    With `skip_before`, launches before the first one whose kernel name contains it are left out
    (the set-up and autotuner launches ahead of the solves)."""
    import csv
    rows = []
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    rd = csv.reader(lines)
    hdr = next(rd)
    ik, iu, iv = hdr.index("Kernel Name"), hdr.index("Metric Unit"), hdr.index("Metric Value")
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}
    for r in rd:
        name = r[ik].split("(")[0].replace("void ", "")
        rows.append((name, float(r[iv].replace(",", "")) * scale[r[iu]]))
    if skip_before:
        first = next((i for i, (nm, _) in enumerate(rows) if skip_before in nm), 0)
        rows = rows[first:]
    tot = sum(t for _, t in rows)
    agg = {}
    for nm, t in rows:
        a = agg.setdefault(nm, [0, 0.0])
        a[0] += 1
        a[1] += t
    print("launches=%d total_us=%.1f" % (len(rows), tot))
    print("%-48s %8s %12s %7s %9s" % ("kernel", "launches", "total_us", "share", "mean_us"))
    for nm, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print("%-48s %8d %12.1f %6.1f%% %9.2f" % (nm[:48], c, t, 100.0 * t / tot, t / c))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serving"], default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=16,
                    help="requests in the serving sample added to the line (0: none)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mixed-precision companion line and the stencil bandwidth figure")
    ap.add_argument("--concurrent", type=int, default=1,
                    help="run the step's independent solves concurrently (1) or one after another (0)")
    ap.add_argument("--setup-cache", default=None,
                    help=".npz file holding the untimed spectral set-up (created if missing)")
    ap.add_argument("--profile-case", choices=["direct", "multishift", "dslash"], default=None,
                    help="run one small fixed case for a profiler capture instead of the benchmark")
    ap.add_argument("--lattice", type=int, default=8, help="--profile-case: extent L of the L^4 lattice")
    ap.add_argument("--prec", choices=["f64", "f32", "f16"], default="f64", help="--profile-case: precision")
    ap.add_argument("--nrhs", type=int, default=1, help="--profile-case: right-hand sides")
    ap.add_argument("--fixed-k", type=int, default=40, help="--profile-case: Lanczos steps / BiCG iterations")
    ap.add_argument("--pair-variant", type=int, default=-1,
                    help="pin the pair-stencil shape of the workload (or of --profile-case) with ovl_set_pair_variant; "
                         "-1 autotunes")
    ap.add_argument("--summarize-launches", metavar="CSV", default=None,
                    help="print per-kernel totals of an ncu launch list (gpu__time_duration.sum) and exit")
    ap.add_argument("--from-kernel", default=None,
                    help="--summarize-launches: start at the first launch of this kernel")
    args = ap.parse_args()
    if args.summarize_launches:
        summarize_launches(args.summarize_launches, args.from_kernel)
        return
    if args.profile_case:
        run_profile_case(args)
        return
    if args.workload == "serving":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the serving stream has no oracle counterpart "
                              "(the oracle is timed per solve by the other workloads)"}))
        else:
            run_serving(args)
        return
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
