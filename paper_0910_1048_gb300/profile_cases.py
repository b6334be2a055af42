"""Small, self-contained cases for Nsight Compute captures, and a launch-list summariser.

  python -m paper_0910_1048_gb300.profile_cases dslash --L 28      FP32 / FP16-link stencil, 3 launches each
  python -m paper_0910_1048_gb300.profile_cases pair --L 8         fixed-k FP64 direct solve (pair stencil)
  python -m paper_0910_1048_gb300.profile_cases pair --L 16 --prec f32 --nrhs 16   the batched FP32 step
  python -m paper_0910_1048_gb300.profile_cases multishift --L 8   fixed-iteration FP64 multishift solve
  python -m paper_0910_1048_gb300.profile_cases multishift --L 8 --prec f16   1e-8 FP16-link solve with
                                                                    FP64 reliable updates
  python -m paper_0910_1048_gb300.profile_cases summarize launches.csv out.txt

The cases hold at most a few GB on the device and a handful of launches, so that a capture with
many passes ends by itself; `summarize` turns an `ncu --csv` list of gpu__time_duration.sum
values into launches / total time / share per kernel.
"""
from __future__ import annotations

import argparse
import collections
import csv
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def case_dslash(L: int):
    import torch

    import paper_0910_1048_gb300 as ovl
    import synth

    ctx = ovl.ovl_ctx_create(0)
    dims = (L, L, L, L)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, synth.unit_links(dims), ovl.OVL_F64 | ovl.OVL_F32 | ovl.OVL_F16R12)
    x = torch.randn(12 * L ** 4, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for fl in (ovl.OVL_LINKS_F32, ovl.OVL_LINKS_F16R12):
        for _ in range(3):
            ovl.ovl_apply_DW(lat, -2.0, 0.3, fl | ovl.OVL_NATIVE | ovl.OVL_GAMMA5, x, y)
    torch.cuda.synchronize()
    ovl.ovl_destroy_lattice(lat)
    ovl.ovl_ctx_destroy(ctx)


def case_pair(L: int, multishift: bool = False, prec: str = "f64", nrhs: int = 1):
    import torch

    import paper_0910_1048_gb300 as ovl
    import synth

    ctx = ovl.ovl_ctx_create(0)
    dims = (L, L, L, L)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, synth.gauge_links(dims, 0), ovl.OVL_F64)
    b = torch.from_numpy(synth.gaussian_source(dims, 1000, nrhs=nrhs if nrhs > 1 else None)).cuda()
    x = torch.empty_like(b)
    pr = {"f64": ovl.OVL_PREC_F64, "f32": ovl.OVL_PREC_F32, "f16": ovl.OVL_PREC_F32_F16LINKS}[prec]
    if prec != "f64":
        ovl.ovl_set_links(lat, synth.gauge_links(dims, 0), ovl.OVL_F64 | ovl.OVL_F32 | ovl.OVL_F16R12)
    if multishift:
        # FP64: 30 iterations with the poles of tol 1e-15; reduced precision: a 1e-8 solve, whose
        # FP64 reliable updates run batched correction solves after the main pass
        p = ovl.ovl_sign_params_default(method=ovl.OVL_MULTISHIFT_BICG, mu=0.3, tol=0.0 if prec == "f64" else 1e-8,
                                        k_max=30 if prec == "f64" else 3000, spec_lo=0.06, spec_hi=2.7, use_graphs=0,
                                        precision=pr)
    else:
        p = ovl.ovl_sign_params_default(mu=0.3, fixed_k=30, use_graphs=0, precision=pr)
    ovl.ovl_apply_sign(lat, p, b, x)
    torch.cuda.synchronize()
    ovl.ovl_destroy_lattice(lat)
    ovl.ovl_ctx_destroy(ctx)


def summarize(path: str, out: str):
    tot = collections.defaultdict(float)
    cnt = collections.Counter()
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        v = float(r["Metric Value"].replace(",", ""))
        name = r["Kernel Name"].split("(")[0]
        tot[name] += v * scale.get(r.get("Metric Unit", "ns"), 1e-3)
        cnt[name] += 1
    all_t = sum(tot.values())
    with open(out, "w") as f:
        f.write("launches=%d total_us=%.1f\n" % (sum(cnt.values()), all_t))
        f.write("%-60s %9s %12s %7s %10s\n" % ("kernel", "launches", "total_us", "share", "mean_us"))
        for k, t in sorted(tot.items(), key=lambda x: -x[1]):
            f.write("%-60s %9d %12.1f %6.1f%% %10.2f\n" % (k[:60], cnt[k], t, 100 * t / all_t, t / cnt[k]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["dslash", "pair", "multishift", "summarize"])
    ap.add_argument("args", nargs="*")
    ap.add_argument("--L", type=int, default=8)
    ap.add_argument("--prec", choices=["f64", "f32", "f16"], default="f64")
    ap.add_argument("--nrhs", type=int, default=1)
    a = ap.parse_args()
    if a.case == "dslash":
        case_dslash(a.L)
    elif a.case == "pair":
        case_pair(a.L, prec=a.prec, nrhs=a.nrhs)
    elif a.case == "multishift":
        case_pair(a.L, multishift=True, prec=a.prec, nrhs=a.nrhs)
    else:
        summarize(*a.args)
    print("ok")


if __name__ == "__main__":
    main()
