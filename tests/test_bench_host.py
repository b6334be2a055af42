"""Host logic of bench.py (no GPU): workload table consistency and the roofline's algorithmic
bytes / flops per pair-stencil launch."""
import bench


def test_workloads_consistent():
    for name, wl in bench.WORKLOADS.items():
        assert len(wl["dims"]) == 4 and all(d % 2 == 0 for d in wl["dims"]), name
        assert wl["method"] in ("direct", "multishift", "fom") and wl["precision"] in ("f64", "f32", "f16"), name
        if wl["precision"] == "f16":
            assert wl["method"] == "multishift", "FP16 links only under the multishift's FP64 reliable updates"
    for name, comps in bench.COMPANIONS.items():
        wl = bench.WORKLOADS[name]
        for key, cname in comps:
            m = bench.WORKLOADS[cname]
            if key.startswith("mixed_precision"):
                # a mixed-precision companion solves the same problem to at least the same accuracy
                assert m["dims"] == wl["dims"] and m["mus"] == wl["mus"] and m["m"] == wl["m"], (name, key)
                assert m["tol"] <= wl["tol"], (name, key)
    assert bench.DEFAULT_WORKLOAD in bench.WORKLOADS
    for name, tab in bench.K_TABLE.items():
        assert set(tab) == set(bench.WORKLOADS[name]["mus"]), name
        assert all(0 < k <= bench.WORKLOADS[name]["k_max"] for k in tab.values()), name


def test_reference_arm_runs_full_oracle_solves(capsys, monkeypatch):
    """--impl reference on the 4^4 workload: one full oracle solve at the tabled k, split over the
    timed steps; the JSON line carries the contract's keys."""
    import json
    import sys

    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "lattice4_mu0.3_direct_f64",
                                      "--steps", "3", "--warmup", "1"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["config"]["k_per_mu"] == {"0.3": bench.K_TABLE["lattice4_mu0.3_direct_f64"][0.3]}
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_cpu_baseline_reports_one_core_and_all_cores():
    """The oracle leg of the bench line: one 4^4 solve at the tabled k, and the C oracle's time per
    Lanczos step on one core and on all cores (the thread count is restored afterwards)."""
    from oracle import krylov

    wl = bench.WORKLOADS["lattice4_mu0.3_direct_f64"]
    before = krylov.threads()
    res = bench.cpu_baseline(wl, "lattice4_mu0.3_direct_f64", [], seconds=5.0)
    assert krylov.threads() == before
    assert res["kind"] == "oracle" and res["value"] > 0 and res["cores"] == before
    steps = res["step_ms_by_cores"]
    assert set(steps) == {"1", str(before)} and all(v > 0 for v in steps.values())


def test_pair_bytes_count_links_once_per_batch():
    vol = 16 ** 4
    one = bench.pair_bytes("f32", vol, 1)
    assert one == vol * bench.PAIR_BYTES_PER_SITE["f32"] == vol * (2 * 96 + 4 * 72 + 2 * 96)
    # 16 right-hand sides share the links: 16 x spinor traffic, links once
    assert bench.pair_bytes("f32", vol, 16) == vol * (4 * 72 + 16 * 4 * 96)
    assert bench.pair_bytes("f16", vol, 1) == vol * (4 * 12 * 2 + 4 * 96)
    assert bench.pair_bytes("f64", vol, 1) == vol * (4 * 144 + 4 * 192)
    assert bench.PAIR_FLOPS_PER_SITE == 2 * 1368


def test_roofline_arithmetic():
    """The line's roofline: FP64 pair stencil = algorithmic flops (2 x 1368 per site and rhs) per
    event-timed launch against the FP64 peak; FP32 = algorithmic bytes (links once per batch) per
    launch against the measured HBM copy bandwidth."""
    infos = [[(0, [{"t_kernel_ms": 0.08, "kernel_samples": 4}])], [(0, [{"t_kernel_ms": 0.12, "kernel_samples": 4}])]]
    t = 0.1e-3  # mean of the two steps' samples, seconds
    r = bench._roofline(bench.WORKLOADS["lattice12_mu0.3_direct_f64"], infos, 1.25, "probe")
    assert r["bound"] == "alu" and r["peak"] == 1.25
    assert abs(r["achieved"] - 2 * 1368 * 12 ** 4 / t / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1.25) < 1e-12
    wl = bench.WORKLOADS["lattice16_mu0.2_nrhs16_direct_f32"]
    r = bench._roofline(wl, infos, 1.25, "probe")
    peak = bench._peaks()[0]["hbm_gbs"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == peak
    assert abs(r["achieved"] - bench.pair_bytes("f32", 16 ** 4, 16) / t / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-12


def test_throughput_counts_every_rank():
    assert bench.throughput(steps=5, solves_per_step=3, world=2, max_ms=1000.0) == 30.0


def test_serving_stream_is_the_configured_distribution():
    """The serving stream is deterministic (seed 42) and draws what the configuration states:
    20 fields over four lattice sizes, mu in [0, 1], three tolerances, 1-8 sources, unit-mean gaps."""
    import numpy as np

    a = bench._serving_stream(2000)
    b = bench._serving_stream(2000)
    assert a == b and len(a) == 2000
    assert {r["L"] for r in a} == set(bench.SERVING["sizes"])
    assert {r["fi"] for r in a} == set(range(20))
    assert all(r["L"] == bench.SERVING["sizes"][r["fi"] // 5] for r in a)
    assert all(0.0 <= r["mu"] <= 1.0 for r in a) and {r["tol"] for r in a} == set(bench.SERVING["tols"])
    assert {r["nrhs"] for r in a} == set(range(1, 9))
    assert abs(np.mean([r["gap"] for r in a]) - 1.0) < 0.1
    assert bench._serving_stream(200) == a[:200]  # a prefix is the first requests of the full stream


def test_summarize_launches(tmp_path, capsys):
    """--summarize-launches: per-kernel totals, shares and means of an ncu launch list, starting at
    the first launch of a named kernel."""
    rows = [("probe<double>", 100.0), ("ovl::k_lz_start<double>", 2.0), ("ovl::k_lz_pair_dyn<double, 0>", 80.0),
            ("ovl::k_lz_update<double, 1, 0>", 20.0), ("ovl::k_lz_pair_dyn<double, 0>", 82.0)]
    lines = ["==PROF== Connected to process 1", '"ID","Kernel Name","Metric Unit","Metric Value"']
    for i, (name, us) in enumerate(rows):
        lines.append('"%d","void %s(Geom, LzDev)","ns","%d"' % (i, name, int(us * 1000)))
    p = tmp_path / "launches.csv"
    p.write_text("\n".join(lines) + "\n")
    bench.summarize_launches(str(p), "k_lz_start")
    out = capsys.readouterr().out.splitlines()
    assert out[0] == "launches=4 total_us=184.0"
    first = out[2].split()
    assert first[0] == "ovl::k_lz_pair_dyn<double," and first[-4:] == ["2", "162.0", "88.0%", "81.00"]
