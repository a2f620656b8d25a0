"""Host-side arithmetic of bench.py (CPU): the algorithmic work of each
kernel kind, the roofline fields, the traffic lookup keyed to the kernel
sources, and the reference arm's contract line."""
import json
import math
import os

import pytest

import bench
from paper_2103_12571_gb300 import workloads


def test_residual_flop_count_matches_the_kernel_structure():
    """Per grid point and step with M = 3 and the 5-point stencil, the
    residual does, per node, 1 multiply + 4 FMAs of the stencil (9 flops), 1 FMA
    of -s u_m + w and M FMAs of the node mix, plus one multiply s * u_{l-1,M}
    per point: 3 * (9 + 2 + 6) + 1 = 52 flops, issued as 28 DFMAs (56 flops,
    four of them zero-addend multiplies)."""
    assert bench.fp64_flops_per_dof(3, 5) * 3 == pytest.approx(52.0)
    assert bench.fp64_flops_per_dof(1, 3) == pytest.approx(5 + 2 + 2 + 1)


def test_kernel_counts_are_consistent():
    prob, _, _ = workloads.config(5)
    c = bench.kernel_counts(prob, 16, 5)
    L, M, N = prob["L"], prob["M"], prob["nx"] * prob["ny"]
    F = L // 2 + 1
    P = F * M * N
    # the spatial solve is two row passes and one column pass
    assert c["spatial_solve"]["flops"] == pytest.approx(2 * c["space_rows"]["flops"] + c["space_cols"]["flops"])
    assert c["space_cols"]["flops"] == pytest.approx(P * (10 * 9 + 15))
    # bytes: one read and one write of X per pass; u read (+ write) in the time kernels
    assert c["space_rows"]["bytes"] == 2 * P * 16
    assert c["resid_tfft_mix"]["bytes"] == 8 * L * M * N + P * 16
    assert c["mix_tifft_update"]["bytes"] == P * 16 + 16 * L * M * N
    # the time transforms: a real DFT of length L per column, 2.5 L log2 L flops
    tf = 2.5 * L * math.log2(L) * M * N
    assert c["mix_tifft_update"]["flops"] == pytest.approx(tf + 8 * M * M * F * N + 2 * L * M * N)


def test_roofline_fields():
    prob, _, _ = workloads.config(5)
    counts = bench.kernel_counts(prob, 16, 5)
    row = {"ms_per_launch": 20.0}
    r = bench.roofline("space_cols", row, counts, "c128", 1.2)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(2 * 2 * 152 * 2.07e9 / 1e12)
    assert r["achieved"] == pytest.approx(counts["space_cols"]["flops"] / 20e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["frac_of_measured"] == pytest.approx(r["achieved"] / 1.2)
    counts8 = bench.kernel_counts(prob, 8, 5)
    u = bench.roofline("mix_tifft_update", {"ms_per_launch": 2.0}, counts8, "c64", None)
    assert u["bound"] == "hbm" and u["unit"] == "GB/s"
    assert u["algorithmic_bytes_per_launch"] == counts8["mix_tifft_update"]["bytes"]
    assert u["frac"] == pytest.approx(u["achieved"] / u["peak"])


def test_dominant_kernel_splits_the_three_pass_solve():
    ktab = {"resid_tfft_mix": {"ms_per_launch": 10.0, "launches_per_step": 1},
            "spatial_solve": {"ms_per_launch": 50.0, "launches_per_step": 1},
            "space_rows": {"ms_per_launch": 15.0, "launches_per_step": 2},
            "space_cols": {"ms_per_launch": 20.0, "launches_per_step": 1},
            "mix_tifft_update": {"ms_per_launch": 12.0, "launches_per_step": 1}}
    assert bench.dominant_kernel(ktab) == "space_rows"
    one = {k: v for k, v in ktab.items() if k not in ("space_rows", "space_cols")}
    assert bench.dominant_kernel(one) == "spatial_solve"


def test_traffic_is_scaled_and_null_when_the_kernel_sources_changed(tmp_path, monkeypatch):
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps({"source_sha256": "a" * 64,
                                "kernels": {"space_cols@c128": {"dram_bytes": 1000.0, "alg_bytes": 1100.0}}}))
    monkeypatch.setattr(bench, "source_hash", lambda: "a" * 64)
    assert bench.measured_traffic("space_cols", "c128", 4400.0, str(path)) == pytest.approx(4000.0)
    assert bench.measured_traffic("space_rows", "c128", 4400.0, str(path)) is None
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 64)
    assert bench.measured_traffic("space_cols", "c128", 4400.0, str(path)) is None


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the CPU oracle (no GPU): its steps are
    real sequential collocation steps, and it prints one JSON line with the
    reference keys and the same config dict as the GPU arm."""
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "1", "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [l for l in out.stdout.splitlines() if l.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "DoF*it/s"
    assert d["metric"] == bench.METRIC
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"] == bench.workload_config(1) and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1
    # the timed steps were run: they fit inside the arm's own wall clock
    assert d["steps"] * d["ms_per_step"] * 1e-3 <= d["wall_s"]
    assert d["value"] == pytest.approx(d["config"]["M"] * d["config"]["N"] / (d["ms_per_step"] * 1e-3))
