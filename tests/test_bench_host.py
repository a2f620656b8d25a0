"""Host-side arithmetic of bench.py (CPU): the algorithmic FP64 work of the
residual kernel, the roofline fields, and the traffic lookup keyed to the
kernel sources."""
import json
import os

import pytest

import bench


def test_residual_flop_count_matches_the_kernel_structure():
    """Per grid point and step with M = 3 and the 5-point stencil, the
    residual does, per node, 1 multiply + 4 FMAs of the stencil (9 flops), 1 FMA
    of -s u_m + w and M FMAs of the node mix, plus one multiply s * u_{l-1,M}
    per point: 3 * (9 + 2 + 6) + 1 = 52 flops, issued as 28 DFMAs (56 flops,
    four of them zero-addend multiplies)."""
    assert bench.fp64_flops_per_dof(3, 5) * 3 == pytest.approx(52.0)
    assert bench.fp64_flops_per_dof(1, 3) == pytest.approx(5 + 2 + 2 + 1)


def test_roofline_fields():
    L, M, N = 64, 3, 65536
    D = L * M * N
    r = bench.roofline("resid_tfft_mix", 0.2, D, L, M, N)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(2 * 2 * 152 * 2.07e9 / 1e12)
    assert r["achieved"] == pytest.approx(bench.fp64_flops_per_dof(M, 5) * D / 0.2e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    u = bench.roofline("mix_tifft_update", 0.05, D, L, M, N)
    F = L // 2 + 1
    assert u["bound"] == "hbm" and u["unit"] == "GB/s"
    assert u["algorithmic_bytes_per_launch"] == pytest.approx(F * M * N * 8 + 16.0 * D)
    assert u["frac"] == pytest.approx(u["achieved"] / u["peak"])


def test_traffic_is_null_when_the_kernel_sources_changed(monkeypatch):
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    t = json.load(open(path))
    monkeypatch.setattr(bench, "source_hash", lambda: t["source_sha256"])
    assert bench.measured_traffic("k_fwd") == t["kernels"]["k_fwd"]
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 64)
    assert bench.measured_traffic("k_fwd") is None


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the CPU oracle (no GPU) and prints one
    JSON line with the reference keys."""
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [l for l in out.stdout.splitlines() if l.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "DoF*it/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "heat2d_256x256_M3_L64" and d["higher_is_better"] is True
