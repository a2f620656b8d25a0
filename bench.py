"""Benchmark of the alpha-circulant preconditioned Richardson iteration on
one GB300 (or N independent replicas, one per GPU under torchrun).

Workload: 2D heat u_t = 0.05 Lap u on the periodic unit square, 256 x 256
grid, 5-point Laplacian, Radau IIA with M = 3 nodes, L = 64 time steps,
T = 0.5, u0 a seeded sum of 16 Fourier modes (|k| <= 8) -- the paper's
periodic heat test shape with synthetic data.  One step = one Richardson
iteration u <- u + C_alpha^{-1}(w - C u) of the mixed form (FP64 residual and
update, complex64 preconditioner) with the mixed-rule alpha.

Prints one JSON line (rank 0).  Beside the headline it carries the
end-to-end figure, the time to a 1e-10 residual in FP64 and mixed precision,
the sequential baseline on the same GPU, per-step times and solves of all
five workloads, and the roofline of the dominant kernel.  --impl reference
times the CPU oracle instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIG = 2
TOL = 1e-10


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value, world):
    """Max of a per-rank float over all ranks (the job's step time); works
    with the NCCL and gloo backends."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(dof_per_rank, ms_max, world):
    """Whole-job throughput of independent replicas: all ranks' DoF*it per step
    over the slowest rank's step time."""
    return dof_per_rank * world / (ms_max * 1e-3)


def flush_l2(torch, buf):
    buf.add_(1.0)


def fp64_flops_per_dof(M, taps):
    # residual of one DoF: stencil (1 mul + taps-1 fma), M fma of the node
    # mix, 1 fma of the coupling term, plus 1/M mul for s_l * u_{l-1,M};
    # flops count an fma as 2
    return (1 + 2 * (taps - 1)) + 2 * M + 2 + 1.0 / M


KERNEL_SOURCES = ["paper_2103_12571_gb300/csrc/k_time.cuh", "paper_2103_12571_gb300/csrc/k_upd.cu",
                  "paper_2103_12571_gb300/csrc/fft.cuh", "paper_2103_12571_gb300/csrc/common.cuh",
                  "paper_2103_12571_gb300/csrc/k_space.cu"]


def source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the last ncu capture, if it was
    taken on the current kernel sources (else None)."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None
    if t.get("source_sha256") != source_hash():
        return None
    return t.get("kernels", {}).get(kernel)


def roofline(dom, dom_ms, D, L, M, N):
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # FP64 pipe: 2 DFMA/clk/SM (a probe reached 98% of it) x 152 SMs x 2.07 GHz x 2 flop
    fp64_peak = 2 * 2 * 152 * 2.07e9 / 1e12
    csz = 8
    F = L // 2 + 1
    if dom == "resid_tfft_mix":
        flops = fp64_flops_per_dof(M, 5) * D
        roof = {"bound": "alu", "achieved": flops / (dom_ms * 1e-3) / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2 flop (FP64 pipe)",
                "algorithmic_flops_per_launch": flops,
                "hbm_gbs_algorithmic": (8.0 * D + F * M * N * csz) / (dom_ms * 1e-3) / 1e9}
    else:
        bytes_ = {"spatial_solve": 6 * F * M * N * csz,
                  "mix_tifft_update": F * M * N * csz + 16.0 * D}.get(dom, 16.0 * D)
        roof = {"bound": "hbm", "achieved": bytes_ / (dom_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)", "algorithmic_bytes_per_launch": bytes_}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = dom
    roof["kernel_ms"] = dom_ms
    tr = measured_traffic({"resid_tfft_mix": "k_fwd", "spatial_solve": "k_space", "mix_tifft_update": "k_upd"}.get(dom, dom))
    roof["traffic"] = tr
    return roof


def run_ours(args):
    import torch
    from paper_2103_12571_gb300 import workloads
    from paper_2103_12571_gb300.api import Plan

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prob, u0_np, ex = workloads.config(CONFIG)
    L, M = prob["L"], prob["M"]
    N = prob["nx"] * prob["ny"]
    D = L * M * N
    plan = Plan(prob, precision="c64", alpha="mixed", max_iter=60)
    u0 = torch.from_numpy(u0_np).cuda()
    alpha = min(0.25, max(1e-8, (L * 3 * 2.0 ** -24) ** 0.5))
    u = u0.repeat(L * M).reshape(L, M, N).contiguous()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.richardson_step(alpha, u0, u)
    torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident in HBM), L2 flushed between steps
    plan.profile(True)
    launches0 = plan.info()["launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush_l2(torch, flush)
        ev[i][0].record(st)
        plan.richardson_step(alpha, u0, u)
        ev[i][1].record(st)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    launches = plan.info()["launches"] - launches0
    prof = plan.profile_read()
    plan.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(float(np.mean(step_ms)), world)
    value = job_value(D, ms, world)

    if args.no_extras:
        if rank == 0:
            print(json.dumps({"metric": "space-time DoF*iterations/s", "value": value, "unit": "DoF*it/s",
                              "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                              "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]}}))
        return
    # ---- end to end through the public API: pinned host u0 -> device, one
    # iteration with its residual norm read back to the host
    # (each step timed on its own wall clock; the value uses the median step,
    # so that a host stall in one step does not stand for the steady state;
    # the mean and the slowest step are reported beside it)
    u0_host = torch.from_numpy(u0_np).pin_memory()
    u0_dev = torch.empty_like(u0)
    for _ in range(max(3, args.warmup)):
        u0_dev.copy_(u0_host, non_blocking=True)
        plan.richardson_step(alpha, u0_dev, u, want_residual=True)
    torch.cuda.synchronize()
    e2e_steps = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u0_dev.copy_(u0_host, non_blocking=True)
        plan.richardson_step(alpha, u0_dev, u, want_residual=True)   # returns after the D2H read
        torch.cuda.synchronize()
        e2e_steps.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = max_over_ranks(float(np.median(e2e_steps)), world)
    grid = plan.info()["N"] // plan.info()["tile_fwd"]

    # ---- time to a 1e-10 relative residual: FP64 (Algorithm 2) vs mixed
    ttt = {}
    for name, prec, mode in (("fp64", "c128", "paper"), ("mixed", "c64", "mixed")):
        p2 = plan if prec == "c64" else Plan(prob, precision=prec, alpha=mode, max_iter=60)
        p2.solve(u0, TOL)  # warm
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        uu, stt = p2.solve(u0, TOL)
        b.record(st)
        torch.cuda.synchronize()
        ttt[name] = {"ms": round(a.elapsed_time(b), 3), "iters": stt["iters"],
                     "res_rel": stt["res_rel"][-1], "res_history": [float("%.3e" % v) for v in stt["res_rel"]],
                     "alpha": [float("%.3e" % v) for v in stt["alpha"]]}
        if prec == "c128":
            p2.profile(True)
            p2.richardson_step(1e-6, u0, uu)
            ttt[name]["kernel_ms"] = {k: round(v[0], 4) for k, v in p2.profile_read().items() if v[1]}
            del p2

    # ---- the sequential baseline of Sec. 4.2 on the same GPU: the L steps one
    # after another, each by diagonalisation of Q (FP64, replayed from a CUDA
    # graph), and the speedup of the all-at-once solves to 1e-10 over it
    pseq = Plan(prob, precision="c128")
    useq = pseq.sequential_solve(u0)          # capture the graph, warm
    umix, _ = plan.solve(u0, TOL)
    seq_runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        pseq.sequential_solve(u0, out=useq)
        b.record(st)
        torch.cuda.synchronize()
        seq_runs.append(a.elapsed_time(b))
    seq_ms = float(np.median(seq_runs))
    seq = {"ms": round(seq_ms, 3), "what": "L sequential Radau IIA steps by diagonalisation of Q, FP64, one GPU",
           "speedup_fp64": round(seq_ms / ttt["fp64"]["ms"], 3),
           "speedup_mixed": round(seq_ms / ttt["mixed"]["ms"], 3),
           "rel_diff_mixed_vs_sequential": float("%.3e" % float(torch.linalg.norm(umix - useq) /
                                                                  torch.linalg.norm(useq)))}
    del pseq

    configs = all_configs(torch, st, flush) if not args.no_configs else None

    # ---- roofline of the dominant kernel
    kern = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms = kern[dom][0] / kern[dom][1]
    roof = roofline(dom, dom_ms, D, L, M, N)
    # algorithmic HBM bytes of each kernel group per step and their share of
    # the measured copy bandwidth (the FP64-bound residual kernel included)
    F = L // 2 + 1
    alg = {"resid_tfft_mix": 8.0 * D + F * M * N * 8, "spatial_solve": 6.0 * F * M * N * 8,
           "mix_tifft_update": F * M * N * 8 + 16.0 * D}
    hbm_peak = roof["peak"] if roof["unit"] == "GB/s" else \
        json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)
    hbm_per_kernel = {}
    for k, b in alg.items():
        if k in kern and kern[k][1]:
            t = kern[k][0] / kern[k][1]
            hbm_per_kernel[k] = {"algorithmic_bytes": b, "ms": round(t, 4), "gbs": round(b / (t * 1e-3) / 1e9, 1),
                                 "frac_of_measured_hbm": round(b / (t * 1e-3) / 1e9 / hbm_peak, 3)}
    out = {
        "metric": "space-time DoF*iterations/s (one alpha-circulant Richardson iteration, mixed FP64/c64)",
        "value": value, "unit": "DoF*it/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+c64", "data": "synthetic",
        "config": {"workload": ex["name"], "N": N, "M": M, "L": L, "T": prob["T"], "DoF": D,
                   "precision": "fp64 residual/update + complex64 preconditioner", "alpha": alpha,
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "e2e": {"value": D / (e2e_ms * 1e-3) * world, "unit": "DoF*it/s", "ms_per_step": e2e_ms,
                "ms_per_step_mean": float(np.mean(e2e_steps)), "ms_per_step_max": float(np.max(e2e_steps)),
                "estimator": "median of per-step wall times (max over ranks)",
                "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": grid * 4},
        "gpu_launches": int(launches),
        "kernels_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in kern.items()},
        "time_to_1e-10": ttt,
        "sequential_baseline": seq,
        "all_configs": configs,
        "roofline": roof,
        "hbm_per_kernel": hbm_per_kernel,
        "clocks": clk,
        "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(prob, u0_np, samples=args.cpu_samples)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def _timed(torch, st, fn, reps=1, flush=None):
    """Median device time (ms) of fn() over reps runs, CUDA events on st."""
    out = []
    for _ in range(reps):
        if flush is not None:
            flush_l2(torch, flush)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return float(np.median(out))


def all_configs(torch, st, flush):
    """The five workloads: one Richardson step in each precision (DoF*it/s),
    and their solves (iterations and time to tolerance)."""
    from paper_2103_12571_gb300 import workloads
    from paper_2103_12571_gb300.api import Plan
    res = {}
    for i in range(1, 6):
        prob, u0n, ex = workloads.config(i)
        L, M = prob["L"], prob["M"]
        N = prob["nx"] * prob["ny"]
        D = L * M * N
        u0 = torch.from_numpy(u0n).cuda()
        r = {"DoF": D, "step_ms": {}, "dof_it_per_s": {}, "solve": {}}
        for prec in ("c64", "c128"):
            plan = Plan(prob, precision=prec, alpha="mixed")
            eps = 2.0 ** -24 if prec == "c64" else 2.0 ** -53
            a = min(0.25, max(1e-8, (L * 3 * eps) ** 0.5))      # the mixed-rule alpha
            u = u0.repeat(L * M).reshape(L, M, N).contiguous()
            for _ in range(3):
                plan.richardson_step(a, u0, u)
            ms = _timed(torch, st, lambda: plan.richardson_step(a, u0, u), reps=5, flush=flush)
            r["step_ms"][prec] = round(ms, 4)
            r["dof_it_per_s"][prec] = D / (ms * 1e-3)
            del plan, u
        # solves as each workload is specified
        runs = []
        if i == 1:
            runs.append(("fp64_fixed_alpha", dict(precision="c128", alpha="fixed", alpha0=ex["alpha"]), ex["tol"]))
        else:
            runs.append(("fp64", dict(precision="c128", alpha="paper"), TOL))
            runs.append(("mixed", dict(precision="c64", alpha="mixed"), TOL))
        for name, kw, tol in runs:
            plan = Plan(prob, max_iter=60, **kw)
            plan.solve(u0, tol)                      # warm (tables, allocations)
            box = {}

            def go():
                box["u"], box["st"] = plan.solve(u0, tol)
            ms = _timed(torch, st, go)
            r["solve"][name] = {"ms": round(ms, 3), "iters": box["st"]["iters"], "tol": tol,
                                "res_rel": float("%.3e" % box["st"]["res_rel"][-1])}
            del plan, box
        if i == 4:
            # forward + adjoint + gradients (FP64), the workload's training step
            plan = Plan(prob, precision="c128", alpha="paper", max_iter=60)
            target = torch.from_numpy(ex["u_target"]).cuda()

            def fwd_bwd():
                u, _ = plan.solve(u0, 1e-13, raise_on_fail=False)
                g = torch.zeros_like(u)
                g[-1, -1] = 2.0 * (u[-1, -1] - target)
                lam, _ = plan.adjoint_solve(g, 1e-13, raise_on_fail=False)
                plan.grad_params(u, lam)
            fwd_bwd()
            r["forward_adjoint_grad_ms"] = round(_timed(torch, st, fwd_bwd), 3)
            del plan
        res[ex["name"]] = r
        torch.cuda.empty_cache()
    return res


def cpu_baseline(prob, u0, samples=1):
    t0 = time.perf_counter()
    it = OracleIteration(prob, u0)
    per = [it.step()[0] for _ in range(max(1, samples))]
    spent = time.perf_counter() - t0
    D = prob["L"] * prob["M"] * prob["nx"] * prob["ny"]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": D / float(np.mean(per)), "unit": "DoF*it/s", "cores": cores, "kind": "oracle",
            "sample": "one oracle Richardson iteration estimated from its parts: FP64 residual, numpy time FFTs "
                      "and one of %d per-frequency block solves timed, the block's sparse LU (%.1f s) timed once, "
                      "scaled to all %d blocks; %.1f s of CPU work" % (prob["L"], it.t_factor, prob["L"], spent)}


class OracleIteration:
    """The oracle's Richardson iteration on the benchmark workload, timed in
    parts: the FP64 residual, the forward and inverse time FFTs and one
    per-frequency block solve are timed every step; the sparse LU of a
    frequency block (about 20-30 s) is timed once.  One iteration is
    estimated as residual + FFTs + L x (factor + solve)."""

    def __init__(self, prob, u0, alpha=3e-3):
        import scipy.sparse.linalg as spla
        from oracle import collocation, operators, paradiag
        self.spla, self.ops, self.pd = spla, operators, paradiag
        t = collocation.radau_iia_nodes(prob["M"])
        self.Q = collocation.collocation_matrix(t)
        self.A = operators.spatial_operator(prob)
        self.L, self.M = prob["L"], prob["M"]
        self.dT = prob["T"] / self.L
        self.u0 = u0
        self.alpha = alpha
        self.N = self.A.shape[0]
        self.u = np.broadcast_to(u0, (self.L, self.M, self.N)).copy()
        d = paradiag.eigenvalues_d(self.L, alpha)
        t0 = time.perf_counter()
        self.lu = spla.splu(paradiag.block_matrix(self.A, self.Q, self.dT, d[1]).astype(np.complex128))
        self.t_factor = time.perf_counter() - t0

    def step(self):
        t0 = time.perf_counter()
        r = self.ops.residual(self.u, self.u0, self.A, self.Q, self.dT)
        x = self.pd.time_forward(r.astype(np.complex128), self.alpha)
        t1 = time.perf_counter()
        y = self.lu.solve(x[1].reshape(-1))
        t2 = time.perf_counter()
        x[1] = y.reshape(self.M, self.N)
        e = self.pd.time_inverse(x, self.alpha)
        t3 = time.perf_counter()
        del e
        return (t1 - t0) + (t3 - t2) + self.L * (self.t_factor + (t2 - t1)), t3 - t0


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2103_12571_gb300 import workloads
    prob, u0, ex = workloads.config(CONFIG)
    D = prob["L"] * prob["M"] * prob["nx"] * prob["ny"]
    t_start = time.perf_counter()
    it = OracleIteration(prob, u0)
    for _ in range(args.warmup):
        it.step()
    per = []
    for _ in range(args.steps):
        p, _ = it.step()
        per.append(p)
    spent = time.perf_counter() - t_start
    ms = float(np.mean(per)) * 1e3
    value = D / (ms * 1e-3)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = ("per step: the oracle's FP64 residual, forward and inverse time FFTs and one of the %d "
              "per-frequency sparse-LU block solves, timed; the block factorisation (%.1f s) timed once; "
              "one iteration = residual + FFTs + %d x (factor + solve); %.1f s in total"
              % (prob["L"], it.t_factor, prob["L"], spent))
    out = {"impl": "reference",
           "metric": "space-time DoF*iterations/s (one alpha-circulant Richardson iteration, mixed FP64/c64)",
           "value": value, "unit": "DoF*it/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": ex["name"], "DoF": D},
           "cpu_baseline": {"value": value, "unit": "DoF*it/s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "DoF*it/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-samples", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-workload section")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed steps (used for ncu captures): no e2e, time-to-tolerance or CPU legs")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
