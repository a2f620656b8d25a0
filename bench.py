"""Benchmark of the alpha-circulant preconditioned Richardson iteration on one
GB300 (or N independent replicas, one per GPU under torchrun).

Headline workload: 2D advection-diffusion u_t + c.grad u = nu Lap u with
c = (1, 0.5), nu = 1e-3 on the periodic unit square, 512 x 512 grid,
second-order central stencils, Radau IIA with M = 3 nodes, L = 512 time steps,
T = 2, u0 a seeded random-phase Gaussian bump field: 402.7 M space-time
degrees of freedom, 3.2 GB per FP64 space-time vector (synthetic data shaped
after the paper's periodic advection and heat tests).  One step = one
Richardson iteration u <- u + C_alpha^{-1}(w - C u) in FP64 (complex128
preconditioner, FP64 residual and update).

Prints one JSON line (rank 0).  Beside the headline it carries the end-to-end
figure through the public API with host buffers, the mixed form's iteration
(complex64 preconditioner), the times to a 1e-10 residual in FP64 and mixed
precision, the sequential baseline on the same GPU, the other four workloads,
the roofline of the dominant kernel, and the CPU oracle (sequential sparse-LU
stepping) timed on the host cores.  --impl reference times that CPU oracle
alone.
"""
import argparse
import json
import math
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HEADLINE = 5
TOL = 1e-10
METRIC = "space-time DoF*iterations/s"
UNIT = "DoF*it/s"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(cfg):
    """The workload description both arms print (identical dicts)."""
    from paper_2103_12571_gb300 import workloads
    prob, _, ex = workloads.config(cfg)
    N = prob["nx"] * prob["ny"]
    desc = {
        1: "1D heat, nu = 0.1, 2nd-order central, u0 = sin 2 pi x + 0.5 sin 6 pi x",
        2: "2D heat, nu = 0.05, 5-point Laplacian, u0 = 16 seeded cosine modes",
        3: "1D advection, c = 1, 4th-order central, Gaussian pulse",
        4: "2D heat, nu = 0.05, 5-point Laplacian, smoothed noise (adjoint workload)",
        5: "2D advection-diffusion, c = (1, 0.5), nu = 1e-3, 2nd-order central, random-phase Gaussian bumps",
    }[cfg]
    return {"workload": ex["name"], "pde": desc, "grid": [prob["nx"], prob["ny"]] if prob["dim"] == 2 else [prob["nx"]],
            "N": N, "M": prob["M"], "L": prob["L"], "T": prob["T"], "DoF": prob["L"] * prob["M"] * N,
            "inputs": "seeded synthetic fields (paper_2103_12571_gb300/workloads.py)"}


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


# ------------------------------------------------------ algorithmic counts
def fp64_flops_per_dof(M, taps):
    # residual of one DoF: stencil (1 mul + taps-1 fma), M fma of the node
    # mix, 1 fma of the coupling term, plus 1/M mul for s_l * u_{l-1,M};
    # flops count an fma as 2
    return (1 + 2 * (taps - 1)) + 2 * M + 2 + 1.0 / M


def kernel_counts(prob, csize, taps):
    """Algorithmic flops and HBM bytes per launch of each kernel kind of one
    iteration (the library's profiler names).  FFTs of length n count
    5 n log2 n flops per complex transform (2.5 n log2 n for a real one);
    a complex multiply-add counts 8.  The pointwise shifted division
    v / (1 - mu sigma_x - mu sigma_y), with the products mu sigma tabulated
    per axis, counts 15: 3 to form the denominator, 3 for its squared
    modulus, 1 reciprocal, 6 for the product with its conjugate and 2 to
    scale.
    Bytes: each array read or written once per launch."""
    L, M = prob["L"], prob["M"]
    nx, ny = prob["nx"], prob["ny"] if prob["dim"] == 2 else 1
    N = nx * ny
    D = L * M * N
    F = L // 2 + 1
    P = F * M * N                                   # complex points of the transform buffer X
    lg = math.log2
    tfft = 2.5 * L * lg(L) * M * N                  # real-data DFT along time of all M*N columns
    mix = 8.0 * M * M * F * N                       # M x M complex mix per stored frequency
    return {
        "resid_tfft_mix": {"flops": D * fp64_flops_per_dof(M, taps) + tfft + mix,
                           "bytes": 8.0 * D + P * csize, "points": P},
        "space_rows": {"flops": P * 5.0 * lg(nx), "bytes": 2.0 * P * csize, "points": P},
        "space_cols": {"flops": P * (10.0 * lg(ny) + 15.0), "bytes": 2.0 * P * csize, "points": P},
        "spatial_solve": {"flops": P * (10.0 * lg(N) + 15.0), "bytes": 2.0 * P * csize, "points": P},
        "mix_tifft_update": {"flops": mix + tfft + 2.0 * D, "bytes": P * csize + 16.0 * D, "points": P},
    }


KERNEL_SOURCES = ["paper_2103_12571_gb300/csrc/k_time.cuh", "paper_2103_12571_gb300/csrc/k_upd.cu",
                  "paper_2103_12571_gb300/csrc/fft.cuh", "paper_2103_12571_gb300/csrc/common.cuh",
                  "paper_2103_12571_gb300/csrc/k_space.cu", "paper_2103_12571_gb300/csrc/norm2.cuh"]


def source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def measured_traffic(kind, precision, alg_bytes, path=None):
    """DRAM bytes per launch of a kernel kind from the last ncu capture (taken
    on a smaller case of the same kernel and scaled by the ratio of
    algorithmic bytes, i.e. by the units a launch processes), if the capture
    was taken on the current kernel sources; else None."""
    try:
        t = json.load(open(path or TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    if t.get("source_sha256") != source_hash():
        return None
    e = t.get("kernels", {}).get("%s@%s" % (kind, precision))
    if not e:
        return None
    return e["dram_bytes"] * alg_bytes / e["alg_bytes"]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# FP64 pipe of a GB300: 2 DFMA per clock per SM, 152 SMs, 2.07 GHz max clock
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12


def kernel_table(prof, counts, precision, steps, fp64_measured_tflops):
    """Per kernel kind: time per launch, algorithmic rate, fraction of the
    bound that applies (FP64 pipe for complex128 transforms and the FP64
    residual, HBM otherwise)."""
    hbm = peaks().get("hbm_gbs", 6800.0)
    out = {}
    for kind, (ms, cnt) in prof.items():
        if cnt == 0 or kind not in counts:
            continue
        per = ms / cnt
        c = counts[kind]
        tf = c["flops"] / (per * 1e-3) / 1e12
        gbs = c["bytes"] / (per * 1e-3) / 1e9
        fp64 = precision == "c128" or kind == "resid_tfft_mix"
        row = {"launches_per_step": cnt / steps, "ms_per_launch": round(per, 4),
               "algorithmic_tflops": round(tf, 4), "algorithmic_gbs": round(gbs, 1),
               "frac_of_measured_hbm": round(gbs / hbm, 3)}
        if fp64:
            # the complex128 FFT flops all run on the FP64 pipe; in complex64
            # plans only the residual part of resid_tfft_mix does
            f64 = c["flops"] if precision == "c128" else None
            if f64 is not None:
                row["frac_of_fp64_peak"] = round(tf / FP64_PEAK_TFLOPS, 3)
                if fp64_measured_tflops:
                    row["frac_of_fp64_measured"] = round(tf / fp64_measured_tflops, 3)
        out[kind] = row
    return out


def dominant_kernel(ktab):
    """The kernel with the most time per step.  The three-pass spatial solve
    counts as its row and column kernels (space_rows, space_cols), the
    one-launch spatial paths as spatial_solve."""
    single = {k: v for k, v in ktab.items() if k not in ("space_rows", "space_cols")}
    if "space_rows" in ktab or "space_cols" in ktab:
        single = {k: v for k, v in ktab.items() if k != "spatial_solve"}
    return max(single, key=lambda k: single[k]["ms_per_launch"] * single[k]["launches_per_step"])


def roofline(kind, prof_row, counts, precision, fp64_measured_tflops):
    c = counts[kind]
    per = prof_row["ms_per_launch"]
    if precision == "c128":
        ach = c["flops"] / (per * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2 flop (FP64 pipe)",
                "peak_measured": fp64_measured_tflops,
                "frac_of_measured": ach / fp64_measured_tflops if fp64_measured_tflops else None,
                "peak_measured_source": "ac_measure_fp64_fma_rate on this GPU in this run (register-operand DFMA chains)",
                "algorithmic_flops_per_launch": c["flops"]}
    else:
        hbm = peaks().get("hbm_gbs", 6800.0)
        ach = c["bytes"] / (per * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "algorithmic_bytes_per_launch": c["bytes"]}
    roof["kernel"] = kind
    roof["kernel_ms"] = per
    roof["traffic"] = measured_traffic(kind, precision, c["bytes"])
    roof["traffic_source"] = "profiles/traffic.json (ncu dram__bytes_read.sum + dram__bytes_write.sum on the same grid " \
                             "with L = 64, scaled by algorithmic bytes)"
    return roof


# ------------------------------------------------------------ CPU oracle
def oracle_worker(cfg, warmup, steps, budget_s):
    """The CPU oracle on workload `cfg`: one sparse LU of C_coll, then the
    sequential collocation steps (eq. (seq_collocation_problem)) one at a
    time, as oracle/sequential.py computes them.  Times the factorisation
    and each step; stops after `steps` timed steps or `budget_s` seconds of
    stepping.  Prints one JSON object."""
    from oracle import collocation, operators, sequential
    from paper_2103_12571_gb300 import workloads
    prob, u0, _ = workloads.config(cfg)
    t_start = time.perf_counter()
    Q = collocation.collocation_matrix(collocation.radau_iia_nodes(prob["M"]))
    A = operators.spatial_operator(prob)
    t0 = time.perf_counter()
    st = sequential.Stepper(A, Q, prob["T"] / prob["L"], u0)
    t_factor = time.perf_counter() - t0
    for _ in range(warmup):
        st.step()
    times = []
    t_steps = time.perf_counter()
    while len(times) < steps and (time.perf_counter() - t_steps) < budget_s and len(times) + warmup < prob["L"]:
        t0 = time.perf_counter()
        st.step()
        times.append(time.perf_counter() - t0)
    N = prob["nx"] * prob["ny"]
    M, L = prob["M"], prob["L"]
    step_s = float(np.mean(times))
    threads = os.environ.get("OMP_NUM_THREADS", "?")
    return {"factor_s": t_factor, "step_s": step_s, "step_s_median": float(np.median(times)),
            "steps_timed": len(times), "warmup_steps": warmup, "L": L, "dof_per_step": M * N,
            "value": M * N / step_s, "full_solve_s": t_factor + L * step_s,
            "threads": int(threads) if threads.isdigit() else threads,
            "cpu": platform.machine() + " " + (platform.processor() or ""),
            "cores_available": len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count(),
            "wall_s": time.perf_counter() - t_start}


def start_oracle_worker(cfg, threads, warmup, steps, budget_s):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-worker", str(cfg), "--warmup", str(warmup),
           "--steps", str(steps), "--cpu-budget", str(budget_s)]
    return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)


def finish_oracle_worker(proc, timeout):
    try:
        out, err = proc.communicate(timeout=timeout)
    except subprocess.TimeoutExpired:
        proc.kill()
        return {"unavailable": "the CPU oracle did not finish within %d s" % timeout}
    for line in reversed(out.strip().splitlines()):
        if line.startswith("{"):
            return json.loads(line)
    return {"unavailable": "CPU oracle failed: " + err.strip()[-300:]}


def cpu_sample_text(r, cfg):
    return ("oracle/sequential.py on the %s workload: one sparse LU of C_coll (minimum-degree ordering, "
            "%.1f s), then %d warm-up and %d timed sequential collocation steps (each one forward/back "
            "substitution over M*N = %d DoF, %.3f s); value = M*N / mean step time; the whole sequential solve "
            "(factorisation + L = %d steps) would take %.0f s" %
            (workload_config(cfg)["workload"], r["factor_s"], r["warmup_steps"], r["steps_timed"],
             r["dof_per_step"], r["step_s"], r["L"], r["full_solve_s"]))


# --------------------------------------------------------------- our arm
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


def correction_alpha(L, precision, tau=0.0):
    eps = 2.0 ** -53 if precision == "c128" else 2.0 ** -24
    return min(0.25, max(1e-8, math.sqrt(L * (3 * eps + tau))))


def run_ours(args):
    rank, world, local = dist_env()
    cpu_proc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_extras:
        # the CPU oracle runs in its own process while the GPU is measured
        cpu_proc = start_oracle_worker(args.workload, 1, 2, args.cpu_steps, args.cpu_budget)
    import torch
    from paper_2103_12571_gb300 import workloads
    from paper_2103_12571_gb300.api import Plan, measure_fp64_fma_rate, stencil_taps

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prob, u0_np, ex = workloads.config(args.workload)
    if args.L:
        # profiling captures: the same grid and dT with fewer steps
        prob = dict(prob, L=args.L, T=prob["T"] * args.L / prob["L"])
    L, M = prob["L"], prob["M"]
    N = prob["nx"] * prob["ny"]
    D = L * M * N
    _, _, rad = stencil_taps(prob)
    taps = 1 + 2 * rad * prob["dim"]
    st = torch.cuda.current_stream()
    u0 = torch.from_numpy(u0_np).cuda()
    big = D * 8 > 4 * 126 * 2 ** 20            # inputs larger than L2 (126 MB) by a wide margin
    flush = None if big else torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # ---- headline: one FP64 Richardson iteration, inputs resident in HBM
    # (--mixed, for profiling captures only: the complex64 preconditioner)
    hprec = "c64" if args.mixed else "c128"
    plan = Plan(prob, precision=hprec, alpha="paper", max_iter=60, space_cluster=args.space_cluster)
    alpha = correction_alpha(L, hprec)
    u = u0.repeat(L * M).reshape(L, M, N).contiguous()
    for _ in range(args.warmup):
        plan.richardson_step(alpha, u0, u)
    torch.cuda.synchronize()
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
        if flush is not None:
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
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(float(np.mean(step_ms)), world)
    value = job_value(D, ms, world)
    fp64_tflops = 2 * measure_fp64_fma_rate() / 1e12
    counts64 = kernel_counts(prob, 16 if hprec == "c128" else 8, taps)
    ktab = kernel_table(prof, counts64, hprec, args.steps, fp64_tflops)
    dom = dominant_kernel(ktab)
    roof = roofline(dom, ktab[dom], counts64, hprec, fp64_tflops)
    cfgd = workload_config(args.workload)
    if args.L:
        cfgd = dict(cfgd, L=L, T=prob["T"], DoF=D, workload=cfgd["workload"] + "_L%d" % L)

    if args.no_extras:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms, "steps": args.steps,
                              "warmup": args.warmup, "dtype": "f64" if hprec == "c128" else "f64+c64",
                              "config": cfgd, "kernels": ktab, "roofline": roof}))
        return

    # ---- end to end through the public API with host buffers: every step
    # is one ac_richardson_step_host call on pinned host arrays (the iterate
    # and u0 in, the new iterate out, copied in chunks that overlap the
    # kernels), then a synchronisation; each step timed on its own wall clock
    u_host = torch.empty((L, M, N), dtype=torch.float64, pin_memory=True)
    u_host.copy_(u)
    u0_host = torch.from_numpy(u0_np).pin_memory()
    u0_dev = torch.empty_like(u0)

    def e2e_step():
        plan.richardson_step_host(alpha, u0_host, u_host)
        torch.cuda.synchronize()

    for _ in range(3):
        e2e_step()
    e2e_steps = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        e2e_step()
        e2e_steps.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = max_over_ranks(float(np.median(e2e_steps)), world)

    # ---- time to a 1e-10 relative residual: FP64 (Algorithm 2) and mixed,
    # and the whole solve end to end from a host u0 to the host solution
    plan32 = Plan(prob, precision="c64", alpha="mixed", max_iter=60)
    ttt = {}
    for name, p in (("fp64", plan), ("mixed", plan32)):
        p.solve(u0, TOL, u=u)   # warm (tables)
        box = {}

        def go():
            box["u"], box["st"] = p.solve(u0, TOL)

        tms = _timed(torch, st, go)
        s2 = box["st"]
        ttt[name] = {"ms": round(tms, 3), "iters": s2["iters"], "res_rel": s2["res_rel"][-1],
                     "res_history": [float("%.3e" % v) for v in s2["res_rel"]],
                     "alpha": [float("%.3e" % v) for v in s2["alpha"]]}
        del box
    torch.cuda.empty_cache()

    def e2e_solve():
        u0_dev.copy_(u0_host, non_blocking=True)
        uu, s3 = plan.solve(u0_dev, TOL)
        u_host.copy_(uu, non_blocking=True)
        torch.cuda.synchronize()
        return s3

    t0 = time.perf_counter()
    s3 = e2e_solve()
    e2e_solve_ms = (time.perf_counter() - t0) * 1e3

    # ---- the mixed form's iteration (complex64 preconditioner)
    alpha32 = correction_alpha(L, "c64")
    for _ in range(3):
        plan32.richardson_step(alpha32, u0, u)
    plan32.profile(True)
    mixed_ms = _timed(torch, st, lambda: plan32.richardson_step(alpha32, u0, u), reps=10, flush=flush)
    prof32 = plan32.profile_read()
    plan32.profile(False)
    k32 = kernel_table(prof32, kernel_counts(prob, 8, taps), "c64", 10, fp64_tflops)
    del plan32
    torch.cuda.empty_cache()

    # ---- the sequential baseline of Sec. 4.2 on the same GPU: the L steps one
    # after another, each by diagonalisation of Q (FP64, replayed from a CUDA
    # graph); the speedups of the all-at-once solves to 1e-10 over it
    pseq = Plan(prob, precision="c128")
    useq = pseq.sequential_solve(u0)          # capture the graph, warm
    seq_ms = _timed(torch, st, lambda: pseq.sequential_solve(u0, out=useq), reps=3)
    umix = Plan(prob, precision="c64", alpha="mixed", max_iter=60).solve(u0, TOL)[0]
    seq = {"ms": round(seq_ms, 3), "what": "L sequential Radau IIA steps by diagonalisation of Q, FP64, one GPU",
           "speedup_fp64": round(seq_ms / ttt["fp64"]["ms"], 3),
           "speedup_mixed": round(seq_ms / ttt["mixed"]["ms"], 3),
           "rel_diff_mixed_vs_sequential": float("%.3e" % float(torch.linalg.norm(umix - useq) /
                                                                  torch.linalg.norm(useq)))}
    del pseq, useq, umix
    torch.cuda.empty_cache()
    del plan
    torch.cuda.empty_cache()

    configs = None
    if not args.no_configs:
        configs = all_configs(torch, st, skip=args.workload)
        configs[ex["name"]] = {"DoF": D, "step_ms": {"c128": round(ms, 4), "c64": round(mixed_ms, 4)},
                               "dof_it_per_s": {"c128": value / world, "c64": D / (mixed_ms * 1e-3)},
                               "solve": {"fp64": {k: ttt["fp64"][k] for k in ("ms", "iters", "res_rel")},
                                         "mixed": {k: ttt["mixed"][k] for k in ("ms", "iters", "res_rel")}}}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfgd,
        "step": "one Richardson iteration u <- u + C_alpha^{-1}(w - C u): FP64 residual, complex128 "
                "preconditioner (time FFT, node mix, spatial FFT solves), FP64 update; alpha = %.3e" % alpha,
        "l2": ("inputs larger than L2 (%.1f GB per FP64 space-time vector): no flush" % (D * 8 / 1e9)) if big
              else "flushed between timed steps (256 MB write)",
        "parallelism": "replicas" if world > 1 else "1 GPU",
        "e2e": {"value": D / (e2e_ms * 1e-3) * world, "unit": UNIT, "ms_per_step": e2e_ms,
                "ms_per_step_mean": float(np.mean(e2e_steps)), "ms_per_step_max": float(np.max(e2e_steps)),
                "estimator": "median of per-step wall times (max over ranks)",
                "what": "per step: ac_richardson_step_host on pinned host arrays (H2D of the iterate u and of "
                        "u0, the iteration, D2H of the new iterate, copies in 8 chunks overlapping the residual "
                        "and update kernels), host synchronisation",
                "h2d_bytes_per_step": D * 8 + N * 8, "d2h_bytes_per_step": D * 8},
        "e2e_solve": {"ms": round(e2e_solve_ms, 3), "iters": s3["iters"],
                      "value": D * s3["iters"] / (e2e_solve_ms * 1e-3), "unit": UNIT,
                      "what": "H2D of u0, ac_richardson_solve to a 1e-10 residual (FP64), D2H of the solution",
                      "h2d_bytes": N * 8, "d2h_bytes": D * 8},
        "gpu_launches": int(launches),
        "kernels": ktab,
        "mixed_step": {"ms": round(mixed_ms, 4), "value": D / (mixed_ms * 1e-3), "unit": UNIT, "alpha": alpha32,
                       "kernels": k32},
        "time_to_1e-10": ttt,
        "sequential_baseline": seq,
        "all_configs": configs,
        "roofline": roof,
        "fp64_fma_rate_measured_tflops": fp64_tflops,
        "clocks": clk,
        "wall_s_timed": wall,
    }
    if cpu_proc is not None:
        r = finish_oracle_worker(cpu_proc, args.cpu_timeout)
        if "unavailable" in r:
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": r["unavailable"]}
        else:
            out["cpu_baseline"] = {"value": r["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": cpu_sample_text(r, args.workload), "factor_s": r["factor_s"],
                                   "step_s": r["step_s"], "full_solve_s": r["full_solve_s"],
                                   "full_solve_dof_per_s": D / r["full_solve_s"], "cpu": r["cpu"],
                                   "cores_available": r["cores_available"]}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def all_configs(torch, st, skip):
    """The other workloads: one Richardson step in each precision (DoF*it/s),
    and their solves (iterations and time to tolerance)."""
    from paper_2103_12571_gb300 import workloads
    from paper_2103_12571_gb300.api import Plan
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    res = {}
    for i in range(1, 6):
        if i == skip:
            continue
        prob, u0n, ex = workloads.config(i)
        L, M = prob["L"], prob["M"]
        N = prob["nx"] * prob["ny"]
        D = L * M * N
        u0 = torch.from_numpy(u0n).cuda()
        r = {"DoF": D, "step_ms": {}, "dof_it_per_s": {}, "solve": {}}
        for prec in ("c64", "c128"):
            plan = Plan(prob, precision=prec, alpha="mixed")
            a = correction_alpha(L, prec)
            u = u0.repeat(L * M).reshape(L, M, N).contiguous()
            for _ in range(3):
                plan.richardson_step(a, u0, u)
            ms = _timed(torch, st, lambda: plan.richardson_step(a, u0, u), reps=5, flush=flush)
            r["step_ms"][prec] = round(ms, 4)
            r["dof_it_per_s"][prec] = D / (ms * 1e-3)
            del plan, u
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


# -------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle alone (sequential sparse-LU stepping on the headline
    workload, all host cores available to it), each step one actual
    sequential collocation step."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t0 = time.perf_counter()
    proc = start_oracle_worker(args.workload, cores, args.warmup, args.steps, 1e9)
    r = finish_oracle_worker(proc, args.cpu_timeout)
    wall = time.perf_counter() - t0
    cfgd = workload_config(args.workload)
    if "unavailable" in r:
        print(json.dumps({"impl": "reference", "unavailable": r["unavailable"]}))
        return
    value = r["value"]
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": r["steps_timed"], "warmup": r["warmup_steps"], "ms_per_step": r["step_s"] * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": cfgd,
           "step": "one sequential collocation step of the CPU oracle (forward/back substitution with the "
                   "sparse LU factors of C_coll) over M*N DoF",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": cpu_sample_text(r, args.workload), "threads": r["threads"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "factor_s": r["factor_s"], "full_solve_s": r["full_solve_s"],
           "full_solve_dof_per_s": cfgd["DoF"] / r["full_solve_s"], "wall_s": wall}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=HEADLINE, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--L", type=int, default=0, help="profiling: the workload's grid and dT with L steps")
    ap.add_argument("--cpu-steps", type=int, default=20, help="timed steps of the CPU oracle sample")
    ap.add_argument("--cpu-budget", type=float, default=30.0, help="seconds of CPU oracle stepping at most")
    ap.add_argument("--cpu-timeout", type=int, default=1500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-workload section")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed steps (used for ncu captures): no e2e, time-to-tolerance or CPU legs")
    ap.add_argument("--mixed", action="store_true",
                    help="with --no-extras: time the mixed form's iteration instead (profiling captures)")
    ap.add_argument("--space-cluster", type=int, default=0, choices=[0, 4, 8, 16],
                    help="with --no-extras: the single-pass cluster spatial solve with this many CTAs per "
                         "cluster (profiling captures; the default three passes measured faster)")
    ap.add_argument("--oracle-worker", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_worker:
        print(json.dumps(oracle_worker(args.oracle_worker, args.warmup, args.steps, args.cpu_budget)))
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.mixed and not args.no_extras:
        ap.error("--mixed is a profiling switch: use it with --no-extras")
    if args.space_cluster and not args.no_extras:
        ap.error("--space-cluster is a profiling switch: use it with --no-extras")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
