"""The Richardson step on host arrays (ac_richardson_step_host): the iterate
goes to the device and back in chunks of grid points that overlap the
residual and update kernels.  The kernels and their tiles are those of the
device step, so the new iterate and the reported residual must equal
ac_richardson_step's bit for bit, for any number of chunks (including
chunks smaller than a stencil halo, which the call merges), with and
without u0 and b, from page-locked and from pageable host memory, and over
consecutive calls."""
import numpy as np
import pytest

from gpu_common import torch_cuda
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

CASES = [
    (workloads.problem(2, 64, 64, nu=0.05, cx=0.5, cy=-0.3, order=2, M=3, L=8, T=0.1), "c128", "fft"),
    (workloads.problem(2, 128, 256, nu=0.02, cx=1.0, cy=0.5, order=4, M=2, L=4, T=0.05), "c64", "fft"),
    (workloads.problem(1, 512, cx=1.0, order=5, upwind=True, M=3, L=16, T=0.25), "c128", "fft"),
    (workloads.problem(1, 8, nu=0.3, order=2, M=1, L=2, T=0.1), "c64", "fft"),
    (workloads.problem(2, 24, 20, nu=0.02, cx=0.4, cy=-0.3, order=2, M=3, L=8, T=0.1), "c128", "bicgstab"),
]


def ids(c):
    p, prec, inner = c
    return "d%d_%dx%d_%s_%s" % (p["dim"], p["nx"], p["ny"], prec, inner)


@pytest.mark.parametrize("case", CASES, ids=ids)
@pytest.mark.parametrize("chunks", [0, 1, 3, 32])
def test_host_step_equals_device_step(case, chunks):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, precision, inner = case
    plan = Plan(prob, precision=precision, inner=inner, tau=1e-10)
    L, M, N = plan.shape
    rng = np.random.default_rng(41)
    u_init = torch.from_numpy(rng.standard_normal((L, M, N)))
    u0 = torch.from_numpy(rng.standard_normal(N))
    alpha = 1e-3
    # device reference: two consecutive steps
    ud = u_init.cuda()
    u0d = u0.cuda()
    ref_res = [plan.richardson_step(alpha, u0d, ud, want_residual=True) for _ in range(2)]
    ref = ud.cpu()
    # host: the same two steps, on page-locked arrays
    uh = u_init.clone().pin_memory()
    u0h = u0.clone().pin_memory()
    res = [plan.richardson_step_host(alpha, u0h, uh, chunks=chunks, want_residual=True) for _ in range(2)]
    torch.cuda.synchronize()
    assert torch.equal(uh, ref)
    assert res == ref_res, (res, ref_res)


def test_host_step_with_b_pageable_memory_and_no_residual():
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = CASES[0][0]
    plan = Plan(prob, precision="c128")
    L, M, N = plan.shape
    rng = np.random.default_rng(42)
    u_init = torch.from_numpy(rng.standard_normal((L, M, N)))
    b = torch.from_numpy(rng.standard_normal((L, M, N)))
    ud, bd = u_init.cuda(), b.cuda()
    plan.richardson_step(2e-3, None, ud, b=bd)
    uh = u_init.clone()                               # pageable
    assert plan.richardson_step_host(2e-3, None, uh, b=b.clone(), chunks=5) is None
    torch.cuda.synchronize()
    assert torch.equal(uh, ud.cpu())


def test_host_step_rejects_device_tensors_and_negative_chunks():
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    plan = Plan(CASES[3][0], precision="c64")
    L, M, N = plan.shape
    with pytest.raises(ValueError):
        plan.richardson_step_host(1e-3, None, torch.zeros((L, M, N), dtype=torch.float64, device="cuda"))
    with pytest.raises(RuntimeError):
        plan.richardson_step_host(1e-3, None, torch.zeros((L, M, N), dtype=torch.float64), chunks=-1)
