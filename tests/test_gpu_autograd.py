"""Gradients through the torch.autograd.Function (RichardsonSolve): forward by
the alpha-circulant Richardson solve, backward by the adjoint solve and the
gradient contractions.  Checked against the oracle's sequential discrete
adjoint and against central differences of the GPU forward solve
(fourth-order central differences, h = 1e-6), to 1e-7 relative, for u0, nu,
cx and cy."""
import numpy as np
import pytest

from gpu_common import oracle_setup, rel2, to_dev, torch_cuda
from oracle import sequential
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

H = 1e-6
TOL = 1e-15       # finite-difference solves: as far as FP64 goes (no error raised)
TOL_AD = 1e-13    # the autograd solves (forward and adjoint), which raise if they miss it


def _case(name):
    if name == "advdiff2d_32":
        prob = workloads.problem(2, 32, 32, nu=0.05, cx=0.7, cy=-0.4, order=2, M=3, L=16, T=0.1)
        u0 = workloads.u0_fourier_modes_2d(32, 32, n_modes=6, kmax=5, seed=2)
        target = workloads.smoothed_noise_2d(32, 32, 3.0, seed=5)
    elif name == "config4":
        prob, u0, ex = workloads.config(4)
        target = ex["u_target"]
    else:   # config 5 cut down to 128 x 128 and 64 steps of the same dT
        prob = workloads.problem(2, 128, 128, nu=1e-3, cx=1.0, cy=0.5, order=2, M=3, L=64, T=0.25)
        u0 = workloads.random_phase_bumps_2d(128, 128, 8.0, seed=0)
        target = workloads.random_phase_bumps_2d(128, 128, 8.0, seed=1)
    return prob, u0, target


def _loss(torch, u, target_t):
    # the last node of the last step, plus a second block so that the
    # adjoint carries a source inside the time window too
    L = u.shape[0]
    return ((u[-1, -1] - target_t) ** 2).sum() + 0.25 * (u[L // 2, 0] ** 2).sum()


def _loss_np(u, target):
    L = u.shape[0]
    return float(((u[-1, -1] - target) ** 2).sum() + 0.25 * (u[L // 2, 0] ** 2).sum())


@pytest.mark.parametrize("name,precision", [("advdiff2d_32", "c128"), ("advdiff2d_32", "c64"),
                                            ("config4", "c128"), ("advdiff2d_128_L64", "c64")])
def test_richardson_solve_autograd(name, precision):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan, RichardsonSolve
    prob, u0, target = _case(name)
    mode = "paper" if precision == "c128" else "mixed"
    plan = Plan(prob, precision=precision, alpha=mode, max_iter=80)
    x = to_dev(torch, u0).requires_grad_(True)
    params = torch.tensor(plan.params(), dtype=torch.float64, device="cuda", requires_grad=True)
    target_t = to_dev(torch, target)
    u = RichardsonSolve.apply(x, params, plan, TOL_AD)
    _loss(torch, u, target_t).backward()
    gx = x.grad.cpu().numpy()
    gp = params.grad.cpu().numpy()

    # the oracle's sequential discrete adjoint
    Q, A, dT = oracle_setup(prob)
    L, M = prob["L"], prob["M"]
    useq = sequential.sequential_solve(A, Q, dT, L, u0)
    g = np.zeros_like(useq)
    g[-1, -1] = 2 * (useq[-1, -1] - target)
    g[L // 2, 0] += 0.5 * useq[L // 2, 0]
    lam = sequential.sequential_adjoint(A, Q, dT, g)
    du0_ref, dnu_ref, dc_ref = sequential.grad_params(prob, Q, dT, useq, lam)
    assert rel2(gx, du0_ref) < 1e-7
    for got, ref in zip(gp, [dnu_ref, dc_ref[0], dc_ref[1]]):
        assert abs(got - ref) < 1e-7 * max(abs(ref), 1e-3 * np.max(np.abs(gp))), (gp, dnu_ref, dc_ref)

    # central differences of the GPU forward solve (FP64 preconditioner, so
    # that the solves reach the FP64 floor)
    def J(p, v0):
        pl = Plan(p, precision="c128", alpha="paper", max_iter=80)
        uu, _ = pl.solve(to_dev(torch, v0), tol=TOL, raise_on_fail=False)
        return _loss_np(uu.cpu().numpy(), target)

    def fd4(f):
        # fourth-order central difference with step h: the truncation error
        # O(h^4 f^(5)) stays far below 1e-7 even where J depends strongly on
        # the parameter (nu = 1e-3 multiplies the largest symbols)
        return (-f(2 * H) + 8 * f(H) - 8 * f(-H) + f(-2 * H)) / (12 * H)

    def shifted(key, d):
        p = dict(prob)
        p[key] += d
        return p

    for i, key in enumerate(("nu", "cx", "cy")):
        fd = fd4(lambda d: J(shifted(key, d), u0))
        assert abs(fd - gp[i]) < 1e-7 * max(abs(gp[i]), 1e-3 * np.max(np.abs(gp))), (key, fd, gp[i])
    # a smooth direction with entries of order one
    v = workloads.smoothed_noise_2d(prob["nx"], prob["ny"], 2.0, seed=11)
    v /= np.max(np.abs(v))
    fd = fd4(lambda d: J(prob, u0 + d * v))
    assert abs(fd - gx @ v) < 1e-7 * max(abs(fd), 1e-3 * np.linalg.norm(gx)), (fd, gx @ v)


def test_richardson_solve_rejects_params_of_another_problem():
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan, RichardsonSolve
    prob, u0, _ = _case("advdiff2d_32")
    plan = Plan(prob, precision="c128")
    x = to_dev(torch, u0)
    bad = torch.tensor([prob["nu"], prob["cx"] + 0.1, prob["cy"]], dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        RichardsonSolve.apply(x, bad, plan, TOL_AD)
