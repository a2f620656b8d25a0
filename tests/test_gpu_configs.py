"""The five workloads at their full sizes, in the launch configuration the
benchmark uses.  Full-size references: the Fourier closed form of the
collocation stepping (pinned against the sequential oracle in the CPU tests)
for whole blocks, and properties that hold at any size."""
import numpy as np
import pytest

from gpu_common import oracle_setup, rel2, to_dev, torch_cuda
from oracle import fourier, sequential
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu


def modal(prob, u0, blocks=None):
    from oracle import collocation
    Q = collocation.collocation_matrix(collocation.radau_iia_nodes(prob["M"]))
    return fourier.modal_solution(u0, prob, Q, prob["T"] / prob["L"], prob["L"], blocks=blocks)


@pytest.mark.parametrize("precision,mode,tol", [("c128", "paper", 1e-11), ("c64", "mixed", 1e-10)])
def test_config2_full(precision, mode, tol):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, u0, _ = workloads.config(2)
    ref = modal(prob, u0)
    plan = Plan(prob, precision=precision, alpha=mode, max_iter=40)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-10)
    assert st["converged"] and st["res_rel"][-1] <= 1e-10
    u2, st2 = plan.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    assert rel2(u2.cpu().numpy(), ref) < tol, st2


@pytest.mark.parametrize("precision,mode,tol", [("c128", "paper", 1e-11), ("c64", "mixed", 1e-10)])
def test_config3_full_fft(precision, mode, tol):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, u0, ex = workloads.config(3)
    ref = modal(prob, u0)
    plan = Plan(prob, precision=precision, alpha=mode, max_iter=80)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), ref) < tol, st


def test_config3_full_bicgstab_fp64():
    """BiCGStab inner solves at tau = 1e-8 on the CFL-16 central advection:
    with a small fixed alpha (1e-8) every shifted system is solved to tau
    (condition numbers up to about 320) and the outer iteration reaches the
    FP64 answer."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, u0, ex = workloads.config(3)
    ref = modal(prob, u0)
    plan = Plan(prob, precision="c128", alpha="fixed", alpha0=1e-8, inner="bicgstab", tau=ex["tau"],
                max_iter=40, inner_max_iter=30000)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), ref) < 1e-11, st
    # a few of the 387 systems per iteration may stop above tau (iteration
    # cap or stagnation); the outer iteration absorbs them
    assert max(st["inner_failed"]) <= 0.05 * 387, st["inner_failed"]


def test_config3_full_bicgstab_fp64_adaptive_alpha():
    """The same with Algorithm 2's adaptive alpha (capped at the
    correction-form optimum sqrt(L (3 eps + tau)) = 1.6e-3).  The shifted
    systems are harder there (condition numbers up to about 900 against 320
    at alpha = 1e-8) and a fifth of the inner solves stop above tau; the
    outer iteration still reaches the FP64 answer."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, u0, ex = workloads.config(3)
    ref = modal(prob, u0)
    plan = Plan(prob, precision="c128", alpha="paper", inner="bicgstab", tau=ex["tau"], max_iter=40,
                inner_max_iter=10000)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), ref) < 1e-11, st


@pytest.mark.parametrize("inner", ["bicgstab", "gmres"])
def test_config3_full_krylov_mixed(inner):
    """Mixed form (complex64 preconditioner, FP64 residual) with Krylov inner
    solves at tau = 1e-8 on this CFL-16 central advection, where the shifted
    systems reach condition numbers near 1e3.  Complex64 BiCGStab runs with
    FP64 reliable updates (true residual recomputed in FP64, FP64 solution
    accumulator); GMRES (the paper's inner solver) in complex64 honours a
    floored tau of 2^-20.  Both reach the oracle's solution to 1e-10."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, u0, ex = workloads.config(3)
    ref = modal(prob, u0)
    plan = Plan(prob, precision="c64", alpha="mixed", inner=inner, tau=ex["tau"], max_iter=60,
                inner_max_iter=10000)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), ref) < 1e-10, st
    assert st["res_rel"][-1] < 1e-9, st["res_rel"]


def test_config3_full_bicgstab_mixed_fails_loudly_when_inner_solves_are_cut_short():
    """Inner solves capped at 10 BiCGStab iterations cannot meet tau on this
    problem; the library must report that the outer iteration did not
    converge instead of returning an inaccurate answer."""
    torch = torch_cuda()
    from paper_2103_12571_gb300 import _lib
    from paper_2103_12571_gb300.api import Plan
    prob, u0, ex = workloads.config(3)
    plan = Plan(prob, precision="c64", alpha="mixed", inner="bicgstab", tau=ex["tau"], max_iter=12,
                inner_max_iter=10)
    with pytest.raises(_lib.ACError) as e:
        plan.solve(to_dev(torch, u0), tol=1e-10)
    assert e.value.code in (_lib.AC_ERR_NO_CONVERGENCE, _lib.AC_ERR_NOT_FINITE)


def test_config4_adjoint_gradients_full():
    """Loss J = |u_{L,M} - u_target|^2; gradients w.r.t. u0 and nu against the
    oracle's sequential discrete adjoint and against central differences of
    the GPU forward solve (h = 1e-6), to 1e-7 relative."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, u0, ex = workloads.config(4)
    target = ex["u_target"]
    Q, A, dT = oracle_setup(prob)
    plan = Plan(prob, precision="c128", alpha="paper", max_iter=40)
    u, _ = plan.solve(to_dev(torch, u0), tol=1e-15, raise_on_fail=False)
    un = u.cpu().numpy()
    g = np.zeros_like(un)
    g[-1, -1] = 2 * (un[-1, -1] - target)
    lam, st = plan.adjoint_solve(to_dev(torch, g), tol=1e-15, raise_on_fail=False)
    du0, dp = plan.grad_params(u, lam)
    du0 = du0.cpu().numpy()
    # oracle adjoint
    useq = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    gseq = np.zeros_like(useq)
    gseq[-1, -1] = 2 * (useq[-1, -1] - target)
    lseq = sequential.sequential_adjoint(A, Q, dT, gseq)
    du0_ref, dnu_ref, _ = sequential.grad_params(prob, Q, dT, useq, lseq)
    assert rel2(lam.cpu().numpy(), lseq) < 1e-7
    assert rel2(du0, du0_ref) < 1e-7
    assert abs(dp[0] - dnu_ref) < 1e-7 * abs(dnu_ref)

    def loss(p, v0):
        pl = Plan(p, precision="c128", alpha="paper", max_iter=40)
        uu, _ = pl.solve(to_dev(torch, v0), tol=1e-15, raise_on_fail=False)
        return float(((uu[-1, -1].cpu().numpy() - target) ** 2).sum())

    h = 1e-6
    pp, pm = dict(prob), dict(prob)
    pp["nu"] += h
    pm["nu"] -= h
    fd = (loss(pp, u0) - loss(pm, u0)) / (2 * h)
    assert abs(fd - dp[0]) < 1e-7 * abs(dp[0]), (fd, dp[0])
    rng = np.random.default_rng(7)
    for _ in range(2):
        v = workloads.smoothed_noise_2d(128, 128, 4.0, seed=int(rng.integers(1000)))
        fd = (loss(prob, u0 + h * v) - loss(prob, u0 - h * v)) / (2 * h)
        assert abs(fd - du0 @ v) < 1e-7 * abs(fd), (fd, du0 @ v)


def test_config5_full_field_mixed():
    """512 x 512 advection-diffusion, L = 512, mixed form: every one of the
    L * M = 1536 blocks (402.7 M values) against the closed form, streamed
    block by block."""
    torch = torch_cuda()
    from oracle import collocation
    from paper_2103_12571_gb300.api import Plan
    prob, u0, _ = workloads.config(5)
    L, M = prob["L"], prob["M"]
    plan = Plan(prob, precision="c64", alpha="mixed", max_iter=40)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    Q = collocation.collocation_matrix(collocation.radau_iia_nodes(M))
    num = den = 0.0
    blocks = 0
    for l, m, ref in fourier.modal_blocks(u0, prob, Q, prob["T"] / L, L):
        d = u[l, m].cpu().numpy() - ref
        num += float(d @ d)
        den += float(ref @ ref)
        blocks += 1
    assert blocks == L * M
    assert (num / den) ** 0.5 < 1e-10, ((num / den) ** 0.5, st)


def test_config5_gradients_against_closed_form():
    """Loss J = ||u_{L,M} - u_target||^2 on the full 512 x 512, L = 512
    workload, mixed form: the adjoint solve and the gradient contractions
    against the closed-form gradients w.r.t. u0, nu, cx and cy (the
    derivative of R(z)^L mode by mode), to 1e-7 relative."""
    torch = torch_cuda()
    from oracle import collocation
    from paper_2103_12571_gb300.api import Plan
    prob, u0, _ = workloads.config(5)
    L, M = prob["L"], prob["M"]
    target = workloads.random_phase_bumps_2d(512, 512, 8.0, seed=1)
    Q = collocation.collocation_matrix(collocation.radau_iia_nodes(M))
    J, du0_ref, dnu_ref, dc_ref = fourier.last_node_loss_gradients(u0, target, prob, Q, prob["T"] / L, L)
    plan = Plan(prob, precision="c64", alpha="mixed", max_iter=40)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    res = u[-1, -1] - to_dev(torch, target)
    assert abs(float((res * res).sum()) - J) < 1e-9 * J
    g = torch.zeros_like(u)
    g[-1, -1] = 2.0 * res
    lam, st2 = plan.adjoint_solve(g, tol=1e-13, raise_on_fail=False)
    del g
    du0, dp = plan.grad_params(u, lam)
    assert rel2(du0.cpu().numpy(), du0_ref) < 1e-7, st2
    scale = max(abs(dnu_ref), np.max(np.abs(dc_ref)))
    for got, ref in zip(dp, [dnu_ref, dc_ref[0], dc_ref[1]]):
        assert abs(got - ref) < 1e-7 * max(abs(ref), 1e-3 * scale), (dp, dnu_ref, dc_ref)
