"""Parity of the CUDA path with the oracle for every stencil scheme: centred
orders 2, 4, 6 and upwind orders 1..5 (Sec. 5, Tables 1-2), including the
adjoint and the gradients, Krylov inner solves (GMRES, BiCGStab) on
non-power-of-two grids,
and the paper's advection test (eq. (advection)) with Table 1's parameters
and the setup of Fig. 1."""
import numpy as np
import pytest

from gpu_common import oracle_setup, rel2, to_dev, torch_cuda
from oracle import fourier, operators, paradiag, sequential
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53
SCHEMES = [(p, False) for p in (2, 4, 6)] + [(p, True) for p in (1, 2, 3, 4, 5)]


def sid(s):
    return ("up%d" if s[1] else "c%d") % s[0]


def cases(order, upwind):
    # velocities of both signs on each axis; several tiles and a ragged 2D tile
    return [workloads.problem(1, 64, nu=0.02, cx=-0.8, order=order, upwind=upwind, M=3, L=8, T=0.1),
            workloads.problem(2, 32, 16, nu=0.01, cx=0.6, cy=-0.9, order=order, upwind=upwind, M=2, L=4, T=0.05)]


@pytest.mark.parametrize("scheme", SCHEMES, ids=sid)
def test_apply_C_CT_and_precond_every_scheme(scheme):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    for prob in cases(*scheme):
        Q, A, dT = oracle_setup(prob)
        rng = np.random.default_rng(4)
        u = rng.standard_normal((prob["L"], prob["M"], operators.n_points(prob)))
        plan = Plan(prob, precision="c128")
        ud = to_dev(torch, u)
        assert rel2(plan.apply_C(ud).cpu().numpy(), operators.apply_C(u, A, Q, dT)) < 1e-14
        assert rel2(plan.apply_CT(ud).cpu().numpy(), operators.apply_CT(u, A, Q, dT)) < 1e-14
        alpha = 1e-3
        e = plan.precond_solve(alpha, ud).cpu().numpy()
        ref = paradiag.precond_solve(A, Q, dT, alpha, u).real
        assert rel2(e, ref) < 20 * prob["L"] * 3 * EPS64 / alpha


@pytest.mark.parametrize("scheme", SCHEMES, ids=sid)
@pytest.mark.parametrize("precision,alpha_mode,tol", [("c128", "paper", 1e-11), ("c64", "mixed", 1e-10)])
def test_solve_every_scheme(scheme, precision, alpha_mode, tol):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    for prob in cases(*scheme):
        Q, A, dT = oracle_setup(prob)
        u0 = np.random.default_rng(5).standard_normal(operators.n_points(prob))
        ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
        plan = Plan(prob, precision=precision, alpha=alpha_mode, max_iter=40)
        u, st = plan.solve(to_dev(torch, u0), tol=1e-14 if precision == "c128" else 1e-13, raise_on_fail=False)
        assert rel2(u.cpu().numpy(), ref) < tol, (prob, st)


@pytest.mark.parametrize("scheme", [(6, False), (3, True), (5, True)], ids=sid)
def test_adjoint_and_gradients_new_schemes(scheme):
    """The adjoint reverses the taps (A^T of an upwind stencil is the
    downwind one); the gradient w.r.t. c uses the upwind derivative of the
    velocity's sign."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    for prob in cases(*scheme):
        Q, A, dT = oracle_setup(prob)
        rng = np.random.default_rng(6)
        N = operators.n_points(prob)
        g = rng.standard_normal((prob["L"], prob["M"], N))
        lam_ref = sequential.sequential_adjoint(A, Q, dT, g)
        plan = Plan(prob, precision="c128", alpha="paper", max_iter=40)
        lam, st = plan.adjoint_solve(to_dev(torch, g), tol=1e-14, raise_on_fail=False)
        lam = lam.cpu().numpy()
        assert rel2(lam, lam_ref) < 1e-11, st
        u = sequential.sequential_solve(A, Q, dT, prob["L"], rng.standard_normal(N))
        du0, dp = plan.grad_params(to_dev(torch, u), to_dev(torch, lam))
        du0_ref, dnu_ref, dc_ref = sequential.grad_params(prob, Q, dT, u, lam_ref)
        assert rel2(du0.cpu().numpy(), du0_ref) < 1e-9
        ref = np.array([dnu_ref, dc_ref[0], dc_ref[1]])
        assert np.max(np.abs(np.asarray(dp) - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref))), (dp, ref)


def _advection(dim, N, order, M, L, T):
    prob = workloads.problem(dim, N, N, nu=0.0, cx=1.0, cy=1.0 if dim == 2 else 0.0, order=order,
                             M=M, L=L, T=T, upwind=True)
    x = np.arange(N) / N
    if dim == 2:
        u0 = np.outer(np.sin(2 * np.pi * x), np.sin(2 * np.pi * x)).reshape(-1)
        exact = np.outer(np.sin(2 * np.pi * (x - T)), np.sin(2 * np.pi * (x - T))).reshape(-1)
    else:
        u0, exact = np.sin(2 * np.pi * x), np.sin(2 * np.pi * (x - T))
    return prob, u0, exact


@pytest.mark.parametrize("inner", ["gmres", "bicgstab", "fft"])
def test_fig1_advection_setup_1d(inner):
    """Fig. 1's discretisation (T = 0.0128, L = 64, M = 3, 5th-order upwind,
    N = 700) in 1D, with Krylov inner solves on the upwind stencil (GMRES at
    tau = 1e-15 as in the paper, BiCGStab) and with the exact mixed-radix FFT
    solve (700 = 7 * 5 * 5 * 4): the whole space-time solution against the
    sequential oracle and the last step against the exact solution."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, u0, exact = _advection(1, 700, 5, 3, 64, 0.0128)
    Q, A, dT = oracle_setup(prob)
    ref = sequential.sequential_solve(A, Q, dT, 64, u0)
    plan = Plan(prob, precision="c128", inner=inner, tau=1e-15, alpha="paper", max_iter=30)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-14, raise_on_fail=False)
    u = u.cpu().numpy()
    assert rel2(u, ref) < 1e-11, st
    assert np.max(np.abs(u[-1, -1] - exact)) < 1e-12


@pytest.mark.parametrize("inner", ["gmres", "bicgstab", "fft"])
def test_fig1_advection_setup_2d(inner):
    """Fig. 1's setup in 2D, as the paper runs it: eq. (advection)
    u_t + u_x + u_y = 0 on the periodic unit square with N = 700^2 points,
    5th-order upwind stencils, L = 64, M = 3, T = 0.0128, Krylov inner solves
    at tau = 1e-15 (GMRES, the paper's, and BiCGStab) or the exact
    mixed-radix FFT solve.  All 192 blocks of the space-time solution against the Fourier
    closed form, the last step against the exact solution at 1e-12."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    L, M = 64, 3
    prob, u0, exact = _advection(2, 700, 5, M, L, 0.0128)
    Q, A, dT = oracle_setup(prob)
    plan = Plan(prob, precision="c128", inner=inner, tau=1e-15, alpha="paper", max_iter=30)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-14, raise_on_fail=False)
    num = den = 0.0
    for l, m, ref in fourier.modal_blocks(u0, prob, Q, dT, L):
        d = u[l, m].cpu().numpy() - ref
        num += float(d @ d)
        den += float(ref @ ref)
    assert (num / den) ** 0.5 < 1e-11, ((num / den) ** 0.5, st)
    assert np.max(np.abs(u[-1, -1].cpu().numpy() - exact)) < 1e-12, st


@pytest.mark.parametrize("inner", ["gmres", "bicgstab", "fft"])
@pytest.mark.parametrize("tol,N,order,M,L,tau", [(1e-5, 350, 2, 2, 8, 1e-8), (1e-9, 350, 4, 2, 16, 1e-11),
                                                 (1e-12, 600, 5, 3, 32, 1e-14)])
def test_paper_advection_table1(tol, N, order, M, L, tau, inner):
    """Table 1's advection ladder (2D, T = 1e-2, N x N points, upwind of
    order kappa, GMRES (the paper's) or BiCGStab inner solves at the
    table's tau, or exact mixed-radix FFT solves): the paper's form of the iteration with Algorithm 2 and its
    last-step stop test.  The
    result is checked against the Fourier closed form of the collocation
    solution and against the exact solution at tol."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    T = 1e-2
    prob, u0, exact = _advection(2, N, order, M, L, T)
    Q, A, dT = oracle_setup(prob)
    ref = fourier.modal_solution(u0, prob, Q, dT, L, blocks=[(L - 1, M - 1)])[(L - 1, M - 1)]
    plan = Plan(prob, precision="c128", inner=inner, tau=tau, alpha="paper", max_iter=20,
                stop="paper", form="paper")
    u, st = plan.solve(to_dev(torch, u0), tol=tol, raise_on_fail=False)
    assert st["converged"] and st["iters"] <= 12, st
    uL = u[-1, -1].cpu().numpy()
    assert np.max(np.abs(uL - ref)) <= tol, st
    assert np.max(np.abs(uL - exact)) <= 2 * tol, st
