"""Exact spatial-FFT solves of eq. (d2) on grids whose sizes are not powers of
two (prime factors 2, 3, 5, 7: the paper's N = 700 of Fig. 1 and the 350 and
600 of Table 1), through the mixed-radix Stockham kernels, against the oracle:
C_alpha^{-1} r by Lemma 1 with sparse block solves, and whole Richardson
solves against sequential stepping.  The shapes include a ragged last row
tile and a ragged last column tile of the three-pass 2D solve, every radix
(2, 3, 4, 5, 7, 8) and lengths of a single stage."""
import numpy as np
import pytest

from gpu_common import oracle_setup, rel2, to_dev, torch_cuda
from oracle import operators, paradiag, sequential
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24

CASES = [
    workloads.problem(1, 700, cx=1.0, order=5, upwind=True, M=3, L=16, T=0.05),      # 7*5*5*4
    workloads.problem(1, 350, nu=0.05, order=2, M=2, L=8, T=0.1),                    # 7*5*5*2
    workloads.problem(1, 105, nu=0.01, cx=-0.5, order=4, M=4, L=4, T=0.05),          # 7*5*3
    workloads.problem(1, 6, nu=0.3, order=2, M=1, L=2, T=0.1),                       # 3*2
    workloads.problem(1, 7, nu=0.2, cx=0.3, order=2, M=2, L=4, T=0.1),               # one radix-7 stage
    workloads.problem(2, 45, 28, nu=0.02, cx=0.3, cy=-0.2, order=4, M=2, L=4, T=0.05),  # ragged column tile
    workloads.problem(2, 700, 49, nu=0.01, cx=1.0, cy=0.5, order=2, M=3, L=8, T=0.05),  # ragged row tile
    workloads.problem(2, 24, 40, nu=0.05, order=2, M=3, L=8, T=0.1),                 # 8*3 by 8*5
    workloads.problem(2, 600, 12, nu=0.01, cx=-1.0, cy=1.0, order=5, upwind=True, M=3, L=4, T=0.02),
]


def ids(p):
    return "d%d_%dx%d_o%d_M%d_L%d" % (p["dim"], p["nx"], p["ny"], p["order"], p["M"], p["L"])


@pytest.mark.parametrize("prob", CASES, ids=ids)
def test_mixed_radix_path_is_selected(prob):
    torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    for precision in ("c128", "c64"):
        info = Plan(prob, precision=precision).info()
        assert info["spatial_path"] == (5 if prob["dim"] == 1 else 6), info


@pytest.mark.parametrize("prob", CASES, ids=ids)
@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_precond_solve_mixed_radix(prob, precision):
    """e = C_alpha^{-1} r element by element against the oracle's Lemma-1
    route; tolerance from Theorem 2 (a modest multiple of L 3 eps / alpha)."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(21)
    r = rng.standard_normal((prob["L"], prob["M"], operators.n_points(prob)))
    plan = Plan(prob, precision=precision)
    eps = EPS64 if precision == "c128" else EPS32
    for alpha in (1e-2, 1e-4):
        e = plan.precond_solve(alpha, to_dev(torch, r)).cpu().numpy()
        ref = paradiag.precond_solve(A, Q, dT, alpha, r).real
        tol = 20 * prob["L"] * 3 * eps / alpha
        assert rel2(e, ref) < tol, (alpha, rel2(e, ref), tol)


@pytest.mark.parametrize("prob", [CASES[i] for i in (0, 2, 5, 6, 8)], ids=ids)
@pytest.mark.parametrize("precision,alpha_mode,tol", [("c128", "paper", 1e-11), ("c64", "mixed", 1e-10)])
def test_richardson_solve_mixed_radix(prob, precision, alpha_mode, tol):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(22)
    u0 = rng.standard_normal(operators.n_points(prob))
    ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    plan = Plan(prob, precision=precision, alpha=alpha_mode, max_iter=40)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-14 if precision == "c128" else 1e-13, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), ref) < tol, st


@pytest.mark.parametrize("prob", [CASES[i] for i in (2, 5)], ids=ids)
def test_mixed_radix_adjoint_and_gradients(prob):
    """The adjoint solve C^T lam = g (the transposed preconditioner: the same
    kernels on the mirrored symbols) and the parameter gradients."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(23)
    N = operators.n_points(prob)
    g = rng.standard_normal((prob["L"], prob["M"], N))
    lam_ref = sequential.sequential_adjoint(A, Q, dT, g)
    plan = Plan(prob, precision="c128", alpha="paper", max_iter=40)
    lam, st = plan.adjoint_solve(to_dev(torch, g), tol=1e-14, raise_on_fail=False)
    lam = lam.cpu().numpy()
    assert rel2(lam, lam_ref) < 1e-11, st
    u0 = rng.standard_normal(N)
    u = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    du0, dp = plan.grad_params(to_dev(torch, u), to_dev(torch, lam))
    du0_ref, dnu_ref, dc_ref = sequential.grad_params(prob, Q, dT, u, lam_ref)
    assert rel2(du0.cpu().numpy(), du0_ref) < 1e-9
    ref = np.array([dnu_ref, dc_ref[0], dc_ref[1]])
    assert np.max(np.abs(dp - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref))), (dp, ref)


def test_mixed_radix_sequential_stepping():
    """The same-GPU sequential baseline (one step after another, each an
    exact spatial solve per node) on a 700-point grid."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = CASES[0]
    Q, A, dT = oracle_setup(prob)
    u0 = np.sin(2 * np.pi * np.arange(700) / 700)
    ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    plan = Plan(prob, precision="c128")
    u = plan.sequential_solve(to_dev(torch, u0)).cpu().numpy()
    assert rel2(u, ref) < 1e-12
