"""Edge cases of the CUDA path against the oracle: the largest L, M = 4 with
4th-order 2D stencils, non-unit box lengths, pure advection in 2D, M = 1
(implicit Euler) with the adjoint, and a singleton tile (N below the tile)."""
import numpy as np
import pytest

from gpu_common import oracle_setup, rel2, to_dev, torch_cuda
from oracle import operators, sequential
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

CASES = [
    (workloads.problem(1, 64, nu=0.05, order=2, M=2, L=1024, T=1.0), "c128", "paper", 1e-11),
    (workloads.problem(1, 64, nu=0.05, order=2, M=2, L=1024, T=1.0), "c64", "mixed", 1e-10),
    (workloads.problem(2, 32, 32, nu=0.01, cx=0.4, cy=-0.7, order=4, M=4, L=16, T=0.1), "c128", "paper", 1e-11),
    (workloads.problem(2, 64, 32, nu=0.0, cx=-1.0, cy=0.5, order=2, M=3, L=32, T=0.2), "c64", "mixed", 1e-10),
    (workloads.problem(1, 4, nu=0.2, order=2, M=1, L=2, T=0.1), "c128", "paper", 1e-11),
]


def ids(c):
    p, prec = c[0], c[1]
    return "d%d_%dx%d_o%d_M%d_L%d_%s" % (p["dim"], p["nx"], p["ny"], p["order"], p["M"], p["L"], prec)


@pytest.mark.parametrize("case", CASES, ids=ids)
def test_edge_solves(case):
    prob, precision, mode, tol = case
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    N = operators.n_points(prob)
    u0 = np.random.default_rng(21).standard_normal(N)
    ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    plan = Plan(prob, precision=precision, alpha=mode, max_iter=60)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-13 if precision == "c64" else 1e-14, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), ref) < tol, st


def test_box_lengths_scale_the_stencil():
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(2, 32, 16, nu=0.03, cx=0.5, cy=0.25, order=4, M=3, L=8, T=0.1)
    prob["lx"], prob["ly"] = 2.0, 0.5
    Q, A, dT = oracle_setup(prob)
    u0 = np.random.default_rng(22).standard_normal(512)
    ref = sequential.sequential_solve(A, Q, dT, 8, u0)
    u, st = Plan(prob, precision="c128", alpha="paper").solve(to_dev(torch, u0), tol=1e-14, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), ref) < 1e-11, st


def test_implicit_euler_adjoint():
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(2, 16, 16, nu=0.05, cx=0.3, order=2, M=1, L=8, T=0.1)
    Q, A, dT = oracle_setup(prob)
    g = np.random.default_rng(23).standard_normal((8, 1, 256))
    ref = sequential.sequential_adjoint(A, Q, dT, g)
    lam, st = Plan(prob, precision="c128", alpha="paper").adjoint_solve(to_dev(torch, g), tol=1e-14,
                                                                         raise_on_fail=False)
    assert rel2(lam.cpu().numpy(), ref) < 1e-11, st


def test_non_finite_right_hand_side_is_reported():
    """A NaN in u0 (or in the adjoint's g) makes ||w|| non-finite: the solves
    fail with AC_ERR_NOT_FINITE before iterating."""
    torch = torch_cuda()
    from paper_2103_12571_gb300 import _lib
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(1, 64, nu=0.1, order=2, M=2, L=4, T=0.1)
    plan = Plan(prob, precision="c64", alpha="mixed")
    u0 = to_dev(torch, np.random.default_rng(24).standard_normal(64))
    u0[5] = float("nan")
    for call in (lambda: plan.solve(u0, 1e-10), lambda: plan.krylov_solve(u0, 1e-10),
                 lambda: plan.adjoint_solve(u0.repeat(8).reshape(4, 2, 64).contiguous(), 1e-10)):
        with pytest.raises(_lib.ACError) as e:
            call()
        assert e.value.code == _lib.AC_ERR_NOT_FINITE
