"""The forced heat test of the paper (Sec. 5, eq. (heat)) on the GPU:
forcing assembled by ac_collocation_rhs, solved in the correction form
(FP64 and mixed) against the oracle's forced sequential stepping, and in the
paper's own form with Algorithm 2 over the tolerance ladder of Table 1."""
import numpy as np
import pytest

from gpu_common import oracle_setup, rel2, to_dev, torch_cuda
from oracle import collocation, operators, sequential
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu


def forced_case(n, order, M, L, T=0.1):
    prob = workloads.heat_forcing_problem(n, order=order, M=M, L=L, T=T)
    t = collocation.radau_iia_nodes(M)
    dT = T / L
    times = workloads.HEAT_T0 + dT * (np.arange(L)[:, None] + t[None, :])
    return prob, workloads.heat_forcing_samples(n, times), workloads.heat_forcing_u0(n)


def test_collocation_rhs_matches_oracle():
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, bn, u0 = forced_case(32, 2, 3, 8)
    Q, A, dT = oracle_setup(prob)
    plan = Plan(prob)
    v = plan.collocation_rhs(to_dev(torch, bn)).cpu().numpy()
    assert rel2(v, operators.collocation_rhs(bn, Q, dT)) < 1e-15


@pytest.mark.parametrize("precision,mode,tol", [("c128", "paper", 1e-11), ("c64", "mixed", 1e-10)])
def test_forced_solve_matches_sequential_oracle(precision, mode, tol):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, bn, u0 = forced_case(64, 4, 3, 16)
    Q, A, dT = oracle_setup(prob)
    v = operators.collocation_rhs(bn, Q, dT)
    ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0, v)
    plan = Plan(prob, precision=precision, alpha=mode, max_iter=40)
    vd = plan.collocation_rhs(to_dev(torch, bn))
    u, st = plan.solve(to_dev(torch, u0), tol=1e-13, b=vd, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), ref) < tol, st
    # against the exact PDE solution cos(t) phi at the final time: the error
    # is the spatial truncation of the 4th-order Laplacian on mode (1, 1),
    # |lambda_h + 8 pi^2| / (8 pi^2) ~ (2 pi h)^4 / 90 ~ 1e-6 at n = 64, plus a
    # much smaller dT^5 time error
    exact = np.cos(workloads.HEAT_T0 + prob["T"]) * workloads.heat_forcing_field(64)
    assert np.max(np.abs(u.cpu().numpy()[-1, -1] - exact)) < 3e-6


@pytest.mark.parametrize("tol,M,L,order", [(1e-5, 1, 32, 2), (1e-9, 2, 32, 4), (1e-12, 3, 16, 6)])
def test_paper_form_heat_ladder(tol, M, L, order):
    """Table 1's heat ladder (T = 0.1, centred orders 2/4/6): Algorithm 2 with the paper's
    stop test converges in a handful of iterations to the collocation
    solution."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, bn, u0 = forced_case(64, order, M, L)
    Q, A, dT = oracle_setup(prob)
    ref = sequential.sequential_solve(A, Q, dT, L, u0, operators.collocation_rhs(bn, Q, dT))
    plan = Plan(prob, precision="c128", alpha="paper", max_iter=20, stop="paper", form="paper")
    vd = plan.collocation_rhs(to_dev(torch, bn))
    u, st = plan.solve(to_dev(torch, u0), tol=tol, b=vd, raise_on_fail=False)
    assert st["converged"] and st["iters"] <= 10, st
    err = np.max(np.abs(u.cpu().numpy() - ref))
    assert err <= 10 * tol + 1e-12, (err, st)
