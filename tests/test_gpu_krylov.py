"""Outer Krylov acceleration: flexible GMRES on C u = w right-preconditioned
by C_alpha^{-1} (the coupling Sec. 6 names as future work), against the
sequential oracle."""
import numpy as np
import pytest

from gpu_common import oracle_setup, rel2, to_dev, torch_cuda
from oracle import operators, sequential
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

CASES = [
    workloads.problem(1, 64, nu=0.1, order=2, M=2, L=4, T=0.1),
    workloads.problem(2, 32, 16, nu=0.05, cx=0.3, order=4, M=3, L=8, T=0.1),
    workloads.problem(1, 300, cx=1.0, order=5, upwind=True, M=3, L=16, T=0.05),
]


def ids(p):
    return "d%d_%dx%d_o%d_M%d_L%d" % (p["dim"], p["nx"], p["ny"], p["order"], p["M"], p["L"])


@pytest.mark.parametrize("prob", CASES, ids=ids)
@pytest.mark.parametrize("precision,tol", [("c128", 1e-11), ("c64", 1e-10)])
def test_krylov_solve_matches_oracle(prob, precision, tol):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    N, L, M = operators.n_points(prob), prob["L"], prob["M"]
    rng = np.random.default_rng(41)
    u0 = rng.standard_normal(N)
    inner = "gmres" if prob.get("upwind") else "fft"
    plan = Plan(prob, precision=precision, inner=inner, tau=1e-13 if precision == "c128" else 0.0, max_iter=60)
    u, st = plan.krylov_solve(to_dev(torch, u0), 1e-13, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), sequential.sequential_solve(A, Q, dT, L, u0)) < tol, st
    # forced
    v = operators.collocation_rhs(rng.standard_normal((L, M, N)), Q, dT)
    uf, st = plan.krylov_solve(to_dev(torch, u0), 1e-13, b=to_dev(torch, v), raise_on_fail=False)
    assert rel2(uf.cpu().numpy(), sequential.sequential_solve(A, Q, dT, L, u0, v)) < tol, st


def test_krylov_converges_where_richardson_cannot():
    """alpha = 0.9: Richardson's error factor on a mode, -alpha R^L / (1 -
    alpha R^L), exceeds 1 in modulus for R^L > 0.56 (the slow heat modes;
    here R^L = 0.67 on |k| = 1), so it diverges; the spectrum of
    C C_alpha^{-1}, 1 / (1 - alpha R^L), lies in [1, 10] for heat, where
    GMRES converges."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(2, 32, 32, nu=0.05, order=2, M=3, L=16, T=0.2)
    Q, A, dT = oracle_setup(prob)
    u0 = np.random.default_rng(42).standard_normal(1024) + 0.5
    ref = sequential.sequential_solve(A, Q, dT, 16, u0)
    plan = Plan(prob, precision="c128", alpha="fixed", alpha0=0.9, max_iter=40)
    _, st_r = plan.solve(to_dev(torch, u0), 1e-10, raise_on_fail=False)
    assert not st_r["converged"]
    u, st = plan.krylov_solve(to_dev(torch, u0), 1e-12, restart=20)
    assert st["converged"] and st["iters"] <= 40, st
    assert rel2(u.cpu().numpy(), ref) < 1e-10


def test_krylov_cap_and_zero_rhs():
    """The step cap ends the solve with AC_ERR_NO_CONVERGENCE (u holds the
    last iterate, stats its history); a zero right-hand side returns u = 0."""
    torch = torch_cuda()
    from paper_2103_12571_gb300 import _lib
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(1, 64, nu=0.1, order=2, M=2, L=8, T=0.1)
    plan = Plan(prob, precision="c128", max_iter=3)
    u0 = to_dev(torch, np.random.default_rng(43).standard_normal(64))
    u, st = plan.krylov_solve(u0, 1e-30, restart=2, raise_on_fail=False)
    assert st["iters"] == 3 and not st["converged"]
    assert st["res_rel"][3] < st["res_rel"][0]
    with pytest.raises(_lib.ACError) as e:
        plan.krylov_solve(u0, 1e-30, restart=2)
    assert e.value.code == _lib.AC_ERR_NO_CONVERGENCE
    z, st = plan.krylov_solve(torch.zeros_like(u0), 1e-12)
    assert st["converged"] and float(z.abs().max()) == 0.0
