"""The sequential baseline (Sec. 4.2, T_Mpar): L collocation steps one after
another, each by diagonalisation of Q, against the oracle's sequential
stepping with direct sparse solves."""
import numpy as np
import pytest

from gpu_common import oracle_setup, rel2, to_dev, torch_cuda
from oracle import operators, sequential
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

CASES = [
    (workloads.problem(1, 64, nu=0.1, order=2, M=2, L=4, T=0.1), "fft"),
    (workloads.problem(1, 512, cx=1.0, order=4, M=3, L=16, T=0.25), "fft"),
    (workloads.problem(2, 32, 16, nu=0.05, cx=0.2, order=6, M=3, L=8, T=0.1), "fft"),
    (workloads.problem(2, 128, 256, nu=0.05, order=2, M=3, L=8, T=0.0625), "fft"),    # three-pass 2D path
    (workloads.problem(1, 4, nu=0.2, order=2, M=1, L=2, T=0.1), "fft"),
    (workloads.problem(1, 300, cx=1.0, order=5, upwind=True, M=3, L=16, T=0.05), "gmres"),
    (workloads.problem(2, 24, 20, nu=0.02, cx=0.4, cy=-0.3, order=3, upwind=True, M=4, L=8, T=0.1), "bicgstab"),
]


def ids(c):
    p = c[0]
    return "d%d_%dx%d_o%d%s_M%d_L%d_%s" % (p["dim"], p["nx"], p["ny"], p["order"], "u" if p.get("upwind") else "",
                                          p["M"], p["L"], c[1])


@pytest.mark.parametrize("case", CASES, ids=ids)
def test_sequential_stepping_matches_oracle(case):
    prob, inner = case
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    N, L, M = operators.n_points(prob), prob["L"], prob["M"]
    rng = np.random.default_rng(31)
    u0 = rng.standard_normal(N)
    plan = Plan(prob, precision="c128", inner=inner, tau=1e-14)
    u = plan.sequential_solve(to_dev(torch, u0)).cpu().numpy()
    assert rel2(u, sequential.sequential_solve(A, Q, dT, L, u0)) < 1e-11
    # forced: v = dT (Q x I) b at the nodes
    bn = rng.standard_normal((L, M, N))
    v = operators.collocation_rhs(bn, Q, dT)
    uf = plan.sequential_solve(to_dev(torch, u0), b=to_dev(torch, v)).cpu().numpy()
    assert rel2(uf, sequential.sequential_solve(A, Q, dT, L, u0, v)) < 1e-11


def test_sequential_graph_replay_and_recapture():
    """Replays with the same buffers reuse the captured graph; new buffers
    re-capture it; the results are identical bit for bit."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(2, 64, 64, nu=0.02, cx=0.5, cy=0.25, order=4, M=3, L=16, T=0.1)
    plan = Plan(prob, precision="c128")
    u0 = to_dev(torch, np.random.default_rng(32).standard_normal(64 * 64))
    out1 = plan.sequential_solve(u0)
    first = out1.clone()
    for _ in range(3):
        plan.sequential_solve(u0, out=out1)
    out2 = plan.sequential_solve(u0.clone())
    torch.cuda.synchronize()
    assert torch.equal(out1, first) and torch.equal(out2, first)


def test_sequential_complex64_rounding():
    """In a complex64 plan the step solves carry complex64 rounding (no
    refinement): the error is at the FP32 level, far above FP64's."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(2, 64, 64, nu=0.05, order=2, M=3, L=16, T=0.1)
    Q, A, dT = oracle_setup(prob)
    u0 = np.random.default_rng(33).standard_normal(64 * 64)
    u = Plan(prob, precision="c64").sequential_solve(to_dev(torch, u0)).cpu().numpy()
    err = rel2(u, sequential.sequential_solve(A, Q, dT, 16, u0))
    assert 1e-9 < err < 1e-5
