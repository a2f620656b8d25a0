"""The single-pass 2D spatial solve over a thread-block cluster (each plane of
eq. (d2)'s shifted systems held in the shared memory of 4, 8 or 16 CTAs)
against the oracle's Lemma-1 route with sparse block solves, for every
cluster size that can hold the plane, in both precisions, and against the
three-pass solve."""
import numpy as np
import pytest

from gpu_common import oracle_setup, rel2, to_dev, torch_cuda
from oracle import operators, paradiag, sequential
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24

CASES = [
    workloads.problem(2, 128, 256, nu=0.05, order=2, M=3, L=8, T=0.0625),
    workloads.problem(2, 256, 256, nu=0.05, cx=0.5, cy=-0.25, order=4, M=2, L=4, T=0.05),
    workloads.problem(2, 512, 64, nu=0.01, cx=1.0, cy=0.5, order=2, M=3, L=4, T=0.05),
    workloads.problem(2, 64, 1024, nu=0.02, cx=-0.7, cy=0.3, order=5, upwind=True, M=2, L=2, T=0.02),
    workloads.problem(2, 512, 512, nu=1e-3, cx=1.0, cy=0.5, order=2, M=1, L=2, T=0.01),
]


def ids(p):
    return "%dx%d_o%d_M%d_L%d" % (p["nx"], p["ny"], p["order"], p["M"], p["L"])


def cluster_bytes(prob, cs, csize):
    nx, ny = prob["nx"], prob["ny"]
    if ny % cs or ny // cs < cs:
        return 0
    m = ny // cs
    return csize * (m * nx + nx + 2 * m)


@pytest.mark.parametrize("prob", CASES, ids=ids)
@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_cluster_solve_matches_oracle_and_three_passes(prob, precision):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    csize = 16 if precision == "c128" else 8
    sizes = [c for c in (4, 8, 16) if 0 < cluster_bytes(prob, c, csize) <= 200 * 1024]
    if not sizes:
        pytest.skip("no cluster of 4, 8 or 16 CTAs holds this plane")
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(31)
    r = rng.standard_normal((prob["L"], prob["M"], operators.n_points(prob)))
    alpha = 1e-3
    ref = paradiag.precond_solve(A, Q, dT, alpha, r).real
    three = Plan(prob, precision=precision, space_cluster=-1)
    assert three.info()["spatial_path"] == 2
    e3 = three.precond_solve(alpha, to_dev(torch, r)).cpu().numpy()
    eps = EPS64 if precision == "c128" else EPS32
    tol = 20 * prob["L"] * 3 * eps / alpha
    for cs in sizes:
        plan = Plan(prob, precision=precision, space_cluster=cs)
        info = plan.info()
        assert info["spatial_path"] == 7 and info["space_cluster"] == cs, info
        e = plan.precond_solve(alpha, to_dev(torch, r)).cpu().numpy()
        assert rel2(e, ref) < tol, (cs, rel2(e, ref), tol)
        # the same transforms in another order: rounding-level differences only
        assert rel2(e, e3) < (1e-13 if precision == "c128" else 2e-5), (cs, rel2(e, e3))


def test_three_passes_stay_the_default():
    torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    info = Plan(CASES[1], precision="c64").info()
    assert info["spatial_path"] == 2 and info["space_cluster"] == 0, info
    info = Plan(CASES[1], precision="c64", space_cluster=8).info()
    assert info["spatial_path"] == 7 and info["space_cluster"] == 8, info


def test_cluster_request_that_cannot_hold_a_plane_is_rejected():
    torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    with pytest.raises(RuntimeError):
        Plan(CASES[2], precision="c64", space_cluster=16)   # 64 rows over 16 CTAs: 4 < 16


@pytest.mark.parametrize("precision,alpha_mode,tol", [("c128", "paper", 1e-11), ("c64", "mixed", 1e-10)])
def test_richardson_solve_with_cluster_solves(precision, alpha_mode, tol):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = CASES[1]
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(32)
    u0 = rng.standard_normal(operators.n_points(prob))
    ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    plan = Plan(prob, precision=precision, alpha=alpha_mode, max_iter=40, space_cluster=8)
    assert plan.info()["spatial_path"] == 7
    u, st = plan.solve(to_dev(torch, u0), tol=1e-14 if precision == "c128" else 1e-13, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), ref) < tol, st
