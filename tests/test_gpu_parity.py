"""Parity of the CUDA path (through the C ABI) with the CPU oracle."""
import math

import numpy as np
import pytest

from gpu_common import oracle_setup, rel2, to_dev, torch_cuda
from oracle import fourier, operators, paradiag, sequential
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24

# small problems spanning several tiles, both dimensions, both orders, M = 1..4
SMALL = [
    workloads.problem(1, 64, nu=0.1, order=2, M=2, L=4, T=0.1),
    workloads.problem(1, 8, nu=0.3, cx=0.7, order=2, M=1, L=2, T=0.1),
    workloads.problem(1, 512, cx=1.0, order=4, M=3, L=16, T=0.25),
    workloads.problem(1, 256, nu=0.01, cx=-0.5, order=4, M=4, L=8, T=0.1),
    workloads.problem(2, 32, 16, nu=0.05, order=2, M=3, L=8, T=0.1),
    workloads.problem(2, 64, 64, nu=1e-3, cx=1.0, cy=0.5, order=2, M=3, L=32, T=0.25),
    workloads.problem(2, 16, 32, nu=0.02, cx=0.3, cy=-0.2, order=4, M=2, L=4, T=0.05),
    workloads.problem(2, 128, 256, nu=0.05, order=2, M=3, L=8, T=0.0625),   # three-pass 2D path
]


def ids(p):
    return "d%d_%dx%d_o%d_M%d_L%d" % (p["dim"], p["nx"], p["ny"], p["order"], p["M"], p["L"])


def rand_field(rng, prob):
    N = operators.n_points(prob)
    return rng.standard_normal((prob["L"], prob["M"], N))


@pytest.mark.parametrize("prob", SMALL, ids=ids)
def test_apply_C_and_CT(prob):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(0)
    u = rand_field(rng, prob)
    plan = Plan(prob)
    Cu = plan.apply_C(to_dev(torch, u)).cpu().numpy()
    ref = operators.apply_C(u, A, Q, dT)
    assert rel2(Cu, ref) < 1e-14
    CTu = plan.apply_CT(to_dev(torch, u)).cpu().numpy()
    assert rel2(CTu, operators.apply_CT(u, A, Q, dT)) < 1e-14


@pytest.mark.parametrize("prob", SMALL, ids=ids)
@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_precond_solve(prob, precision):
    """e = C_alpha^{-1} r against the oracle's Lemma-1 route with sparse block
    solves.  Tolerance from Theorem 2: the error is bounded by a modest
    multiple of L (3 eps + tau) / alpha relative to the data."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(1)
    r = rand_field(rng, prob)
    plan = Plan(prob, precision=precision)
    L = prob["L"]
    eps = EPS64 if precision == "c128" else EPS32
    for alpha in (1e-2, 1e-4):
        e = plan.precond_solve(alpha, to_dev(torch, r)).cpu().numpy()
        ref = paradiag.precond_solve(A, Q, dT, alpha, r).real
        tol = 20 * L * 3 * eps / alpha
        assert rel2(e, ref) < tol, (alpha, rel2(e, ref), tol)


@pytest.mark.parametrize("prob", SMALL, ids=ids)
@pytest.mark.parametrize("precision,alpha_mode,tol", [("c128", "paper", 1e-11), ("c64", "mixed", 1e-10)])
def test_richardson_solve_matches_sequential_oracle(prob, precision, alpha_mode, tol):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(2)
    N = operators.n_points(prob)
    u0 = rng.standard_normal(N)
    ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    plan = Plan(prob, precision=precision, alpha=alpha_mode, max_iter=40)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-14 if precision == "c128" else 1e-13, raise_on_fail=False)
    err = rel2(u.cpu().numpy(), ref)
    assert err < tol, (err, st)
    # the residual the library reports is the true one of the returned iterate,
    # up to the rounding noise of evaluating w - C u in FP64 (about
    # eps (1 + dT ||A||_inf) ||u|| / ||w|| per entry)
    uh = u.cpu().numpy()
    Cu = operators.apply_C(uh, A, Q, dT)
    w = operators.rhs_w(u0, prob["L"], prob["M"])
    floor = 64 * EPS64 * (1 + dT * abs(A).sum(axis=1).max()) * np.linalg.norm(uh) / np.linalg.norm(w)
    assert abs(np.linalg.norm(w - Cu) / np.linalg.norm(w) - st["res_rel"][-1]) < 1e-12 * st["res_rel"][-1] + floor


@pytest.mark.parametrize("prob", [SMALL[i] for i in (0, 2, 5, 7)], ids=ids)
@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_reported_residual_norm_is_fp64(prob, precision):
    """The residual norm the library reports (accumulated in FP64-accurate
    form from the residual kernel) equals ||w - C u||_2 / ||w||_2 of numpy to
    1e-12 relative, on iterates far from convergence, where the rounding
    floor of evaluating w - C u is negligible."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(6)
    N = operators.n_points(prob)
    L, M = prob["L"], prob["M"]
    u0 = rng.standard_normal(N)
    plan = Plan(prob, precision=precision)
    w = operators.rhs_w(u0, L, M)
    for scale in (1.0, 1e-6, 1e-9):
        # an iterate whose residual is `scale` times a random field
        ustar = sequential.sequential_solve(A, Q, dT, L, u0)
        un = ustar + scale * rng.standard_normal(ustar.shape)
        u = to_dev(torch, un)
        got = plan.richardson_step(1e-3, to_dev(torch, u0), u, want_residual=True)
        ref = np.linalg.norm(w - operators.apply_C(un, A, Q, dT)) / np.linalg.norm(w)
        floor = 64 * EPS64 * (1 + dT * abs(A).sum(axis=1).max()) * np.linalg.norm(un) / np.linalg.norm(w)
        assert abs(got - ref) < 1e-12 * ref + floor, (scale, got, ref, floor)


def test_config1_fixed_alpha_against_closed_form():
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob, u0, ex = workloads.config(1)
    Q, A, dT = oracle_setup(prob)
    ref = fourier.modal_solution(u0, prob, Q, dT, prob["L"])
    plan = Plan(prob, precision="c128", alpha="fixed", alpha0=ex["alpha"], max_iter=20)
    u, st = plan.solve(to_dev(torch, u0), tol=ex["tol"])
    assert st["converged"]
    assert rel2(u.cpu().numpy(), ref) < 1e-11
    # each iteration contracts the error by about alpha (Theorem 1)
    assert st["iters"] <= 5


def test_richardson_contraction_matches_closed_form_per_mode():
    """With one Fourier mode, each GPU iteration multiplies the last-node
    error by -alpha R^L / (1 - alpha R^L) (derived from eqs. (prec),
    (Riteration)); checked on the FP64 path."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(1, 32, nu=0.2, M=3, L=8, T=0.4)
    Q, A, dT = oracle_setup(prob)
    k = 3
    u0 = np.cos(2 * np.pi * k * np.arange(32) / 32)
    ustar = sequential.sequential_solve(A, Q, dT, 8, u0)
    alpha = 0.05
    plan = Plan(prob, precision="c128")
    u = to_dev(torch, np.broadcast_to(u0, (8, 3, 32)).copy())
    d0 = to_dev(torch, u0)
    errs = []
    for _ in range(5):
        errs.append(u.cpu().numpy()[-1, -1] - ustar[-1, -1])
        plan.richardson_step(alpha, d0, u)
    fac = fourier.contraction_factor(np.array([dT * fourier.symbol(prob)[k]]), alpha, 8, Q)[0].real
    for a, b in zip(errs[:-1], errs[1:]):
        if np.max(np.abs(a)) > 1e-10:
            np.testing.assert_allclose(b, fac * a, atol=1e-13 + 1e-8 * np.max(np.abs(a)))


def test_zero_rhs_gives_zero():
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(1, 64, nu=0.1, M=2, L=4, T=0.1)
    plan = Plan(prob)
    u, st = plan.solve(torch.zeros(64, dtype=torch.float64, device="cuda"), tol=1e-12)
    assert st["converged"] and float(u.abs().max()) == 0.0


@pytest.mark.parametrize("prob", [SMALL[2], SMALL[5], SMALL[6]], ids=ids)
@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_adjoint_and_gradients(prob, precision):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(3)
    N = operators.n_points(prob)
    g = rng.standard_normal((prob["L"], prob["M"], N))
    lam_ref = sequential.sequential_adjoint(A, Q, dT, g)
    plan = Plan(prob, precision=precision, alpha="paper" if precision == "c128" else "mixed", max_iter=40)
    lam, st = plan.adjoint_solve(to_dev(torch, g), tol=1e-14 if precision == "c128" else 1e-13,
                                 raise_on_fail=False)
    lam = lam.cpu().numpy()
    assert rel2(lam, lam_ref) < (1e-11 if precision == "c128" else 1e-10), st
    u0 = rng.standard_normal(N)
    u = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    du0, dp = plan.grad_params(to_dev(torch, u), to_dev(torch, lam))
    du0_ref, dnu_ref, dc_ref = sequential.grad_params(prob, Q, dT, u, lam_ref)
    assert rel2(du0.cpu().numpy(), du0_ref) < 1e-9
    ref = np.array([dnu_ref, dc_ref[0], dc_ref[1]])
    for i in range(3):
        assert abs(dp[i] - ref[i]) <= 1e-9 * max(1.0, np.max(np.abs(ref))), (i, dp, ref)


# ----------------------------------------------------------------- BiCGStab
# non-power-of-two grids give ragged last tiles in the time kernels
BICG = [
    workloads.problem(1, 300, cx=1.0, order=4, M=3, L=16, T=0.25),
    workloads.problem(1, 97, nu=0.05, cx=0.5, order=2, M=2, L=8, T=0.2),
    workloads.problem(2, 24, 20, nu=0.02, cx=0.4, cy=-0.3, order=2, M=3, L=8, T=0.1),
    workloads.problem(1, 4096, cx=1.0, order=4, M=3, L=8, T=1.0 / 32),   # vectors in global scratch for c128
]


@pytest.mark.parametrize("inner", ["bicgstab", "gmres"])
@pytest.mark.parametrize("prob", BICG, ids=ids)
@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_precond_solve_krylov(prob, precision, inner):
    """Inexact inner solves (BiCGStab, or GMRES as in the paper): the
    preconditioner error is bounded by a multiple of L (3 eps + tau) / alpha
    (Theorem 2)."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(4)
    r = rand_field(rng, prob)
    eps = EPS64 if precision == "c128" else EPS32
    tau = 1e-12 if precision == "c128" else 1e-6
    plan = Plan(prob, precision=precision, inner=inner, tau=tau)
    alpha = 1e-2
    e = plan.precond_solve(alpha, to_dev(torch, r)).cpu().numpy()
    ref = paradiag.precond_solve(A, Q, dT, alpha, r).real
    tol = 20 * prob["L"] * (3 * eps + tau) / alpha
    assert rel2(e, ref) < tol, (rel2(e, ref), tol)


@pytest.mark.parametrize("inner", ["bicgstab", "gmres"])
@pytest.mark.parametrize("prob", BICG[:3], ids=ids)
@pytest.mark.parametrize("precision,alpha_mode,tol,tau", [("c128", "paper", 1e-11, 1e-10), ("c64", "mixed", 1e-10, 1e-6)])
def test_richardson_solve_krylov(prob, precision, alpha_mode, tol, tau, inner):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(5)
    N = operators.n_points(prob)
    u0 = rng.standard_normal(N)
    ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    plan = Plan(prob, precision=precision, inner=inner, tau=tau, alpha=alpha_mode, max_iter=60)
    u, st = plan.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    err = rel2(u.cpu().numpy(), ref)
    assert err < tol, (err, st)
    assert all(v > 0 for v in st["inner_iters"]), st
    if precision == "c128":   # in complex64, systems stagnating at the FP32 floor are expected
        assert not any(st["inner_failed"]), st


@pytest.mark.parametrize("restart", [1, 4, 32])
def test_gmres_restart_lengths(restart):
    """GMRES(m) for m = 1 (a minimal-residual iteration), 4 and 32 (the
    largest): the preconditioner solve meets the Theorem 2 bound and the
    reported inner iteration counts are consistent with the restart length."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(2, 24, 20, nu=0.02, cx=0.4, cy=-0.3, order=4, M=3, L=8, T=0.05)
    Q, A, dT = oracle_setup(prob)
    r = rand_field(np.random.default_rng(14), prob)
    plan = Plan(prob, precision="c128", inner="gmres", tau=1e-12, inner_restart=restart)
    alpha = 1e-2
    e = plan.precond_solve(alpha, to_dev(torch, r)).cpu().numpy()
    ref = paradiag.precond_solve(A, Q, dT, alpha, r).real
    assert rel2(e, ref) < 20 * prob["L"] * (3 * EPS64 + 1e-12) / alpha
    u0 = np.random.default_rng(15).standard_normal(480)
    plan2 = Plan(prob, precision="c128", inner="gmres", tau=1e-12, inner_restart=restart, alpha="paper", max_iter=30)
    u, st = plan2.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), sequential.sequential_solve(A, Q, dT, 8, u0)) < 1e-11, st
    assert not any(st["inner_failed"]), st
    assert all(v > 0 for v in st["inner_iters"]), st


def test_unaligned_buffers_take_the_scalar_path():
    """A caller may pass buffers that are only 8-byte aligned (a view one
    double into a tensor); vector and asynchronous accesses are then off and
    the results must not change."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(2, 32, 16, nu=0.05, cx=0.3, order=2, M=3, L=8, T=0.1)
    N = 32 * 16
    rng = np.random.default_rng(12)
    u0 = to_dev(torch, rng.standard_normal(N))
    base = to_dev(torch, rng.standard_normal(8 * 3 * N))
    plan = Plan(prob, precision="c64")
    ua = base.clone().reshape(8, 3, N)
    big = torch.empty(8 * 3 * N + 1, dtype=torch.float64, device="cuda")
    ub = big[1:].view(8, 3, N)          # 8-byte aligned only
    ub.copy_(ua)
    for _ in range(2):
        plan.richardson_step(3e-3, u0, ua)
        plan.richardson_step(3e-3, u0, ub)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)


@pytest.mark.parametrize("prob", [workloads.problem(2, 256, 256, nu=0.05, order=2, M=3, L=64, T=0.5),
                                  workloads.problem(1, 1024, cx=1.0, order=4, M=3, L=128, T=0.5)],
                         ids=["heat2d_256_L64", "adv1d_1024_L128"])
def test_tma_staged_update_equals_plain_update(prob):
    """A complex64 plan built with update_kernel = AC_UPDATE_TMA updates
    u += e with the TMA-staged kernel (2D tensor tiles of X and u copied into
    shared memory, double-buffered) when u is 16-byte aligned, and with the
    plain kernel otherwise.  The arithmetic is the same, so the iterates must
    agree bit for bit with the plain plan's and with its own unaligned
    fallback.  The second case needs two boxes per tile for the rows of u
    (L*M = 384 > 256)."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    L, M = prob["L"], prob["M"]
    N = prob["nx"] * prob["ny"]
    rng = np.random.default_rng(13)
    u0 = to_dev(torch, rng.standard_normal(N))
    tma = Plan(prob, precision="c64", update_kernel="tma")
    plain = Plan(prob, precision="c64")
    assert tma.info()["update_kernel"] == 1 and tma.info()["update_tile_tma"] >= 8
    assert plain.info()["update_kernel"] == 0
    ua = to_dev(torch, rng.standard_normal((L, M, N)))
    uc = ua.clone()
    big = torch.empty(L * M * N + 1, dtype=torch.float64, device="cuda")
    ub = big[1:].view(L, M, N)          # 8-byte aligned only: the plain kernel
    ub.copy_(ua)
    for _ in range(3):
        ra = tma.richardson_step(2e-3, u0, ua, want_residual=True)
        rb = tma.richardson_step(2e-3, u0, ub, want_residual=True)
        rc = plain.richardson_step(2e-3, u0, uc, want_residual=True)
        assert ra == rb == rc
    torch.cuda.synchronize()
    assert torch.equal(ua, ub) and torch.equal(ua, uc)


def test_tma_staged_update_solve_matches_oracle():
    """A whole mixed-form solve with the TMA-staged update kernel against the
    sequential oracle (1e-10)."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = SMALL[5]
    Q, A, dT = oracle_setup(prob)
    u0 = np.random.default_rng(14).standard_normal(operators.n_points(prob))
    ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    plan = Plan(prob, precision="c64", alpha="mixed", max_iter=40, update_kernel="tma")
    assert plan.info()["update_kernel"] == 1
    u, st = plan.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    assert rel2(u.cpu().numpy(), ref) < 1e-10, st


# ------------------------------------------------- eq. (Riteration) as printed
@pytest.mark.parametrize("prob", [SMALL[0], SMALL[4], SMALL[6]], ids=ids)
def test_paper_form_iterates_match_oracle(prob):
    """AC_FORM_PAPER: u^{k+1} = C_alpha^{-1}(w - alpha H u_L^k e_1), compared
    iterate by iterate with the oracle's recompute-form Richardson."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(13)
    N = operators.n_points(prob)
    u0 = rng.standard_normal(N)
    alpha = 1e-3
    its = paradiag.richardson(A, Q, dT, prob["L"], u0, [alpha] * 3, form="paper")
    for k in (1, 2, 3):
        plan = Plan(prob, precision="c128", alpha="fixed", alpha0=alpha, max_iter=k, stop="paper", form="paper")
        u, st = plan.solve(to_dev(torch, u0), tol=0.0, raise_on_fail=False)
        assert st["iters"] == k
        err = rel2(u.cpu().numpy(), its[k])
        assert err < 20 * prob["L"] * 3 * EPS64 / alpha, (k, err)
        # the recorded last-step difference is the paper's stop quantity
        assert abs(st["diff_last"][-1] - np.max(np.abs(its[k][-1] - its[k - 1][-1]))) < 1e-6 * max(st["diff_last"][-1], 1e-30) + 1e-13


def test_paper_form_algorithm2_converges_and_follows_the_alpha_recursion():
    torch = torch_cuda()
    from oracle import alpha_rule
    from paper_2103_12571_gb300.api import Plan
    prob = SMALL[4]
    Q, A, dT = oracle_setup(prob)
    rng = np.random.default_rng(14)
    N = operators.n_points(prob)
    u0 = rng.standard_normal(N)
    ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    m0 = 0.5
    plan = Plan(prob, precision="c128", alpha="paper", m0=m0, max_iter=20, stop="paper", form="paper")
    u, st = plan.solve(to_dev(torch, u0), tol=1e-12, raise_on_fail=False)
    assert st["converged"], st
    assert rel2(u.cpu().numpy(), ref) < 1e-9
    gam = alpha_rule.gamma(prob["L"], EPS64, 0.0, np.max(np.abs(u0)))
    alphas, ms = alpha_rule.alpha_sequence(m0, gam, kmax=st["iters"])
    np.testing.assert_allclose(st["alpha"], alphas, rtol=1e-12)
    np.testing.assert_allclose(st["m"][:st["iters"]], ms[:st["iters"]], rtol=1e-12)
    assert 0 < st["res_rel"][-1] < 1e-9


def test_paper_form_in_complex64_stalls_where_the_correction_form_refines():
    """Without a residual the complex64 preconditioner's round-off stays in
    the answer (about L eps_32 / alpha); the correction form refines it away."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = SMALL[4]
    Q, A, dT = oracle_setup(prob)
    u0 = np.random.default_rng(15).standard_normal(operators.n_points(prob))
    ref = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    p1 = Plan(prob, precision="c64", alpha="fixed", alpha0=1e-2, max_iter=30, stop="paper", form="paper")
    u1, _ = p1.solve(to_dev(torch, u0), tol=1e-14, raise_on_fail=False)
    p2 = Plan(prob, precision="c64", alpha="mixed", max_iter=30)
    u2, _ = p2.solve(to_dev(torch, u0), tol=1e-13, raise_on_fail=False)
    e1, e2 = rel2(u1.cpu().numpy(), ref), rel2(u2.cpu().numpy(), ref)
    assert e1 > 1e-8 and e2 < 1e-10, (e1, e2)


def test_moving_window_equals_long_sequential_sweep():
    """Four windows of L = 8 steps cover the same 32 steps as one sequential
    sweep of the oracle (Sec. 5.2's moving window)."""
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    prob = workloads.problem(2, 32, 32, nu=0.02, cx=0.5, cy=0.25, order=2, M=3, L=8, T=0.05)
    Q, A, dT = oracle_setup(prob)
    u0 = workloads.random_phase_bumps_2d(32, 32, 4.0, seed=5)
    ref = sequential.sequential_solve(A, Q, dT, 4 * prob["L"], u0)[-1, -1]
    plan = Plan(prob, precision="c64", alpha="mixed", max_iter=30)
    u_end, iters, st = plan.window_solve(to_dev(torch, u0), 4, tol=1e-13)
    assert rel2(u_end.cpu().numpy(), ref) < 1e-10
    assert iters >= 4 and st["converged"]
