"""Pins of the CPU oracle against the paper, closed forms, textbook special
cases, invariants and brute force (CPU only)."""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from conftest import golden_path, read_golden
from oracle import alpha_rule, collocation, fourier, operators, paradiag, sequential, stencils
from paper_2103_12571_gb300 import workloads


def small_prob(dim=1, nx=8, ny=4, nu=0.3, cx=0.0, cy=0.0, order=2, M=2, L=4, T=0.2):
    return workloads.problem(dim, nx, ny, nu=nu, cx=cx, cy=cy, order=order, M=M, L=L, T=T)


def setup(prob):
    t = collocation.radau_iia_nodes(prob["M"])
    Q = collocation.collocation_matrix(t)
    A = operators.spatial_operator(prob)
    return t, Q, A, prob["T"] / prob["L"]


# ---------------------------------------------------------------- nodes / Q
def test_nodes_match_printed_node_polynomials():
    g = read_golden("radau_node_polynomials.txt")
    for M, key in ((2, "w2"), (3, "w3")):
        t = collocation.radau_iia_nodes(M)
        np.testing.assert_allclose(np.poly(t), g[key], rtol=0, atol=1e-14)
        assert t[-1] == 1.0
    np.testing.assert_allclose(collocation.radau_iia_nodes(3)[:2],
                               [(4 - math.sqrt(6)) / 10, (4 + math.sqrt(6)) / 10], atol=1e-15)
    assert collocation.radau_iia_nodes(1).tolist() == [1.0]


def test_Q_two_stage_is_textbook_radau_iia():
    g = read_golden("radau_iia_m2_butcher.txt")
    Q = collocation.collocation_matrix(collocation.radau_iia_nodes(2))
    np.testing.assert_allclose(Q, [g["row1"], g["row2"]], atol=1e-15)


def test_Q_three_stage_closed_form():
    # exact entries of the three-stage Radau IIA matrix
    s6 = math.sqrt(6)
    ref = np.array([[(88 - 7 * s6) / 360, (296 - 169 * s6) / 1800, (-2 + 3 * s6) / 225],
                    [(296 + 169 * s6) / 1800, (88 + 7 * s6) / 360, (-2 - 3 * s6) / 225],
                    [(16 - s6) / 36, (16 + s6) / 36, 1 / 9]])
    Q = collocation.collocation_matrix(collocation.radau_iia_nodes(3))
    np.testing.assert_allclose(Q, ref, atol=2e-15)


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5])
def test_Q_maps_monomials(M):
    # eq. (vandermonde): Q W = D_M W, W_{mk} = t_m^k; last row = quadrature
    # weights, exact for degree <= 2M - 2 (Radau)
    t = collocation.radau_iia_nodes(M)
    Q = collocation.collocation_matrix(t)
    W = np.vander(t, M, increasing=True)
    Wp = np.stack([t ** (k + 1) / (k + 1) for k in range(M)], axis=1)
    np.testing.assert_allclose(Q @ W, Wp, atol=1e-13)
    np.testing.assert_allclose(Q.sum(axis=1), t, atol=1e-14)
    for k in range(2 * M - 1):
        assert abs(Q[-1] @ t ** k - 1.0 / (k + 1)) < 1e-13


# ------------------------------------------------------- Lemma 2 / eq. (QGL)
def test_G_inverse_and_QH_identity():
    for M in (2, 3):
        t = collocation.radau_iia_nodes(M)
        Q = collocation.collocation_matrix(t)
        H = collocation.H_matrix(M)
        for d in (-0.3 + 0.2j, 0.7, -1e-3j):
            G = d * H + np.eye(M)
            np.testing.assert_allclose(np.linalg.inv(G), np.eye(M) - d / (1 + d) * H, atol=1e-14)
        np.testing.assert_allclose(Q @ H, np.diag(t) @ H, atol=1e-15)


@pytest.mark.parametrize("M", [2, 3, 4])
def test_lemma2_roots_are_eigenvalues(M):
    t = collocation.radau_iia_nodes(M)
    Q = collocation.collocation_matrix(t)
    rng = np.random.default_rng(M)
    for r in [0.0, 0.3, -0.2 + 0.1j] + list(rng.standard_normal(3) * 0.4 + 1j * rng.standard_normal(3) * 0.4):
        B = Q - r * np.diag(t) @ collocation.H_matrix(M)
        c = paradiag.lemma2_char_poly(t, r)
        roots = np.sort_complex(np.roots(c[::-1]))
        ev = np.sort_complex(np.linalg.eigvals(B))
        np.testing.assert_allclose(roots, ev, atol=1e-11)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_QGinv_is_Q_times_dense_inverse_of_G(M):
    # eq. (QGL): Q G_l^{-1} with G_l = I + d_l H_M (Lemma 1's eigenvalues d_l).
    # Pinned against a dense inverse of G_l and against Lemma 2's roots.
    t = collocation.radau_iia_nodes(M)
    Q = collocation.collocation_matrix(t)
    H = collocation.H_matrix(M)
    for L, alpha in ((8, 1e-3), (16, 0.3)):
        for d in paradiag.eigenvalues_d(L, alpha):
            B = paradiag.QGinv(Q, t, d)
            G = np.eye(M) + d * H
            np.testing.assert_allclose(B @ G, Q, atol=1e-14)
            np.testing.assert_allclose(B, Q @ np.linalg.inv(G), atol=1e-13)
            r = d / (1 + d)
            roots = list(np.roots(paradiag.lemma2_char_poly(t, r)[::-1]))
            for ev in np.linalg.eigvals(B):   # the same multiset
                j = int(np.argmin([abs(ev - z) for z in roots]))
                assert abs(ev - roots.pop(j)) < 1e-10


def test_lemma2_printed_sign_is_the_other_shift():
    # The lemma as printed (c_0 = (r+1) b_0, minus sign in c_m) gives the
    # spectrum of Q + r D_t H_M, i.e. eq. (QGL) with r -> -r.
    t = collocation.radau_iia_nodes(2)
    Q = collocation.collocation_matrix(t)
    r = 0.37
    printed = paradiag.lemma2_char_poly(t, -r)
    ev = np.sort_complex(np.linalg.eigvals(Q + r * np.diag(t) @ collocation.H_matrix(2)))
    np.testing.assert_allclose(np.sort_complex(np.roots(printed[::-1])), ev, atol=1e-12)


def test_M2_double_eigenvalue_where_discriminant_vanishes():
    # p_2 = 2 l^2 + (2r - 4/3) l + (1 - r)/3 has discriminant
    # proportional to 9 r^2 - 6 r - 2, zero at r = (1 +- sqrt 3)/3
    t = collocation.radau_iia_nodes(2)
    Q = collocation.collocation_matrix(t)
    for r in ((1 + math.sqrt(3)) / 3, (1 - math.sqrt(3)) / 3):
        c = paradiag.lemma2_char_poly(t, r)
        np.testing.assert_allclose(c, [(1 - r) / 3, 2 * r - 4 / 3, 2], atol=1e-15)
        ev = np.linalg.eigvals(Q - r * np.diag(t) @ collocation.H_matrix(2))
        assert abs(ev[0] - ev[1]) < 1e-6
    ev = np.linalg.eigvals(Q - 0.1 * np.diag(t) @ collocation.H_matrix(2))
    assert abs(ev[0] - ev[1]) > 1e-2


# ------------------------------------------------------------------ stencils
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("dim", [1, 2])
def test_stencil_symbol_is_eigenvalue(order, dim):
    prob = small_prob(dim=dim, nx=16, ny=8, nu=0.7, cx=1.3, cy=-0.4, order=order)
    A = operators.spatial_operator(prob)
    sig = fourier.symbol(prob)
    nx, ny = prob["nx"], prob["ny"]
    for (kx, ky) in [(0, 0), (1, 0), (3, 2), (nx - 1, ny // 2)]:
        if dim == 1:
            e = np.exp(2j * np.pi * kx * np.arange(nx) / nx)
            s = sig[kx]
        else:
            e = np.exp(2j * np.pi * (kx * np.arange(nx)[None, :] / nx + ky * np.arange(ny)[:, None] / ny)).reshape(-1)
            s = sig[ky, kx]
        np.testing.assert_allclose(A @ e, s * e, atol=1e-9 * max(1, abs(s)))


def _fd_table():
    rows = []
    with open(golden_path("fd_weights.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, deriv, order, lo, den, *nums = line.split()
            lo, den = int(lo), int(den)
            w = {lo + j: Fraction(int(v), den) for j, v in enumerate(nums) if int(v) != 0}
            rows.append((kind, int(deriv), int(order), w))
    return rows


def test_fd_weights_match_textbook_tables():
    rows = _fd_table()
    assert len(rows) == 11
    for kind, deriv, order, w in rows:
        if kind == "central":
            got = stencils.d1_weights(order) if deriv == 1 else stencils.d2_weights(order)
        else:
            got = stencils.d1_weights(order, upwind=True, c=1.0)
        assert got == w, (kind, deriv, order)


def _rate(op, f, df, ns=(64, 128)):
    errs = []
    for n in ns:
        x = np.arange(n) / n
        errs.append(np.max(np.abs(op(n) @ f(x) - df(x))))
    return math.log2(errs[0] / errs[1])


@pytest.mark.parametrize("order", [2, 4, 6])
def test_central_stencils_converge_at_their_order(order):
    f = lambda x: np.sin(2 * np.pi * x) + 0.3 * np.cos(6 * np.pi * x)
    df = lambda x: 2 * np.pi * np.cos(2 * np.pi * x) - 1.8 * np.pi * np.sin(6 * np.pi * x)
    d2f = lambda x: -4 * np.pi ** 2 * np.sin(2 * np.pi * x) - 10.8 * np.pi ** 2 * np.cos(6 * np.pi * x)
    ns = (32, 64)
    assert abs(_rate(lambda n: operators.first_derivative_1d(n, order=order), f, df, ns) - order) < 0.15
    assert abs(_rate(lambda n: operators.second_derivative_1d(n, order=order), f, d2f, ns) - order) < 0.15


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("c", [1.0, -0.5])
def test_upwind_stencils_converge_at_their_order(order, c):
    f = lambda x: np.sin(2 * np.pi * x) + 0.3 * np.cos(6 * np.pi * x)
    df = lambda x: 2 * np.pi * np.cos(2 * np.pi * x) - 1.8 * np.pi * np.sin(6 * np.pi * x)
    ns = (64, 128) if order < 4 else (32, 64)
    rate = _rate(lambda n: operators.first_derivative_1d(n, order=order, upwind=True, c=c), f, df, ns)
    assert abs(rate - order) < 0.2


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
def test_upwind_mirror_and_dissipation(order):
    """For c < 0 the stencil is the mirror image: D(c<0) = -D(c>0)^T.  The
    upwind operator A = -c D is dissipative for either sign: every
    eigenvalue has Re <= 0, with Re < 0 on all modes but k = 0."""
    n = 24
    Dp = operators.first_derivative_1d(n, order=order, upwind=True, c=1.0).toarray()
    Dm = operators.first_derivative_1d(n, order=order, upwind=True, c=-2.0).toarray()
    np.testing.assert_array_equal(Dm, -Dp.T)
    for c, D in ((1.0, Dp), (-2.0, Dm)):
        lam = np.linalg.eigvals(-c * D)
        assert np.all(lam.real <= 1e-10 * n)
        assert np.sum(lam.real > -1e-8) == 1
        # symbol = eigenvalues on the Fourier modes
        prob = dict(dim=1, nx=n, ny=1, nu=0.0, cx=c, cy=0.0, order=order, upwind=True)
        sig = fourier.symbol(prob)
        e = np.exp(2j * np.pi * 5 * np.arange(n) / n)
        np.testing.assert_allclose(-c * D @ e, sig[5] * e, atol=1e-10 * n)


def test_central_symbols_closed_forms():
    """Central symbols: i sin(t)/h, i (8 sin t - sin 2t)/(6h),
    i (45 sin t - 9 sin 2t + sin 3t)/(30h); (2 cos t - 2)/h^2,
    (-2 cos 2t + 32 cos t - 30)/(12 h^2),
    (4 cos 3t - 54 cos 2t + 540 cos t - 490)/(180 h^2), t = 2 pi k / n."""
    n, L = 40, 2.0
    h = L / n
    t = 2 * np.pi * np.arange(n) / n
    d1 = {2: 1j * np.sin(t) / h, 4: 1j * (8 * np.sin(t) - np.sin(2 * t)) / (6 * h),
          6: 1j * (45 * np.sin(t) - 9 * np.sin(2 * t) + np.sin(3 * t)) / (30 * h)}
    d2 = {2: (2 * np.cos(t) - 2) / h ** 2, 4: (-2 * np.cos(2 * t) + 32 * np.cos(t) - 30) / (12 * h ** 2),
          6: (4 * np.cos(3 * t) - 54 * np.cos(2 * t) + 540 * np.cos(t) - 490) / (180 * h ** 2)}
    for p in (2, 4, 6):
        np.testing.assert_allclose(fourier.symbol_d1(n, L, p), d1[p], atol=1e-12 / h)
        np.testing.assert_allclose(fourier.symbol_d2(n, L, p), d2[p], atol=1e-12 / h ** 2)


def test_upwind_problem_laplacian_order():
    # the Laplacian beside an order-p upwind derivative is centred of order p rounded up to even
    assert [stencils.laplacian_order(p, True) for p in (1, 2, 3, 4, 5)] == [2, 2, 4, 4, 6]
    with pytest.raises(ValueError):
        stencils.check_scheme(6, True)
    with pytest.raises(ValueError):
        stencils.check_scheme(3, False)


# ------------------------------------------------------ sequential = C^{-1} w
@pytest.mark.parametrize("M", [1, 2, 3])
@pytest.mark.parametrize("dim", [1, 2])
def test_sequential_equals_dense_allatonce_solve(M, dim):
    prob = small_prob(dim=dim, nx=6, ny=4, nu=0.5, cx=0.8, cy=0.3, M=M, L=5, T=0.3)
    t, Q, A, dT = setup(prob)
    rng = np.random.default_rng(1)
    N = operators.n_points(prob)
    u0 = rng.standard_normal(N)
    C = operators.allatonce_matrix(A, Q, dT, prob["L"]).toarray()
    w = operators.rhs_w(u0, prob["L"], M)
    dense = np.linalg.solve(C, w.reshape(-1)).reshape(w.shape)
    seq = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    np.testing.assert_allclose(seq, dense, atol=1e-13 * np.max(np.abs(dense)))
    # apply_C block form equals the Kronecker matrix
    np.testing.assert_allclose(operators.apply_C(seq, A, Q, dT).reshape(-1), C @ seq.reshape(-1), atol=1e-12)
    assert np.max(np.abs(operators.residual(seq, u0, A, Q, dT))) < 1e-13


def test_general_rhs_sweep_equals_dense():
    prob = small_prob(dim=1, nx=8, M=3, L=4)
    t, Q, A, dT = setup(prob)
    rng = np.random.default_rng(2)
    w = rng.standard_normal((4, 3, 8))
    C = operators.allatonce_matrix(A, Q, dT, 4).toarray()
    np.testing.assert_allclose(sequential.sequential_solve_general(A, Q, dT, w).reshape(-1),
                               np.linalg.solve(C, w.reshape(-1)), atol=1e-13)


def test_sequential_equals_fourier_closed_form_config1():
    prob, u0, _ = workloads.config(1)
    t, Q, A, dT = setup(prob)
    seq = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    modal = fourier.modal_solution(u0, prob, Q, dT, prob["L"])
    np.testing.assert_allclose(seq, modal, atol=1e-14)


def test_sequential_equals_fourier_closed_form_2d_advdiff():
    prob = small_prob(dim=2, nx=16, ny=8, nu=0.01, cx=1.0, cy=0.5, M=3, L=8, T=0.1)
    t, Q, A, dT = setup(prob)
    u0 = workloads.random_phase_bumps_2d(16, 8, 3.0, seed=3)
    seq = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    modal = fourier.modal_solution(u0, prob, Q, dT, prob["L"])
    np.testing.assert_allclose(seq, modal, atol=1e-13)
    sel = fourier.modal_solution(u0, prob, Q, dT, prob["L"], blocks=[(7, 2), (3, 0)])
    np.testing.assert_allclose(sel[(7, 2)], seq[7, 2], atol=1e-13)
    np.testing.assert_allclose(sel[(3, 0)], seq[3, 0], atol=1e-13)


@pytest.mark.parametrize("order", [1, 3, 5])
def test_sequential_equals_fourier_closed_form_upwind(order):
    """The oracle's two routes agree for upwind stencils (sparse matrix of the
    mirrored stencil for the negative velocity, and its symbol)."""
    prob = workloads.problem(2, 16, 12, nu=0.02, cx=0.8, cy=-0.6, order=order, M=3, L=6, T=0.1, upwind=True)
    t, Q, A, dT = setup(prob)
    u0 = workloads.random_phase_bumps_2d(16, 12, 3.0, seed=4)
    seq = sequential.sequential_solve(A, Q, dT, prob["L"], u0)
    np.testing.assert_allclose(seq, fourier.modal_solution(u0, prob, Q, dT, prob["L"]), atol=1e-13)


# --------------------------------------------- stability function and order
def test_modal_blocks_equal_modal_solution():
    prob = small_prob(dim=2, nx=8, ny=4, nu=0.3, cx=0.7, cy=-0.4, M=3, L=5, T=0.3)
    t, Q, A, dT = setup(prob)
    u0 = np.random.default_rng(4).standard_normal(32)
    full = fourier.modal_solution(u0, prob, Q, dT, 5)
    seen = 0
    for l, m, blk in fourier.modal_blocks(u0, prob, Q, dT, 5):
        np.testing.assert_allclose(blk, full[l, m], atol=1e-14)
        seen += 1
    assert seen == 15


@pytest.mark.parametrize("dim,order,upwind,cx,cy", [(1, 2, False, 0.8, 0.0), (2, 2, False, 1.0, 0.5),
                                                    (2, 4, False, -0.6, 0.3), (2, 3, True, 0.9, -0.7)])
def test_closed_form_loss_gradients_equal_sequential_adjoint(dim, order, upwind, cx, cy):
    """The closed-form gradients of J = ||u_{L,M} - target||^2 against the
    sequential discrete adjoint (sparse LU, backward sweep) and against
    central differences of the closed-form loss."""
    prob = workloads.problem(dim, 12, 8, nu=0.05, cx=cx, cy=cy, order=order, M=3, L=6, T=0.3, upwind=upwind)
    t, Q, A, dT = setup(prob)
    N = operators.n_points(prob)
    rng = np.random.default_rng(9)
    u0, target = rng.standard_normal(N), rng.standard_normal(N)
    J, du0, dnu, dc = fourier.last_node_loss_gradients(u0, target, prob, Q, dT, 6)
    u = sequential.sequential_solve(A, Q, dT, 6, u0)
    assert abs(J - np.sum((u[-1, -1] - target) ** 2)) < 1e-12 * J
    g = np.zeros_like(u)
    g[-1, -1] = 2 * (u[-1, -1] - target)
    lam = sequential.sequential_adjoint(A, Q, dT, g)
    du0_s, dnu_s, dc_s = sequential.grad_params(prob, Q, dT, u, lam)
    np.testing.assert_allclose(du0, du0_s, rtol=0, atol=1e-11 * np.max(np.abs(du0_s)))
    assert abs(dnu - dnu_s) < 1e-10 * max(1.0, abs(dnu_s))
    np.testing.assert_allclose(dc[: dim], dc_s[: dim], rtol=1e-10, atol=1e-12)
    h = 1e-6
    for key, val in (("nu", dnu), ("cx", dc[0])) + ((("cy", dc[1]),) if dim == 2 else ()):
        pp, pm = dict(prob), dict(prob)
        pp[key] += h
        pm[key] -= h
        Jp = fourier.last_node_loss_gradients(u0, target, pp, Q, dT, 6)[0]
        Jm = fourier.last_node_loss_gradients(u0, target, pm, Q, dT, 6)[0]
        assert abs((Jp - Jm) / (2 * h) - val) < 1e-6 * max(1.0, abs(val)), key


def test_stability_function_is_pade():
    z = np.array([-0.3, -5.0 + 2j, 0.2j, -40.0, -1e-3])
    Q2 = collocation.collocation_matrix(collocation.radau_iia_nodes(2))
    Q3 = collocation.collocation_matrix(collocation.radau_iia_nodes(3))
    R2 = (1 + z / 3) / (1 - 2 * z / 3 + z ** 2 / 6)
    R3 = (1 + 2 * z / 5 + z ** 2 / 20) / (1 - 3 * z / 5 + 3 * z ** 2 / 20 - z ** 3 / 60)
    np.testing.assert_allclose(fourier.stability_function(z, Q2), R2, rtol=1e-13)
    np.testing.assert_allclose(fourier.stability_function(z, Q3), R3, rtol=1e-13)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_convergence_order_2M_minus_1(M):
    # one Fourier mode of the semi-discrete heat equation decays like
    # exp(sigma t); the collocation error at T is O(dT^(2M-1))
    prob = small_prob(dim=1, nx=16, nu=0.05, M=M, L=4, T=1.0)
    k = 1
    sig = fourier.symbol(prob)[k].real
    Q = collocation.collocation_matrix(collocation.radau_iia_nodes(M))
    errs = []
    Ls = (4, 8, 16) if M < 3 else (2, 4, 8)
    for L in Ls:
        z = sig / L
        errs.append(abs(fourier.stability_function(np.array([z]), Q)[0].real ** L - math.exp(sig)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert abs(rates[-1] - (2 * M - 1)) < 0.35, rates
    # the same through the sequential solver on a grid mode
    A = operators.spatial_operator(prob)
    x = np.arange(16) / 16
    u0 = np.cos(2 * np.pi * k * x)
    uL = sequential.sequential_solve(A, Q, 1.0 / Ls[-1], Ls[-1], u0)[-1, -1]
    assert np.max(np.abs(uL - math.exp(sig) * u0)) < 1.5 * errs[-1]


# ------------------------------------------------------- Lemma 1 / C_alpha
def test_lemma1_diagonalises_E_alpha():
    for L, alpha in ((8, 1e-3), (5, 0.3), (16, 1e-6)):
        V, Vinv, d = paradiag.lemma1(L, alpha)
        E = operators.E_alpha(L, alpha).toarray()
        # round-off scales with ||V|| ||V^{-1}|| <= L / alpha (proof of Theorem 2)
        tol = 8 * L * 2.0 ** -52 * L / alpha
        np.testing.assert_allclose(V @ np.diag(d) @ Vinv, E, atol=tol)
        np.testing.assert_allclose(V @ Vinv, np.eye(L), atol=tol)
        # time_forward / time_inverse are V^{-1}, V
        rng = np.random.default_rng(L)
        r = rng.standard_normal((L, 3))
        np.testing.assert_allclose(paradiag.time_forward(r, alpha), Vinv @ r, atol=1e-12)
        np.testing.assert_allclose(paradiag.time_inverse(r, alpha), V @ r, atol=tol)


@pytest.mark.parametrize("dim,M", [(1, 2), (1, 3), (2, 3)])
def test_precond_solve_inverts_C_alpha(dim, M):
    prob = small_prob(dim=dim, nx=8, ny=4, nu=0.4, cx=0.7, cy=0.2, M=M, L=8, T=0.4)
    t, Q, A, dT = setup(prob)
    rng = np.random.default_rng(5)
    N = operators.n_points(prob)
    r = rng.standard_normal((8, M, N))
    for alpha in (1e-2, 1e-5):
        e = paradiag.precond_solve(A, Q, dT, alpha, r)
        assert np.max(np.abs(e.imag)) < 1e-9
        Ca = operators.allatonce_matrix(A, Q, dT, 8, alpha)
        np.testing.assert_allclose(Ca @ e.real.reshape(-1), r.reshape(-1), atol=1e-10)


# --------------------------------------------------- Richardson / Theorem 1
def test_richardson_contraction_is_exact_per_mode():
    prob = small_prob(dim=1, nx=8, nu=0.2, M=3, L=8, T=0.4)
    t, Q, A, dT = setup(prob)
    k = 2
    x = np.arange(8) / 8
    u0 = np.cos(2 * np.pi * k * x)
    ustar = sequential.sequential_solve(A, Q, dT, 8, u0)
    alpha = 0.05
    its = paradiag.richardson(A, Q, dT, 8, u0, [alpha] * 4)
    z = dT * fourier.symbol(prob)[k]
    fac = fourier.contraction_factor(np.array([z]), alpha, 8, Q)[0].real
    errs = [it[-1, -1] - ustar[-1, -1] for it in its]
    for a, b in zip(errs[:-1], errs[1:]):
        if np.max(np.abs(a)) > 1e-12:
            np.testing.assert_allclose(b, fac * a, atol=1e-14 + 1e-9 * np.max(np.abs(a)))
    assert abs(fac) <= alpha / (1 - alpha) + 1e-15
    # mean mode: R = 1, factor is exactly -alpha / (1 - alpha) (Theorem 1 bound attained)
    f0 = fourier.contraction_factor(np.array([0.0]), alpha, 8, Q)[0]
    assert abs(f0 + alpha / (1 - alpha)) < 1e-15


def test_richardson_forms_agree_and_converge():
    prob = small_prob(dim=2, nx=4, ny=4, nu=0.3, cx=0.5, M=2, L=4, T=0.2)
    t, Q, A, dT = setup(prob)
    u0 = np.random.default_rng(7).standard_normal(16)
    ustar = sequential.sequential_solve(A, Q, dT, 4, u0)
    a = paradiag.richardson(A, Q, dT, 4, u0, [1e-3] * 6, form="paper")
    b = paradiag.richardson(A, Q, dT, 4, u0, [1e-3] * 6, form="correction")
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, atol=1e-12)
    assert np.max(np.abs(a[-1] - ustar)) < 1e-13


# --------------------------------------------------------------- Algorithm 2
def test_alpha_sequence_reproduces_fig1():
    g = read_golden("fig1_alpha_sequence.txt")
    dT = g["T"][0] / g["L"][0]
    m0 = g["m0_over_dT"][0] * dT
    printed = g["alphas"]
    # gamma is not printed; fit it to the first value, then the recursion
    # must reproduce the other three to the printed digits
    gam = printed[0] ** 2 * m0
    alphas, ms = alpha_rule.alpha_sequence(m0, gam, kmax=4)
    for a, p in zip(alphas, printed):
        assert abs(a - p) / p < 0.5 * 10 ** -2 + 1e-3, (a, p)
    for k in range(5):
        assert abs(ms[k] - alpha_rule.m_closed_form(k, gam, m0)) <= 1e-12 * ms[k]
    assert all(a <= 0.5 for a in alphas) and alphas == sorted(alphas)


def test_alpha_sequence_limit():
    alphas, ms = alpha_rule.alpha_sequence(1.0, 1e-10, kmax=60)
    assert abs(ms[-1] - 4e-10) < 1e-15 and abs(alphas[-1] - 0.5) < 1e-9


@pytest.mark.parametrize("L", [8, 32])
@pytest.mark.parametrize("alpha", [0.5, 1e-2])
@pytest.mark.parametrize("tau", [1e-6, 1e-9])
@pytest.mark.parametrize("scale", [1.0, 1e3])
def test_gamma_is_theorem2_error_of_an_inexact_preconditioner(L, alpha, tau, scale):
    """gamma / alpha is Theorem 2's bound (eq. (errr1)) on the error one
    preconditioner application makes when every block solve of eq. (s2) is
    inexact with relative residual tau (kappa(B) ~ 1, ||r|| = ||w||).

    Scalar problem u' = lam u with dT lam = -1 (C_coll = 2, so
    ||B^{-1}||_inf <= 1), r = scale * (1, ..., 1).  The block residuals are
    given size tau ||x||_inf and phases that add up coherently in the last
    step: the measured error then lies between gamma / 3 (attained: the sum
    of the L frequency contributions, each at least tau ||x|| / (3 L) after
    the inverse transform, times alpha^{-(L-1)/L} ||x||_inf >= L) and
    ||B^{-1}|| gamma / alpha (the theorem).  A gamma without the factor L,
    without tau or without the norm of w fails one side."""
    Q = collocation.collocation_matrix(collocation.radau_iia_nodes(1))
    A = np.array([[-1.0]])
    import scipy.sparse as sp
    A = sp.csr_matrix(A)
    dT = 1.0
    r = scale * np.ones((L, 1, 1))
    x = paradiag.time_forward(r.astype(np.complex128), alpha)
    d = paradiag.eigenvalues_d(L, alpha)
    B = np.array([paradiag.block_matrix(A, Q, dT, dk).toarray()[0, 0] for dk in d])
    xinf = np.max(np.abs(x))
    # exact preconditioner and the inexact one (B_k (y_k + dy_k) = x_k + rho_k)
    g = np.exp(2j * np.pi * (L - 1) * np.arange(L) / L) / B
    rho = tau * xinf * np.conj(g) / np.abs(g)
    dy = (rho / B).reshape(L, 1, 1)
    du = paradiag.time_inverse(dy, alpha)
    err = np.max(np.abs(du))
    nB = np.max(1.0 / np.abs(B))
    kappa = np.max(np.abs(B)) * nB
    eps = 2.0 ** -53
    upper = nB / (1 - eps * kappa) * alpha_rule.gamma(L, eps * kappa, tau, scale) / alpha
    lower = alpha_rule.gamma(L, 0.0, tau, scale) / 3.0
    assert nB <= 1.0 + 1e-15
    assert lower <= err <= upper, (lower, err, upper)


def test_algorithm2_driver_stops_on_last_block_difference():
    prob = small_prob(dim=1, nx=8, nu=0.2, M=2, L=8, T=0.4)
    t, Q, A, dT = setup(prob)
    u0 = np.cos(2 * np.pi * np.arange(8) / 8)
    w_inf = np.max(np.abs(u0))
    gam = alpha_rule.gamma(8, 2.0 ** -53, 0.0, w_inf)

    def iterate(u, m, alpha):
        return paradiag.richardson(A, Q, dT, 8, u0, [alpha], u_init=u)[-1]

    u_init = np.broadcast_to(u0, (8, 2, 8)).copy()
    u, alphas, ms = alpha_rule.run_algorithm2(iterate, u_init, lambda v: v[-1], m0=dT * 8, gam=gam, tol=1e-12)
    ustar = sequential.sequential_solve(A, Q, dT, 8, u0)
    assert np.max(np.abs(u - ustar)) < 1e-11
    assert len(alphas) <= 6


# ------------------------------------------------------------------- adjoint
def test_apply_CT_is_transpose():
    prob = small_prob(dim=2, nx=4, ny=4, nu=0.3, cx=0.9, cy=-0.6, M=3, L=4, T=0.2)
    t, Q, A, dT = setup(prob)
    C = operators.allatonce_matrix(A, Q, dT, 4).toarray()
    lam = np.random.default_rng(3).standard_normal((4, 3, 16))
    np.testing.assert_allclose(operators.apply_CT(lam, A, Q, dT).reshape(-1), C.T @ lam.reshape(-1), atol=1e-12)


def test_sequential_adjoint_dot_product():
    prob = small_prob(dim=2, nx=8, ny=4, nu=0.3, cx=0.9, cy=-0.6, M=3, L=6, T=0.3)
    t, Q, A, dT = setup(prob)
    rng = np.random.default_rng(4)
    w = rng.standard_normal((6, 3, 32))
    g = rng.standard_normal((6, 3, 32))
    u = sequential.sequential_solve_general(A, Q, dT, w)
    lam = sequential.sequential_adjoint(A, Q, dT, g)
    assert abs(np.sum(u * g) - np.sum(w * lam)) < 1e-12 * np.sum(np.abs(u * g))
    C = operators.allatonce_matrix(A, Q, dT, 6).toarray()
    np.testing.assert_allclose(C.T @ lam.reshape(-1), g.reshape(-1), atol=1e-12)


def test_gradients_match_central_differences():
    base = small_prob(dim=2, nx=8, ny=8, nu=0.05, cx=1.0, cy=0.5, M=3, L=4, T=0.1)
    u0 = workloads.smoothed_noise_2d(8, 8, 1.0, seed=0)
    target = workloads.smoothed_noise_2d(8, 8, 1.0, seed=1)
    Q = collocation.collocation_matrix(collocation.radau_iia_nodes(3))
    dT = base["T"] / base["L"]

    def loss(p, v0):
        A = operators.spatial_operator(p)
        uL = sequential.sequential_solve(A, Q, dT, p["L"], v0)[-1, -1]
        return np.sum((uL - target) ** 2)

    A = operators.spatial_operator(base)
    u = sequential.sequential_solve(A, Q, dT, base["L"], u0)
    g = np.zeros_like(u)
    g[-1, -1] = 2 * (u[-1, -1] - target)
    lam = sequential.sequential_adjoint(A, Q, dT, g)
    du0, dnu, dc = sequential.grad_params(base, Q, dT, u, lam)
    h = 1e-6
    for key, val in (("nu", dnu), ("cx", dc[0]), ("cy", dc[1])):
        pp, pm = dict(base), dict(base)
        pp[key] += h
        pm[key] -= h
        fd = (loss(pp, u0) - loss(pm, u0)) / (2 * h)
        assert abs(fd - val) <= 1e-7 * max(1.0, abs(val)), (key, fd, val)
    rng = np.random.default_rng(9)
    for _ in range(3):
        v = rng.standard_normal(64)
        fd = (loss(base, u0 + h * v) - loss(base, u0 - h * v)) / (2 * h)
        assert abs(fd - du0 @ v) <= 1e-7 * max(1.0, abs(fd))


def test_workloads_deterministic_and_shaped():
    for i in (1, 3, 4):
        p, u0, ex = workloads.config(i)
        p2, u02, _ = workloads.config(i)
        assert u0.shape == (operators.n_points(p),)
        np.testing.assert_array_equal(u0, u02)
    u = workloads.random_phase_bumps_2d(32, 32, 4.0, seed=1)
    assert abs(np.max(np.abs(u)) - 1) < 1e-15


# ---------------------------------------------------- forcing (eq. (heat))
def _forced_mode_exact(lam, t, t0, g0):
    """g' = lam g + 8 pi^2 cos t - sin t, g(t0) = g0, in closed form."""
    a, b = 8 * np.pi ** 2, -1.0
    B = (a - lam * b) / (1 + lam ** 2)
    A = -lam * B - b
    gp = lambda s: A * np.cos(s) + B * np.sin(s)
    return gp(t) + (g0 - gp(t0)) * np.exp(lam * (t - t0))


def test_printed_heat_forcing_has_solution_cos_t():
    # u = cos(t) phi satisfies u_t = Lap u + (8 pi^2 cos t - sin t) phi exactly
    t = np.linspace(3.1, 3.5, 7)
    assert np.allclose(_forced_mode_exact(-8 * np.pi ** 2, t, np.pi, np.cos(np.pi)), np.cos(t), atol=1e-13)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_forced_collocation_converges_at_order_2M_minus_1(M):
    """Forcing enters as v_l = dT (Q (x) I) b_l with b sampled at T_l + dT t_m
    (eq. (collocation)); on one discrete Fourier mode the end-point error
    against the semi-discrete exact solution falls like dT^(2M-1)."""
    n = 16
    phi = workloads.heat_forcing_field(n)
    t = collocation.radau_iia_nodes(M)
    Q = collocation.collocation_matrix(t)
    errs = []
    Ls = (4, 8, 16) if M < 3 else (2, 4, 8)
    for L in Ls:
        prob = workloads.heat_forcing_problem(n, order=2, M=M, L=L, T=0.1)
        A = operators.spatial_operator(prob)
        dT = prob["T"] / L
        times = workloads.HEAT_T0 + dT * (np.arange(L)[:, None] + t[None, :])
        v = operators.collocation_rhs(workloads.heat_forcing_samples(n, times), Q, dT)
        u = sequential.sequential_solve(A, Q, dT, L, workloads.heat_forcing_u0(n), v)
        lam = fourier.symbol(prob)[1, 1].real
        g = _forced_mode_exact(lam, workloads.HEAT_T0 + prob["T"], workloads.HEAT_T0, -1.0)
        errs.append(np.max(np.abs(u[-1, -1] - g * phi)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert abs(rates[-1] - (2 * M - 1)) < 0.4, (rates, errs)


# --------------------------------------------- the paper's advection test
def _advection_error(N, order, M, L, T, dim=2):
    """max |u_L,M - u(T)| of the collocation stepping (Fourier closed form)
    for eq. (advection), u_t + u_x (+ u_y) = 0 with the upwind stencil, against
    its exact solution sin(2 pi (x - t)) (sin(2 pi (y - t)))."""
    prob = workloads.problem(dim, N, N, nu=0.0, cx=1.0, cy=1.0 if dim == 2 else 0.0, order=order,
                             M=M, L=L, T=T, upwind=True)
    Q = collocation.collocation_matrix(collocation.radau_iia_nodes(M))
    x = np.arange(N) / N
    if dim == 2:
        u0 = np.outer(np.sin(2 * np.pi * x), np.sin(2 * np.pi * x)).reshape(-1)
        ex = np.outer(np.sin(2 * np.pi * (x - T)), np.sin(2 * np.pi * (x - T))).reshape(-1)
    else:
        u0, ex = np.sin(2 * np.pi * x), np.sin(2 * np.pi * (x - T))
    u = fourier.modal_solution(u0, prob, Q, T / L, L, blocks=[(L - 1, M - 1)])[(L - 1, M - 1)]
    return np.max(np.abs(u - ex))


@pytest.mark.parametrize("tol,N,order,M,L", [(1e-5, 350, 2, 2, 8), (1e-9, 350, 4, 2, 16), (1e-12, 600, 5, 3, 32)])
def test_table1_advection_parameters_reach_their_tolerance(tol, N, order, M, L):
    """Table 1 (advection, T = 1e-2): with the chosen N, upwind order, M and L
    the sequential solution is within tol of the exact one.  A pin of the
    upwind reading: a wrong bias or order misses these tolerances."""
    err = _advection_error(N, order, M, L, 1e-2)
    assert err < tol
    assert err > tol / 1000      # the paper did not over-resolve (Sec. 5)


def test_fig1_advection_setup_reaches_1e_12():
    """Sec. 5.1 (Fig. 1): T = 0.0128, L = 64, M = 3, 5th-order upwind,
    N = 700, chosen so that the error is below 1e-12."""
    assert _advection_error(700, 5, 3, 64, 0.0128) < 1e-12
    # a 1st-order upwind stencil on the same grid misses it by far
    assert _advection_error(700, 1, 3, 64, 0.0128, dim=1) > 1e-6
