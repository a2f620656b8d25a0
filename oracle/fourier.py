"""Closed-form Fourier-mode solution of the collocation stepping (second,
independent oracle for periodic constant-coefficient A; test infrastructure
only).

On a periodic grid every stencil operator is diagonal in the discrete Fourier
basis: A e_k = sigma(k) e_k with e_k(x_j) = exp(2 pi i k j / n).  For one mode
with z = dT sigma(k), the stepping of eq. (seq_collocation_problem) reads
    (I - z Q) uhat_1 = uhat_0 1_M,   (I - z Q) uhat_l = uhat_{l-1,M} 1_M,
so with s(z) = (I - z Q)^{-1} 1_M and R(z) = s_M(z) (the stability function
of the collocation method),
    uhat_{l,m} = s_m(z) R(z)^{l-1} uhat_0,   l = 1..L.
"""
import numpy as np

from . import stencils


def taps_symbol(n, taps, scale):
    """Eigenvalues scale * sum_o w_o exp(2 pi i k o / n), k = 0..n-1, of the
    periodic stencil {o: w_o} (e_k(x_j) = exp(2 pi i k j / n))."""
    k = np.arange(n)
    s = np.zeros(n, dtype=np.complex128)
    for o, w in taps.items():
        s += float(w) * np.exp(2j * np.pi * ((k * o) % n) / n)
    return scale * s


def symbol_d1(n, length=1.0, order=2, upwind=False, c=1.0):
    """Eigenvalues of the periodic first derivative, mode k = 0..n-1."""
    return taps_symbol(n, stencils.d1_weights(order, upwind, c), n / length)


def symbol_d2(n, length=1.0, order=2, upwind=False):
    """Eigenvalues of the periodic second derivative."""
    return taps_symbol(n, stencils.d2_weights(order, upwind), (n / length) ** 2)


def symbol(prob):
    """sigma(k) for A = nu Lap - c . grad; shape (nx,) in 1D, (ny, nx) in 2D
    (matching numpy.fft.fft2 of a field stored as [iy, ix])."""
    nx, lx, order = prob["nx"], prob.get("lx", 1.0), prob["order"]
    up = bool(prob.get("upwind", False))
    cx, cy = prob.get("cx", 0.0), prob.get("cy", 0.0)
    sx = prob["nu"] * symbol_d2(nx, lx, order, up) - cx * symbol_d1(nx, lx, order, up, cx)
    if prob["dim"] == 1:
        return sx
    ny, ly = prob["ny"], prob.get("ly", 1.0)
    sy = prob["nu"] * symbol_d2(ny, ly, order, up) - cy * symbol_d1(ny, ly, order, up, cy)
    return sy[:, None] + sx[None, :]


def stage_vector(z, Q):
    """s(z) = (I - z Q)^{-1} 1_M for an array of z; shape z.shape + (M,)."""
    z = np.asarray(z, dtype=np.complex128)
    M = Q.shape[0]
    Az = np.eye(M) - z[..., None, None] * Q
    rhs = np.ones(z.shape + (M, 1), dtype=np.complex128)
    return np.linalg.solve(Az, rhs)[..., 0]


def stability_function(z, Q):
    """R(z) = e_M^T (I - z Q)^{-1} 1_M."""
    return stage_vector(z, Q)[..., -1]


def _fwd(u, prob):
    if prob["dim"] == 1:
        return np.fft.fft(u)
    return np.fft.fft2(u.reshape(prob["ny"], prob["nx"]))


def _inv(uh, prob):
    if prob["dim"] == 1:
        return np.fft.ifft(uh)
    return np.fft.ifft2(uh).reshape(-1)


def modal_solution(u0, prob, Q, dT, L, blocks=None):
    """u of shape (L, M, N) from uhat_{l,m} = s_m R^{l-1} uhat_0.

    ``blocks`` (optional list of (l, m) pairs, 0-based) restricts the output
    to those blocks: returns a dict {(l, m): u_lm}."""
    z = dT * symbol(prob)
    s = stage_vector(z, Q)
    R = s[..., -1]
    u0h = _fwd(np.asarray(u0, np.float64), prob)
    M = Q.shape[0]
    if blocks is not None:
        return {(l, m): _inv(s[..., m] * R ** l * u0h, prob).real for (l, m) in blocks}
    N = np.asarray(u0).shape[0]
    u = np.empty((L, M, N))
    for l in range(L):
        Rl = R ** l
        for m in range(M):
            u[l, m] = _inv(s[..., m] * Rl * u0h, prob).real
    return u


def contraction_factor(z, alpha, L, Q):
    """Per-mode error factor of one Richardson iteration with exact inner
    solves: -alpha R^L / (1 - alpha R^L).  Derived from eqs. (prec) and
    (Riteration): (C_alpha - C) e^k lives in block 1 only and equals
    -alpha H e^k_L, and C_alpha^{-1} of such a vector is computed mode by mode
    with the recursion above."""
    R = stability_function(z, Q)
    return -alpha * R ** L / (1.0 - alpha * R ** L)


def modal_blocks(u0, prob, Q, dT, L):
    """The closed form above one block at a time: yields (l, m, u_lm) for
    l = 0..L-1, m = 0..M-1 (0-based), keeping only R^l uhat_0 between
    blocks, so that full-size problems can be compared block by block."""
    z = dT * symbol(prob)
    s = stage_vector(z, Q)
    R = s[..., -1]
    uh = _fwd(np.asarray(u0, np.float64), prob)
    M = Q.shape[0]
    for l in range(L):
        for m in range(M):
            yield l, m, _inv(s[..., m] * uh, prob).real
        uh = uh * R


def _symbol_parts(prob):
    """(d sigma / d nu, d sigma / d cx, d sigma / d cy) on the fft layout of
    ``symbol``: sigma = nu Lap_hat - cx Dx_hat - cy Dy_hat (upwind
    derivatives biased by the sign of their own velocity component)."""
    nx, lx, order = prob["nx"], prob.get("lx", 1.0), prob["order"]
    up = bool(prob.get("upwind", False))
    cx, cy = prob.get("cx", 0.0), prob.get("cy", 0.0)
    lap_x = symbol_d2(nx, lx, order, up)
    d1x = symbol_d1(nx, lx, order, up, cx)
    if prob["dim"] == 1:
        return lap_x, -d1x, np.zeros_like(d1x)
    ny, ly = prob["ny"], prob.get("ly", 1.0)
    lap_y = symbol_d2(ny, ly, order, up)
    d1y = symbol_d1(ny, ly, order, up, cy)
    shape = (ny, nx)
    return (lap_y[:, None] + lap_x[None, :],
            np.broadcast_to(-d1x[None, :], shape), np.broadcast_to(-d1y[:, None], shape))


def last_node_loss_gradients(u0, target, prob, Q, dT, L):
    """J = ||u_{L,M} - target||_2^2 (last node of the last step) and its
    gradients (dJ/du0, dJ/dnu, dJ/dcx, dJ/dcy) from the closed form
        uhat_{L,M} = R(z)^L uhat_0,  z = dT sigma(k),
        dR/dz = e_M^T (I - z Q)^{-1} Q (I - z Q)^{-1} 1_M,
    with Parseval's identity for the numpy DFT (sum |x|^2 = sum |X|^2 / N).
    The derivative of J through the periodic, constant-coefficient
    collocation stepping, written mode by mode (an oracle independent of the
    sequential adjoint)."""
    u0 = np.asarray(u0, np.float64)
    N = u0.shape[0]
    z = dT * symbol(prob)
    s = stage_vector(z, Q)
    R = s[..., -1]
    M = Q.shape[0]
    Az = np.eye(M) - z[..., None, None] * Q
    dR = np.linalg.solve(Az, (Q @ s[..., None]))[..., -1, 0]
    u0h = _fwd(u0, prob)
    RL = R ** L
    uLh = RL * u0h
    uL = _inv(uLh, prob).real
    res = uL - np.asarray(target, np.float64)
    J = float(res @ res)
    resh = _fwd(res, prob)
    du0 = 2.0 * _inv(np.conj(RL) * resh, prob).real
    base = L * R ** (L - 1) * dR * dT * u0h
    grads = [float(2.0 / N * np.real(np.sum(np.conj(resh) * base * ds))) for ds in _symbol_parts(prob)]
    return J, du0, grads[0], np.array(grads[1:])
