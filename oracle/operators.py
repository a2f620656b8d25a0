"""Spatial operator A and the all-at-once matrices (oracle; test
infrastructure only).

Problem (paper Sec. 2, eq. (genericlinearform)) with b = 0:  u_t = A u.
A = nu * Laplacian_h - c . grad_h on a periodic grid.  The stencils are the
finite-difference formulas of `stencils.py`: centred of order 2, 4 or 6, or,
with prob["upwind"], an upwind first derivative of order 1..5 (biased
against the sign of each velocity component) with the centred Laplacian of
the order rounded up to even.  h = length / n per axis and, in 2D, the flat
index n = iy * nx + ix.

C_coll = I_{MN} - dT Q (x) A and H = H_M (x) I_N (Sec. 2.1);
C = I_L (x) C_coll + E (x) H (eq. (globalsys)), E = -1 on the sub-diagonal;
C_alpha = I_L (x) C_coll + E_alpha (x) H (eq. (prec)), E_alpha = E with -alpha
in the top-right corner.
"""
import numpy as np
import scipy.sparse as sp

from . import stencils
from .collocation import H_matrix

def _periodic(n, taps, scale):
    """Sparse n x n periodic matrix with (Au)_j = scale * sum_o taps[o] u_{j+o}."""
    rows, cols, vals = [], [], []
    j = np.arange(n)
    acc = {}
    for o, w in taps.items():
        for jj in j:
            key = (jj, (jj + o) % n)
            acc[key] = acc.get(key, 0.0) + w * scale
    for (r, c), v in acc.items():
        rows.append(r)
        cols.append(c)
        vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def first_derivative_1d(n, length=1.0, order=2, upwind=False, c=1.0):
    h = length / n
    taps = {o: float(w) for o, w in stencils.d1_weights(order, upwind, c).items()}
    return _periodic(n, taps, 1.0 / h)


def second_derivative_1d(n, length=1.0, order=2, upwind=False):
    h = length / n
    taps = {o: float(w) for o, w in stencils.d2_weights(order, upwind).items()}
    return _periodic(n, taps, 1.0 / (h * h))


def operator_parts(prob):
    """(Lap, Dx, Dy) sparse matrices for a problem dict
    {dim, nx, ny, lx, ly, nu, cx, cy, order[, upwind]}.  Dy is None in 1D.
    With upwind stencils Dx and Dy depend on the signs of cx and cy."""
    dim, order = prob["dim"], prob["order"]
    up = bool(prob.get("upwind", False))
    stencils.check_scheme(order, up)
    nx, lx = prob["nx"], prob.get("lx", 1.0)
    cx, cy = prob.get("cx", 0.0), prob.get("cy", 0.0)
    if dim == 1:
        return (second_derivative_1d(nx, lx, order, up),
                first_derivative_1d(nx, lx, order, up, cx), None)
    ny, ly = prob["ny"], prob.get("ly", 1.0)
    Ix, Iy = sp.identity(nx, format="csr"), sp.identity(ny, format="csr")
    Lap = sp.kron(Iy, second_derivative_1d(nx, lx, order, up)) + \
        sp.kron(second_derivative_1d(ny, ly, order, up), Ix)
    Dx = sp.kron(Iy, first_derivative_1d(nx, lx, order, up, cx))
    Dy = sp.kron(first_derivative_1d(ny, ly, order, up, cy), Ix)
    return Lap.tocsr(), Dx.tocsr(), Dy.tocsr()


def spatial_operator(prob):
    """A = nu Lap - cx Dx - cy Dy (sparse CSR, float64)."""
    Lap, Dx, Dy = operator_parts(prob)
    A = prob["nu"] * Lap - prob.get("cx", 0.0) * Dx
    if Dy is not None:
        A = A - prob.get("cy", 0.0) * Dy
    return A.tocsr()


def n_points(prob):
    return prob["nx"] * (prob["ny"] if prob["dim"] == 2 else 1)


def C_coll(A, Q, dT):
    """C_coll = I_{MN} - dT Q (x) A (Sec. 2.1)."""
    M, N = Q.shape[0], A.shape[0]
    return (sp.identity(M * N, format="csr") - dT * sp.kron(Q, A)).tocsr()


def H_full(M, N):
    """H = H_M (x) I_N."""
    return sp.kron(H_matrix(M), sp.identity(N)).tocsr()


def E_alpha(L, alpha):
    """E_alpha of eq. (prec); alpha = 0 gives E of eq. (globalsys)."""
    E = sp.lil_matrix((L, L))
    for l in range(1, L):
        E[l, l - 1] = -1.0
    if L > 0 and alpha != 0.0:
        E[0, L - 1] += -alpha
    return E.tocsr()


def allatonce_matrix(A, Q, dT, L, alpha=0.0):
    """C (alpha = 0, eq. (globalsys)) or C_alpha (eq. (prec)) as sparse."""
    M, N = Q.shape[0], A.shape[0]
    return (sp.kron(sp.identity(L), C_coll(A, Q, dT)) +
            sp.kron(E_alpha(L, alpha), H_full(M, N))).tocsr()


def rhs_w(u0, L, M, b=None):
    """w = (u_0 + v_1, v_2, ..., v_L) with u_0 stacked over the M nodes
    (eq. (globalsys)); b, if given, is a full (L, M, N) array added to it."""
    u0 = np.asarray(u0)
    N = u0.shape[0]
    w = np.zeros((L, M, N), dtype=np.result_type(u0, np.float64))
    w[0, :, :] = u0[None, :]
    if b is not None:
        w = w + b
    return w


def apply_C(u, A, Q, dT):
    """(C u)_l = C_coll u_l - H u_{l-1}, u of shape (L, M, N) (eq. (globalsys)).

    Written block by block: (C_coll u_l)_m = u_{l,m} - dT sum_j Q_{mj} A u_{l,j}
    and (H u_{l-1})_m = u_{l-1,M}."""
    L, M, N = u.shape
    out = np.empty_like(u)
    for l in range(L):
        Au = np.stack([A @ u[l, j] for j in range(M)])
        out[l] = u[l] - dT * (Q @ Au)
        if l > 0:
            out[l] += -u[l - 1, M - 1][None, :]
    return out


def apply_CT(lam, A, Q, dT):
    """(C^T lam)_l = C_coll^T lam_l - H^T lam_{l+1}.

    C_coll^T = I - dT Q^T (x) A^T; (H^T x)_m = delta_{mM} sum_j x_j."""
    L, M, N = lam.shape
    AT = A.T.tocsr()
    out = np.empty_like(lam)
    for l in range(L):
        ATl = np.stack([AT @ lam[l, j] for j in range(M)])
        out[l] = lam[l] - dT * (Q.T @ ATl)
        if l + 1 < L:
            out[l, M - 1] += -lam[l + 1].sum(axis=0)
    return out


def residual(u, u0, A, Q, dT, b=None):
    """r = w - C u."""
    L, M, N = u.shape
    return rhs_w(u0, L, M, b) - apply_C(u, A, Q, dT)


def collocation_rhs(bnodes, Q, dT):
    """v_l = dT (Q (x) I_N) b_l for forcing samples bnodes[l][m][n] at the
    collocation nodes T_l + dT t_m of step l (eq. (collocation), Sec. 2.1)."""
    return dT * np.einsum("mj,ljn->lmn", Q, bnodes)
