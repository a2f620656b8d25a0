"""Sequential Radau IIA collocation stepping, its discrete adjoint and the
parameter gradients (THE oracle; test infrastructure only).

Forward (paper Sec. 2.1, eq. (seq_collocation_problem), with b = 0 and the
reading v_l, not v_{l-1}, on the right-hand side):
    C_coll u_1 = u_0 (x) 1_M + v_1,   C_coll u_l = H u_{l-1} + v_l,  l = 2..L.
C is block lower triangular with the nonsingular C_coll on its diagonal, so
this sweep is the unique solution of C u = w (eq. (globalsys)), which is the
fixed point every Richardson iteration (eq. (Riteration)) converges to.

Adjoint (derived from eq. (globalsys); the paper has no adjoint):
C^T = I_L (x) C_coll^T + E^T (x) H^T, block upper triangular, so
    C_coll^T lam_L = g_L,  C_coll^T lam_l = g_l + H^T lam_{l+1},  l = L-1..1,
with (H^T x)_m = delta_{mM} sum_j x_j.

Gradients of a scalar loss J(u) with C(theta) u = w(u_0) and g = dJ/du:
    dJ/du_0   = sum_m lam_{1,m}
    dJ/dtheta = lam^T (dw/dtheta - (dC/dtheta) u),  dC/dtheta = -dT I_L (x) Q (x) dA/dtheta
with dA/dnu = Lap, dA/dc_x = -D_x, dA/dc_y = -D_y.
"""
import numpy as np
import scipy.sparse.linalg as spla

from .operators import C_coll, operator_parts


def ordering(A):
    """Fill-reducing ordering for the LU of C_coll = I - dT Q (x) A (SuperLU's
    permc_spec).  C_coll has a symmetric sparsity pattern.  On 2D grids
    (A couples points more than the stencil radius apart, periodic wrap
    aside) minimum degree on A^T + A keeps the fill small (512^2, M = 3:
    202 s instead of 591 s to factor); on 1D rings it fills the factors badly
    (N = 4096, M = 3: 38 M entries instead of 0.37 M), and the column
    ordering is kept."""
    Ac = A.tocoo()
    n = A.shape[0]
    d = np.abs(Ac.row - Ac.col)
    d = np.minimum(d, n - d)
    return "MMD_AT_PLUS_A" if np.any(d > 3) else "COLAMD"


def factor(A, Q, dT, dtype=np.float64):
    """Sparse LU of C_coll = I - dT Q (x) A."""
    return spla.splu(C_coll(A, Q, dT).tocsc().astype(dtype), permc_spec=ordering(A))


class Stepper:
    """The forward sweep one step at a time: C_coll u_l = H u_{l-1} (+ v_l),
    with u_{-1} standing for u_0 (so the first right-hand side is u_0 stacked
    over the M nodes)."""

    def __init__(self, A, Q, dT, u0, dtype=np.float64):
        self.M, self.N = Q.shape[0], A.shape[0]
        self.lu = factor(A, Q, dT, dtype)
        self.last = np.asarray(u0, dtype=dtype)   # u_{l-1, M}, or u_0 before the first step
        self.dtype = dtype

    def step(self, v_l=None):
        rhs = np.tile(self.last, self.M)
        if v_l is not None:
            rhs = rhs + v_l.reshape(-1)
        u_l = self.lu.solve(rhs).reshape(self.M, self.N)
        self.last = u_l[self.M - 1]
        return u_l


def sequential_solve(A, Q, dT, L, u0, v=None):
    """u of shape (L, M, N): one sparse LU of C_coll, then L forward/back
    substitutions.  v (optional, shape (L, M, N)) is the forcing block v_l."""
    M, N = Q.shape[0], A.shape[0]
    dtype = np.result_type(np.asarray(u0).dtype, A.dtype, np.float64)
    st = Stepper(A, Q, dT, u0, dtype)
    u = np.empty((L, M, N), dtype=dtype)
    for l in range(L):
        u[l] = st.step(None if v is None else v[l])
    return u


def sequential_solve_general(A, Q, dT, w):
    """Solve C u = w for an arbitrary right-hand side w of shape (L, M, N)
    by the same forward sweep: C_coll u_l = w_l + H u_{l-1}."""
    L, M, N = w.shape
    dtype = np.result_type(w.dtype, A.dtype, np.float64)
    lu = factor(A, Q, dT, dtype)
    u = np.empty((L, M, N), dtype=dtype)
    for l in range(L):
        rhs = w[l].astype(dtype).copy()
        if l > 0:
            rhs += u[l - 1, M - 1][None, :]
        u[l] = lu.solve(rhs.reshape(-1)).reshape(M, N)
    return u


def sequential_adjoint(A, Q, dT, g):
    """lam = C^{-T} g by the backward sweep above; g of shape (L, M, N)."""
    L, M, N = g.shape
    dtype = np.result_type(g.dtype, A.dtype, np.float64)
    lu = factor(A, Q, dT, dtype)
    lam = np.empty((L, M, N), dtype=dtype)
    for l in range(L - 1, -1, -1):
        rhs = g[l].astype(dtype).copy()
        if l + 1 < L:
            rhs[M - 1] += lam[l + 1].sum(axis=0)
        lam[l] = lu.solve(rhs.reshape(-1), trans="T").reshape(M, N)
    return lam


def grad_params(prob, Q, dT, u, lam):
    """(dJ/du0, dJ/dnu, dJ/dc) for C u = w(u0) and lam = C^{-T} dJ/du.

    dJ/dtheta = dT sum_l sum_{m,j} Q_{mj} lam_{l,m}^T (dA/dtheta) u_{l,j}."""
    Lap, Dx, Dy = operator_parts(prob)
    L, M, N = u.shape
    du0 = lam[0].sum(axis=0)

    def contract(B):
        tot = 0.0
        for l in range(L):
            Bu = np.stack([B @ u[l, j] for j in range(M)])
            tot += np.sum(lam[l] * (Q @ Bu))
        return dT * tot

    dnu = contract(Lap)
    dcx = -contract(Dx)
    dcy = -contract(Dy) if Dy is not None else 0.0
    return du0, dnu, np.array([dcx, dcy])
