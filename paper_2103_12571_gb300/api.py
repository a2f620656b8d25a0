"""Python front end of the GB300 alpha-circulant Richardson solver.

``Plan`` wraps an ``ac_plan`` of the C ABI (include/alphacirc.h).  Tensors are
torch CUDA float64 tensors in the layout u[l][m][n]; torch provides device
memory and the current stream, the library does all the arithmetic.
``RichardsonSolve`` is a torch.autograd.Function whose backward runs the
hand-written adjoint solve and gradient contractions.
"""
import ctypes

import numpy as np
import torch

from . import _lib as C


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t):
    if t is None:
        return None
    if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CPU tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_problem(prob):
    return C.Problem(dim=int(prob["dim"]), nx=int(prob["nx"]), ny=int(prob.get("ny", 1)),
                     lx=float(prob.get("lx", 1.0)), ly=float(prob.get("ly", 1.0)),
                     nu=float(prob.get("nu", 0.0)), cx=float(prob.get("cx", 0.0)),
                     cy=float(prob.get("cy", 0.0)), order=int(prob.get("order", 2)),
                     upwind=int(bool(prob.get("upwind", False))))


PRECISION = {"c128": C.AC_C128, "fp64": C.AC_C128, "c64": C.AC_C64, "mixed": C.AC_C64}
INNER = {"fft": C.AC_INNER_FFT, "bicgstab": C.AC_INNER_BICGSTAB, "gmres": C.AC_INNER_GMRES}
ALPHA = {"fixed": C.AC_ALPHA_FIXED, "paper": C.AC_ALPHA_PAPER, "mixed": C.AC_ALPHA_MIXED}
STOP = {"residual": C.AC_STOP_RESIDUAL, "paper": C.AC_STOP_PAPER}
FORM = {"correction": C.AC_FORM_CORRECTION, "paper": C.AC_FORM_PAPER}
UPDATE = {"plain": C.AC_UPDATE_PLAIN, "tma": C.AC_UPDATE_TMA}


def stats_dict(st):
    k = st.iters
    return dict(iters=k, converged=bool(st.converged), res_rel=list(st.res_rel[:k + 1]),
                alpha=list(st.alpha[:k]), m=list(st.m[:k + 1]), diff_last=list(st.diff_last[:k]),
                inner_iters=list(st.inner_iters[:k]), inner_failed=list(st.inner_failed[:k]),
                w_norm2=st.w_norm2, w_inf=st.w_inf)


class Plan:
    """Plan for a problem dict (see ``workloads.problem``) with M nodes, L steps."""

    def __init__(self, prob, M=None, L=None, dT=None, precision="c128", inner="fft", alpha="paper",
                 alpha0=1e-4, m0=0.0, tau=0.0, max_iter=50, stop="residual", inner_max_iter=0,
                 form="correction", inner_restart=0, update_kernel="plain", space_cluster=0):
        M = int(M if M is not None else prob["M"])
        L = int(L if L is not None else prob["L"])
        dT = float(dT if dT is not None else prob["T"] / L)
        self.M, self.L, self.dT = M, L, dT
        self.N = int(prob["nx"]) * (int(prob.get("ny", 1)) if int(prob["dim"]) == 2 else 1)
        self.prob = dict(prob)
        sched = C.Schedule(mode=ALPHA[alpha], alpha0=float(alpha0), m0=float(m0), tau=float(tau),
                           max_iter=int(max_iter), stop_rule=STOP[stop], inner_max_iter=int(inner_max_iter),
                           form=FORM[form], inner_restart=int(inner_restart),
                           update_kernel=UPDATE[update_kernel], space_cluster=int(space_cluster))
        handle = ctypes.c_void_p()
        C.check(C.lib().ac_setup(ctypes.byref(make_problem(prob)), M, L, dT, ctypes.byref(sched),
                                 PRECISION[precision], INNER[inner], ctypes.byref(handle)), "ac_setup")
        self._h = handle

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            C.lib().ac_destroy(h)
            self._h = None

    def params(self):
        """[nu, cx, cy] of the plan's spatial operator (cy = 0 in 1D)."""
        p = self.prob
        return [float(p.get("nu", 0.0)), float(p.get("cx", 0.0)),
                float(p.get("cy", 0.0)) if int(p["dim"]) == 2 else 0.0]

    @property
    def shape(self):
        return (self.L, self.M, self.N)

    def info(self):
        i = C.PlanInfo()
        C.check(C.lib().ac_plan_get_info(self._h, ctypes.byref(i)), "ac_plan_get_info")
        return {f: getattr(i, f) for f, _ in C.PlanInfo._fields_}

    def empty(self):
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    def apply_C(self, u, out=None):
        out = self.empty() if out is None else out
        C.check(C.lib().ac_apply_C(self._h, _ptr(u), _ptr(out), _stream()), "ac_apply_C")
        return out

    def apply_CT(self, lam, out=None):
        out = self.empty() if out is None else out
        C.check(C.lib().ac_apply_CT(self._h, _ptr(lam), _ptr(out), _stream()), "ac_apply_CT")
        return out

    def collocation_rhs(self, bnodes, out=None):
        """v_l = dT (Q (x) I) b_l from forcing samples at the collocation nodes."""
        out = self.empty() if out is None else out
        C.check(C.lib().ac_collocation_rhs(self._h, _ptr(bnodes), _ptr(out), _stream()), "ac_collocation_rhs")
        return out

    def nodes(self):
        return radau_nodes(self.M)

    def precond_solve(self, alpha, r, out=None):
        out = self.empty() if out is None else out
        C.check(C.lib().ac_precond_solve(self._h, float(alpha), _ptr(r), _ptr(out), _stream()),
                "ac_precond_solve")
        return out

    def richardson_step(self, alpha, u0, u, b=None, want_residual=False):
        res = ctypes.c_double(0.0)
        C.check(C.lib().ac_richardson_step(self._h, float(alpha), _ptr(u0), _ptr(b), _ptr(u),
                                           ctypes.byref(res) if want_residual else None, _stream()),
                "ac_richardson_step")
        return res.value if want_residual else None

    def richardson_step_host(self, alpha, u0, u, b=None, chunks=0, want_residual=False):
        """ac_richardson_step on CPU tensors (u0: N doubles or None, u: L*M*N
        doubles in/out, b: L*M*N doubles or None), copied in and out in
        chunks that overlap the kernels (page-locked tensors for overlap).
        Returns once the work is queued on the current stream (u is final
        after it has run), or with the residual when want_residual."""
        res = ctypes.c_double(0.0)
        C.check(C.lib().ac_richardson_step_host(self._h, float(alpha), _host_ptr(u0), _host_ptr(b), _host_ptr(u),
                                                int(chunks),
                                                ctypes.byref(res) if want_residual else None, _stream()),
                "ac_richardson_step_host")
        return res.value if want_residual else None

    def solve(self, u0, tol, b=None, u=None, raise_on_fail=True):
        """Richardson solve of C u = w; returns (u, stats dict)."""
        init = u is not None
        u = self.empty() if u is None else u
        st = C.Stats()
        rc = C.lib().ac_richardson_solve(self._h, _ptr(u0), _ptr(b), _ptr(u), int(init), float(tol),
                                         ctypes.byref(st), _stream())
        if rc != C.AC_OK and (raise_on_fail or rc != C.AC_ERR_NO_CONVERGENCE):
            C.check(rc, "ac_richardson_solve")
        return u, stats_dict(st)

    def window_solve(self, u0, n_windows, tol):
        """Moving window: n_windows consecutive L-step solves; returns (u at
        the end, total iterations, stats of the last window)."""
        u_end = torch.empty(self.N, dtype=torch.float64, device="cuda")
        work = self.empty()
        st = C.Stats()
        tot = ctypes.c_int(0)
        C.check(C.lib().ac_window_solve(self._h, _ptr(u0), int(n_windows), _ptr(u_end), _ptr(work), float(tol),
                                        ctypes.byref(st), ctypes.byref(tot), _stream()), "ac_window_solve")
        return u_end, tot.value, stats_dict(st)

    def krylov_solve(self, u0, tol, b=None, u=None, restart=10, raise_on_fail=True):
        """Outer flexible GMRES(restart) on C u = w, right-preconditioned by
        C_alpha^{-1}; returns (u, stats)."""
        init = u is not None
        u = self.empty() if u is None else u
        st = C.Stats()
        rc = C.lib().ac_krylov_solve(self._h, _ptr(u0), _ptr(b), _ptr(u), int(init), float(tol), int(restart),
                                     ctypes.byref(st), _stream())
        if rc != C.AC_OK and (raise_on_fail or rc != C.AC_ERR_NO_CONVERGENCE):
            C.check(rc, "ac_krylov_solve")
        return u, stats_dict(st)

    def sequential_solve(self, u0, b=None, out=None):
        """The L steps one after another by diagonalisation of Q (the
        paper's sequential baseline), replayed from a CUDA graph."""
        out = self.empty() if out is None else out
        C.check(C.lib().ac_sequential_solve(self._h, _ptr(u0), _ptr(b), _ptr(out), _stream()),
                "ac_sequential_solve")
        return out

    def adjoint_solve(self, g, tol, lam=None, raise_on_fail=True):
        lam = self.empty() if lam is None else lam
        st = C.Stats()
        rc = C.lib().ac_adjoint_solve(self._h, _ptr(g), _ptr(lam), float(tol), ctypes.byref(st), _stream())
        if rc != C.AC_OK and (raise_on_fail or rc != C.AC_ERR_NO_CONVERGENCE):
            C.check(rc, "ac_adjoint_solve")
        return lam, stats_dict(st)

    def grad_params(self, u, lam, want_du0=True):
        du0 = torch.empty(self.N, dtype=torch.float64, device="cuda") if want_du0 else None
        dp = (ctypes.c_double * 3)()
        C.check(C.lib().ac_grad_params(self._h, _ptr(u), _ptr(lam), _ptr(du0), ctypes.cast(dp, ctypes.c_void_p),
                                       _stream()), "ac_grad_params")
        return du0, np.array(dp[:])

    def profile(self, on=True):
        C.check(C.lib().ac_profile_enable(self._h, int(on)), "ac_profile_enable")

    def profile_read(self):
        cap = 8
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        cnt = (ctypes.c_longlong * cap)()
        n = C.lib().ac_profile_read(self._h, cap, names, ctypes.cast(ms, ctypes.c_void_p),
                                    ctypes.cast(cnt, ctypes.c_void_p))
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(n, cap))}


def measure_fp64_fma_rate():
    """FP64 FMAs per second of the current device (instrumentation)."""
    r = ctypes.c_double(0.0)
    C.check(C.lib().ac_measure_fp64_fma_rate(ctypes.byref(r), _stream()), "ac_measure_fp64_fma_rate")
    return r.value


# ------------------------------------------------------------------ host planner
def radau_nodes(M):
    t = np.zeros(M)
    C.check(C.lib().ac_radau_nodes(M, t.ctypes.data_as(ctypes.c_void_p)), "ac_radau_nodes")
    return t


def stencil_taps(prob):
    """(tx, ty, rad): per-axis taps of A on the offsets -3..3 (index o + 3)."""
    tx, ty, rad = np.zeros(7), np.zeros(7), ctypes.c_int(0)
    pr = make_problem(prob)
    C.check(C.lib().ac_stencil_taps(ctypes.byref(pr), tx.ctypes.data_as(ctypes.c_void_p),
                                    ty.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rad)), "ac_stencil_taps")
    return tx, ty, rad.value


def plan_shape(prob, M=None, L=None, precision="c128", inner="fft", space_cluster=0):
    """The launch shape ac_setup would choose (spatial path, time-kernel tiles,
    cluster size), computed on the host without a GPU."""
    M = int(M if M is not None else prob["M"])
    L = int(L if L is not None else prob["L"])
    sched = C.Schedule(space_cluster=int(space_cluster))
    info = C.PlanInfo()
    C.check(C.lib().ac_plan_shape(ctypes.byref(make_problem(prob)), M, L, PRECISION[precision], INNER[inner],
                                  ctypes.byref(sched), ctypes.byref(info)), "ac_plan_shape")
    return {f: getattr(info, f) for f, _ in C.PlanInfo._fields_}


def collocation_matrix(M):
    Q = np.zeros(M * M)
    C.check(C.lib().ac_collocation_matrix(M, Q.ctypes.data_as(ctypes.c_void_p)), "ac_collocation_matrix")
    return Q.reshape(M, M)


def freq_tables(M, L, alpha, transposed=False):
    F = L // 2 + 1
    mu = np.zeros((F, M, 2))
    Sinv = np.zeros((F, M, M, 2))
    P = np.zeros((F, M, M, 2))
    cond = np.zeros(F)
    rc = C.lib().ac_freq_tables(M, L, float(alpha), int(transposed), mu.ctypes.data_as(ctypes.c_void_p),
                                Sinv.ctypes.data_as(ctypes.c_void_p), P.ctypes.data_as(ctypes.c_void_p),
                                cond.ctypes.data_as(ctypes.c_void_p))
    c = lambda a: a[..., 0] + 1j * a[..., 1]
    return rc, c(mu), c(Sinv), c(P), cond


def alpha_sequence(m0, gamma, n):
    a = np.zeros(n)
    m = np.zeros(n + 1)
    C.check(C.lib().ac_alpha_sequence(float(m0), float(gamma), int(n), a.ctypes.data_as(ctypes.c_void_p),
                                      m.ctypes.data_as(ctypes.c_void_p)), "ac_alpha_sequence")
    return a, m


# ------------------------------------------------------------------ autograd
class RichardsonSolve(torch.autograd.Function):
    """u = C(nu, c)^{-1} w(u0) by the alpha-circulant Richardson solver.

    forward(u0, params, plan, tol): params = tensor([nu, cx, cy]) must match the
    plan's problem (the plan is built for those values); the gradient w.r.t.
    params comes from the adjoint contractions.  Returns u of shape (L, M, N)."""

    @staticmethod
    def forward(ctx, u0, params, plan, tol):
        plan_params = plan.params()
        given = [float(v) for v in params.detach().cpu().reshape(-1).tolist()]
        if len(given) != 3 or given != plan_params:
            raise ValueError("params %s differ from the plan's (nu, cx, cy) = %s: build the plan for these values"
                             % (given, plan_params))
        u, st = plan.solve(u0.contiguous(), tol)
        ctx.plan, ctx.tol = plan, tol
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        plan = ctx.plan
        lam, _ = plan.adjoint_solve(gu.contiguous(), ctx.tol)
        du0, dp = plan.grad_params(u, lam, want_du0=True)
        return du0, torch.tensor(dp, dtype=torch.float64, device=gu.device), None, None
