"""The C ABI library on the CPU: it builds, loads, exports every declared
symbol, and its host-side planner agrees with the oracle (no GPU calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import alpha_rule, collocation, paradiag, stencils


@pytest.fixture(scope="module")
def api():
    from paper_2103_12571_gb300 import build
    build.build()
    from paper_2103_12571_gb300 import api as A
    return A


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ac_[A-Za-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol(api):
    from paper_2103_12571_gb300 import _lib
    L = ctypes.CDLL(_lib.LIB_PATH)
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 6])
def test_host_nodes_and_Q_match_oracle(api, M):
    t = collocation.radau_iia_nodes(M)
    np.testing.assert_allclose(api.radau_nodes(M), t, atol=2e-15)
    np.testing.assert_allclose(api.collocation_matrix(M), collocation.collocation_matrix(t), atol=5e-14)


@pytest.mark.parametrize("M,L,alpha", [(2, 4, 1e-4), (3, 64, 3e-3), (3, 512, 1e-2), (4, 16, 0.3), (1, 8, 1e-6)])
@pytest.mark.parametrize("transposed", [False, True])
def test_host_eigen_tables(api, M, L, alpha, transposed):
    rc, mu, Sinv, P, cond = api.freq_tables(M, L, alpha, transposed)
    assert rc == 0
    t = collocation.radau_iia_nodes(M)
    Q = collocation.collocation_matrix(t)
    H = collocation.H_matrix(M)
    d = paradiag.eigenvalues_d(L, alpha)
    for f in range(L // 2 + 1):
        r = d[f] / (1 + d[f])
        Hm = H.T if transposed else H
        Ginv = np.eye(M) - r * Hm
        B = (Q.T if transposed else Q) @ Ginv
        S = np.linalg.inv(Sinv[f])
        np.testing.assert_allclose(B @ S, S @ np.diag(mu[f]), atol=1e-12 * cond[f])
        np.testing.assert_allclose(P[f], Ginv @ S, atol=1e-12 * cond[f])
        # eigenvalues against Lemma 2 / numpy
        if not transposed:
            ev = list(np.roots(paradiag.lemma2_char_poly(t, r)[::-1]))
            for x in mu[f]:
                j = int(np.argmin([abs(x - e) for e in ev]))
                assert abs(x - ev.pop(j)) < 1e-10
        assert cond[f] < 1e6


def test_host_eigen_guard_on_defective_block(api):
    # M = 2: Q G^{-1} is defective where 9 r^2 - 6 r - 2 = 0, r = (1 - sqrt 3)/3,
    # i.e. d = r / (1 - r); with L = 2 the f = 0 block has d = -alpha^{1/2}
    r = (1 - 3 ** 0.5) / 3
    d = r / (1 - r)
    alpha = d * d
    rc, mu, Sinv, P, cond = api.freq_tables(2, 2, alpha, False)
    assert rc == -2 and cond[0] > 1e10 or cond[0] > 1e6
    rc2, *_ = api.freq_tables(2, 2, alpha * 1.5, False)
    assert rc2 == 0


def test_host_alpha_sequence_matches_oracle(api):
    a, m = api.alpha_sequence(2e-3, 7.66e-16, 6)
    ao, mo = alpha_rule.alpha_sequence(2e-3, 7.66e-16, kmax=6)
    np.testing.assert_allclose(a, ao, rtol=1e-15)
    np.testing.assert_allclose(m, mo, rtol=1e-15)


def test_setup_rejects_bad_arguments(api):
    from paper_2103_12571_gb300 import workloads
    from paper_2103_12571_gb300._lib import ACError
    p = workloads.problem(1, 64, nu=0.1, M=2, L=4, T=0.1)
    for kw in (dict(L=6), dict(M=0), dict(M=5), dict(L=1), dict(dT=-1.0)):
        with pytest.raises(ACError) as e:
            api.Plan(p, **kw)
        assert e.value.code == -1
    with pytest.raises(ACError):
        api.Plan(workloads.problem(1, 48, nu=0.1, M=2, L=4), inner="fft")


SCHEMES = [(p, False) for p in (2, 4, 6)] + [(p, True) for p in (1, 2, 3, 4, 5)]


@pytest.mark.parametrize("order,upwind", SCHEMES)
def test_host_stencil_taps_match_oracle(api, order, upwind):
    """ac_stencil_taps against the oracle's finite-difference weights (derived
    there from the moment conditions), both signs of each velocity, 1D and
    2D, non-unit box lengths."""
    from paper_2103_12571_gb300 import workloads
    for dim, cx, cy in ((1, 0.7, 0.0), (1, -1.3, 0.0), (2, -0.4, 0.9), (2, 1.1, -0.2)):
        prob = workloads.problem(dim, 48, 40, nu=0.03, cx=cx, cy=cy, order=order, upwind=upwind)
        prob["lx"], prob["ly"] = 2.0, 0.5
        tx, ty, rad = api.stencil_taps(prob)
        want = {}
        for axis, n, length, c in (("x", 48, 2.0, cx), ("y", 40, 0.5, cy)):
            h = length / n
            w = np.zeros(7)
            if axis == "x" or dim == 2:
                for o, v in stencils.d2_weights(order, upwind).items():
                    w[o + 3] += 0.03 * float(v) / h ** 2
                for o, v in stencils.d1_weights(order, upwind, c).items():
                    w[o + 3] -= c * float(v) / h
            want[axis] = w
        np.testing.assert_allclose(tx, want["x"], rtol=1e-14, atol=1e-12)
        np.testing.assert_allclose(ty, want["y"], rtol=1e-14, atol=1e-12)
        sup = max(abs(o) for o in list(stencils.d1_weights(order, upwind, 1.0)) +
                  list(stencils.d2_weights(order, upwind)))
        assert rad == sup


def test_host_stencil_taps_reject_unsupported(api):
    from paper_2103_12571_gb300 import workloads
    from paper_2103_12571_gb300._lib import ACError
    for order, upwind in ((3, False), (8, False), (0, True), (6, True)):
        with pytest.raises(ACError):
            api.stencil_taps(workloads.problem(1, 32, nu=0.1, cx=1.0, order=order, upwind=upwind))
        with pytest.raises(ACError):
            api.Plan(workloads.problem(1, 32, nu=0.1, cx=1.0, order=order, upwind=upwind, M=2, L=4))


def test_new_entry_points_reject_null_arguments(api):
    """Argument checks of the C ABI run before any device work (no GPU)."""
    from paper_2103_12571_gb300 import _lib
    L = _lib.lib()
    st = _lib.Stats()
    assert L.ac_sequential_solve(None, None, None, None, None) == _lib.AC_ERR_INVALID_ARG
    assert L.ac_krylov_solve(None, None, None, None, 0, ctypes.c_double(1e-10), 10, ctypes.byref(st),
                             None) == _lib.AC_ERR_INVALID_ARG
    assert L.ac_window_solve(None, None, 1, None, None, ctypes.c_double(1e-10), None, None, None) == \
        _lib.AC_ERR_INVALID_ARG
    assert L.ac_stencil_taps(None, None, None, None) == _lib.AC_ERR_INVALID_ARG
    msg = L.ac_last_error()
    assert msg is not None


def test_binding_declares_every_header_function(api):
    """Every function the header declares has a ctypes prototype in the
    binding (so no call goes through ctypes' default int conversions)."""
    from paper_2103_12571_gb300 import _lib
    assert sorted(declared_symbols()) == sorted(_lib._PROTOS)


# ---- the planner's launch shapes (host logic, no GPU)
def _shape(prob, **kw):
    from paper_2103_12571_gb300.api import plan_shape
    return plan_shape(prob, **kw)


def test_plan_shape_spatial_paths():
    """Power-of-two grids take the FFT paths 0 (1D), 1 (2D plane of at most
    160 KB) and 2 (three passes); sizes with prime factors 2, 3, 5, 7 take the
    mixed-radix paths 5 (1D) and 6 (2D); the Krylov solvers are paths 3 and 4;
    the cluster solve (path 7) runs only on request."""
    from paper_2103_12571_gb300 import workloads
    P = workloads.problem
    assert _shape(P(1, 4096, cx=1.0, order=4, M=3, L=256, T=1.0))["spatial_path"] == 0
    assert _shape(P(2, 64, 64, nu=0.05, M=3, L=8, T=0.1))["spatial_path"] == 1
    assert _shape(P(2, 512, 512, nu=1e-3, M=3, L=512, T=2.0))["spatial_path"] == 2
    assert _shape(P(2, 512, 512, nu=1e-3, M=3, L=512, T=2.0), precision="c64")["spatial_path"] == 2
    assert _shape(P(1, 700, cx=1.0, order=5, upwind=True, M=3, L=64, T=0.0128))["spatial_path"] == 5
    assert _shape(P(2, 700, 700, cx=1.0, cy=1.0, order=5, upwind=True, M=3, L=64, T=0.0128))["spatial_path"] == 6
    assert _shape(P(2, 350, 600, nu=0.01, M=2, L=8, T=0.01), precision="c64")["spatial_path"] == 6
    prob = P(2, 24, 20, nu=0.02, M=3, L=8, T=0.1)
    assert _shape(prob, inner="bicgstab")["spatial_path"] == 3
    assert _shape(prob, inner="gmres")["spatial_path"] == 4
    s = _shape(P(2, 256, 256, nu=0.05, M=3, L=64, T=0.5), precision="c64", space_cluster=8)
    assert s["spatial_path"] == 7 and s["space_cluster"] == 8
    assert _shape(P(2, 256, 256, nu=0.05, M=3, L=64, T=0.5), precision="c64")["space_cluster"] == 0


def test_plan_shape_rejects_what_setup_rejects():
    from paper_2103_12571_gb300 import workloads
    from paper_2103_12571_gb300._lib import ACError
    P = workloads.problem
    for prob, kw in [
        (P(1, 11 * 13, nu=0.1, M=2, L=8, T=0.1), {}),                          # prime factors 11, 13: no FFT
        (P(2, 512, 64, nu=0.01, M=3, L=4, T=0.05), dict(precision="c64", space_cluster=16)),  # 4 rows per CTA
        (P(2, 256, 256, nu=0.05, M=3, L=8, T=0.1), dict(space_cluster=5)),    # not a cluster size
        (P(1, 64, nu=0.1, M=5, L=8, T=0.1), {}),                               # M > 4
        (P(1, 64, nu=0.1, M=2, L=12, T=0.1), {}),                              # L not a power of two
        (P(2, 2, 2, nu=0.1, order=6, M=2, L=8, T=0.1), dict(inner="bicgstab")),  # grid below the stencil
    ]:
        with pytest.raises(ACError):
            _shape(prob, **kw)
    # the same sizes with a Krylov inner solve are accepted
    assert _shape(P(1, 11 * 13, nu=0.1, M=2, L=8, T=0.1), inner="gmres")["spatial_path"] == 4


def test_plan_shape_time_tiles():
    """Time-kernel tiles: L*M*P transform values within the shared-memory
    budget (about 50 KB), at least two CTAs per SM where the grid allows, a
    quarter or half tile for complex64 residual kernels."""
    from paper_2103_12571_gb300 import workloads
    prob = workloads.config(5)[0]
    s128 = _shape(prob)
    s64 = _shape(prob, precision="c64")
    assert s128["tile_fwd"] == 4 and s128["F"] == 257 and s128["N"] == 512 * 512
    assert s64["tile_fwd"] == 8
    for s, rsz in ((s128, 8), (s64, 4)):
        assert prob["L"] * prob["M"] * s["tile_fwd"] * rsz <= 50 * 1024
