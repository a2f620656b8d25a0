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
