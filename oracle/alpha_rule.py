"""Algorithm 2: the adaptive alpha sequence and stopping rule (oracle; test
infrastructure only).

Sec. 3.3: with gamma := L (3 eps + tau) ||w||_inf and an estimate m_0 of
||u^{(0)} - u^*||_inf, minimising m_{k+1} = alpha m_k + gamma / alpha gives
    alpha_{k+1} = sqrt(gamma / m_k),   m_{k+1} = 2 sqrt(m_k gamma),
and, telescoped, m_k = (4 gamma)^{1 - 2^{-k}} m_0^{2^{-k}}.  Algorithm 2 runs
while m_k > tol and also stops as soon as ||u_L^{(k+1)} - u_L^{(k)}||_inf <= tol.
"""
import math


def gamma(L, eps, tau, w_inf):
    """gamma = L (3 eps + tau) ||w||_inf (Algorithm 2, first step)."""
    return L * (3.0 * eps + tau) * w_inf


def alpha_sequence(m0, gam, tol=None, kmax=64):
    """(alphas, ms) with alphas[k] = alpha_{k+1} and ms[k] = m_k (ms[0] = m0),
    generated while m_k > tol (all kmax terms when tol is None)."""
    alphas, ms = [], [m0]
    m = m0
    for _ in range(kmax):
        if tol is not None and m <= tol:
            break
        alphas.append(math.sqrt(gam / m))
        m = 2.0 * math.sqrt(m * gam)
        ms.append(m)
    return alphas, ms


def m_closed_form(k, gam, m0):
    """m_k = (4 gamma)^{1 - 2^{-k}} m_0^{2^{-k}} (Sec. 3.3)."""
    return (4.0 * gam) ** (1.0 - 2.0 ** (-k)) * m0 ** (2.0 ** (-k))


def run_algorithm2(iterate, u_init, last_block, m0, gam, tol, kmax=64):
    """Algorithm 2 around a user ``iterate(u, m, alpha) -> u_next``.

    ``last_block(u)`` returns u_L as an array.  Returns (u, alphas_used, ms)."""
    import numpy as np
    u, m = u_init, m0
    alphas, ms = [], [m0]
    k = 0
    while m > tol and k < kmax:
        m_next = 2.0 * math.sqrt(m * gam)
        alpha = math.sqrt(gam / m)
        u_next = iterate(u, m_next, alpha)
        alphas.append(alpha)
        ms.append(m_next)
        diff = np.max(np.abs(last_block(u_next) - last_block(u)))
        u, m = u_next, m_next
        k += 1
        if diff <= tol:
            break
    return u, alphas, ms
