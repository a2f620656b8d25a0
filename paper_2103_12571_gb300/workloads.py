"""Seeded synthetic inputs and the five benchmark problem definitions.

This module holds no arithmetic of the method: it only builds initial fields
u0 and problem descriptions (plain dicts) that the CUDA path and the CPU
oracle both receive as arguments.  The fields are shaped after the paper's
periodic heat and advection tests (Sec. 5, eqs. (heat), (advection)).

Problem dict keys: dim, nx, ny, lx, ly, nu, cx, cy, order  (spatial operator
A = nu Lap_h - cx D_x - cy D_y, periodic central differences of ``order``),
plus M (Radau IIA nodes), L (time steps), T (end time); dT = T / L.
"""
import numpy as np


def _grid(n, length=1.0):
    return np.arange(n) * (length / n)


def u0_sines_1d(nx):
    """sin(2 pi x) + 0.5 sin(6 pi x) on x_j = j / nx."""
    x = _grid(nx)
    return np.sin(2 * np.pi * x) + 0.5 * np.sin(6 * np.pi * x)


def u0_fourier_modes_2d(nx, ny, n_modes=16, kmax=8, seed=0):
    """Sum of n_modes distinct cosines cos(2 pi k.x) with integer wavevectors
    drawn uniformly from {0 < |k|_2 <= kmax} and N(0,1) amplitudes."""
    rng = np.random.default_rng(seed)
    ks = [(kx, ky) for kx in range(-kmax, kmax + 1) for ky in range(-kmax, kmax + 1)
          if 0 < kx * kx + ky * ky <= kmax * kmax]
    pick = rng.choice(len(ks), size=n_modes, replace=False)
    amp = rng.standard_normal(n_modes)
    x = _grid(nx)[None, :]
    y = _grid(ny)[:, None]
    u = np.zeros((ny, nx))
    for a, i in zip(amp, pick):
        kx, ky = ks[i]
        u += a * np.cos(2 * np.pi * (kx * x + ky * y))
    return u.reshape(-1)


def u0_gaussian_pulse_1d(nx, center=0.5, width=0.05):
    """exp(-((x - center) / width)^2)."""
    x = _grid(nx)
    return np.exp(-((x - center) / width) ** 2)


def smoothed_noise_2d(nx, ny, sigma_cells=4.0, seed=0):
    """N(0,1) white noise filtered by a periodic Gaussian of width sigma_cells
    grid cells (applied in Fourier space with exp(-2 pi^2 sigma^2 (k/n)^2))."""
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((ny, nx))
    kx = np.fft.fftfreq(nx)[None, :]
    ky = np.fft.fftfreq(ny)[:, None]
    g = np.exp(-2 * np.pi ** 2 * sigma_cells ** 2 * (kx ** 2 + ky ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(xi) * g)).reshape(-1)


def random_phase_bumps_2d(nx, ny, kscale=8.0, seed=0):
    """Random-phase field with Gaussian spectrum exp(-|k|^2 / (2 kscale^2)),
    Hermitian (real), normalised to max |u0| = 1."""
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((ny, nx))
    xh = np.fft.fft2(xi)
    xh = xh / np.maximum(np.abs(xh), 1e-300)
    kx = np.fft.fftfreq(nx, d=1.0 / nx)[None, :]
    ky = np.fft.fftfreq(ny, d=1.0 / ny)[:, None]
    env = np.exp(-(kx ** 2 + ky ** 2) / (2 * kscale ** 2))
    u = np.real(np.fft.ifft2(xh * env))
    return (u / np.max(np.abs(u))).reshape(-1)


def problem(dim, nx, ny=1, nu=0.0, cx=0.0, cy=0.0, order=2, M=3, L=4, T=1.0, upwind=False):
    return dict(dim=dim, nx=nx, ny=ny if dim == 2 else 1, lx=1.0, ly=1.0, nu=nu,
                cx=cx, cy=cy, order=order, M=M, L=L, T=T, upwind=bool(upwind))


def config(i):
    """(problem, u0, extras) of the five workloads, i = 1..5."""
    if i == 1:
        p = problem(1, 64, nu=0.1, order=2, M=2, L=4, T=0.1)
        return p, u0_sines_1d(64), dict(alpha=1e-4, tol=1e-12, name="heat1d_N64_M2_L4")
    if i == 2:
        p = problem(2, 256, 256, nu=0.05, order=2, M=3, L=64, T=0.5)
        return p, u0_fourier_modes_2d(256, 256, seed=0), dict(name="heat2d_256x256_M3_L64")
    if i == 3:
        p = problem(1, 4096, nu=0.0, cx=1.0, order=4, M=3, L=256, T=1.0)
        return p, u0_gaussian_pulse_1d(4096), dict(tau=1e-8, name="advection1d_N4096_M3_L256")
    if i == 4:
        p = problem(2, 128, 128, nu=0.05, order=2, M=3, L=32, T=0.25)
        return p, smoothed_noise_2d(128, 128, 4.0, seed=0), dict(
            u_target=smoothed_noise_2d(128, 128, 4.0, seed=1), name="heat2d_adjoint_128x128_M3_L32")
    if i == 5:
        p = problem(2, 512, 512, nu=1e-3, cx=1.0, cy=0.5, order=2, M=3, L=512, T=2.0)
        return p, random_phase_bumps_2d(512, 512, 8.0, seed=0), dict(name="advdiff2d_512x512_M3_L512")
    raise ValueError(i)


# ---- the paper's forced heat test (Sec. 5, eq. (heat)) on [pi, pi + T] x [0,1]^2
HEAT_T0 = np.pi


def heat_forcing_problem(n, order=2, M=3, L=16, T=0.1):
    """u_t = Lap u + sin(2 pi x) sin(2 pi y) (8 pi^2 cos t - sin t), periodic."""
    return problem(2, n, n, nu=1.0, order=order, M=M, L=L, T=T)


def heat_forcing_field(n):
    """phi(x, y) = sin(2 pi x) sin(2 pi y) on the n x n grid (flat index iy*n + ix)."""
    x = _grid(n)
    return (np.sin(2 * np.pi * x)[None, :] * np.sin(2 * np.pi * x)[:, None]).reshape(-1)


def heat_forcing_samples(n, times):
    """b at the given times (array of shape (L, M)): b[l, m] = (8 pi^2 cos t - sin t) phi."""
    times = np.asarray(times)
    f = 8 * np.pi ** 2 * np.cos(times) - np.sin(times)
    return f[..., None] * heat_forcing_field(n)[None, None, :]


def heat_forcing_u0(n):
    """u(pi) of cos(t) phi, the exact solution under the printed forcing
    (substitution gives cos t, not the printed sin t)."""
    return np.cos(HEAT_T0) * heat_forcing_field(n)
