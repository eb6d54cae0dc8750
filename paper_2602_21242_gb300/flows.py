"""Seeded synthetic inputs shaped like the paper's benchmark flows.

This module holds flow set-ups and random draws only -- no lattice Boltzmann
arithmetic (no equilibrium, no collision, no streaming). It is the one module
that both the CUDA path's tests/benchmarks and the CPU oracle receive inputs
from; each side turns (rho0, u0) into populations with its own code.

Generators are numpy ``Generator(PCG64(seed))``. Every field is returned as
float64 arrays of shape (ny, nx), row-major with x fastest.

Flow recipes (arXiv 2602.21242, Sec. 5, and the benchmark configurations built
on it):
  * Taylor-Green vortex, doubly periodic (decay check).
  * Advected shear wave u_y = A sin(2 pi x / nx) on a background u_x = U
    (bandwidth benchmark; Galilean check through U).
  * Doubly periodic shear layer (Sec. 5.3 form, with a tanh width in cells).
  * Random divergence-free Fourier modes |k| <= kmax (differentiation runs).
  * Batches of independent Taylor-Green domains of uneven size.
  * Random positive populations around a fixed shape (parity on generic,
    non-equilibrium states).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 2602212420

# Standard D2Q9 rest weights, used here only as a positive SHAPE for random
# populations (data, not the method's equilibrium).
_SHAPE9 = np.array([16, 4, 4, 4, 4, 1, 1, 1, 1], dtype=np.float64) / 36.0


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _grid(nx: int, ny: int):
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    return x, y


def taylor_green(nx: int, ny: int, u0: float, theta: float, rho0: float = 1.0):
    """Doubly periodic Taylor-Green vortex with k = 2 pi / n per axis.

    u_x = -u0 cos(k_x x) sin(k_y y), u_y = u0 sin(k_x x) cos(k_y y), and the
    pressure-consistent density rho = rho0 - rho0 u0^2/(4 theta) (cos 2k_x x + cos 2k_y y)
    (isothermal p = rho theta).
    """
    x, y = _grid(nx, ny)
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    ux = -u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = u0 * np.sin(kx * x) * np.cos(ky * y)
    rho = rho0 - rho0 * u0 * u0 / (4.0 * theta) * (np.cos(2 * kx * x) + np.cos(2 * ky * y))
    return np.ascontiguousarray(rho), np.ascontiguousarray(ux), np.ascontiguousarray(uy)


def shear_wave(nx: int, ny: int, U: float = 0.0, amp: float = 0.01, rho0: float = 1.0):
    """Advected transverse shear wave: u_x = U, u_y = amp sin(2 pi x / nx), rho = rho0."""
    x, y = _grid(nx, ny)
    ux = np.full((ny, nx), float(U))
    uy = np.broadcast_to(amp * np.sin(2 * math.pi * x / nx), (ny, nx)).copy()
    rho = np.full((ny, nx), float(rho0))
    return rho, ux, uy


def shear_layer(nx: int, ny: int, U: float = 0.1, width: float = 80.0, delta_amp: float = 0.005,
                rho0: float = 1.0):
    """Doubly periodic shear layer: two mirrored tanh layers at y = ny/4 and 3ny/4.

    u_x = U tanh((y - ny/4)/width) for y <= ny/2 and U tanh((3ny/4 - y)/width) otherwise;
    u_y = delta_amp sin(2 pi x / nx).
    """
    x, y = _grid(nx, ny)
    lower = U * np.tanh((y - ny / 4.0) / width)
    upper = U * np.tanh((3.0 * ny / 4.0 - y) / width)
    ux = np.broadcast_to(np.where(y <= ny / 2.0, lower, upper), (ny, nx)).copy()
    uy = np.broadcast_to(delta_amp * np.sin(2 * math.pi * x / nx), (ny, nx)).copy()
    rho = np.full((ny, nx), float(rho0))
    return rho, ux, uy


def random_modes(n: int, seed: int, kmax: int = 8, amp: float = 0.02, rho0: float = 1.0):
    """Divergence-free velocity from a random stream function.

    psi_s = sum_{0 < |k| <= kmax} (a_k cos(k.x) + b_k sin(k.x)) / |k|^2 with
    a, b ~ N(0, 1); u = (d_y psi_s, -d_x psi_s) (analytic derivatives), scaled to
    max |u| = amp; rho = rho0.
    """
    g = rng(seed)
    x, y = _grid(n, n)
    ux = np.zeros((n, n))
    uy = np.zeros((n, n))
    two_pi_n = 2 * math.pi / n
    for mx in range(-kmax, kmax + 1):
        for my in range(-kmax, kmax + 1):
            k2 = mx * mx + my * my
            if k2 == 0 or k2 > kmax * kmax:
                continue
            a, b = g.standard_normal(2)
            kx, ky = mx * two_pi_n, my * two_pi_n
            phase = kx * x + ky * y
            # d/dy and d/dx of (a cos + b sin)(phase) / |k|^2
            dpsi = (-a * np.sin(phase) + b * np.cos(phase)) / k2
            ux += ky * dpsi
            uy -= kx * dpsi
    speed = np.sqrt(ux * ux + uy * uy).max()
    scale = amp / speed if speed > 0 else 0.0
    return np.full((n, n), float(rho0)), ux * scale, uy * scale


def random_populations(nx: int, ny: int, seed: int, spread: float = 0.2, rho_scale: float = 1.0):
    """Positive random populations (9, ny, nx): a fixed positive shape times (1 + spread*U(-1, 1))."""
    g = rng(seed)
    noise = g.uniform(-1.0, 1.0, size=(9, ny, nx))
    return np.ascontiguousarray(rho_scale * _SHAPE9[:, None, None] * (1.0 + spread * noise))


@dataclass(frozen=True)
class Domain:
    n: int
    theta: float
    nu: float
    u0: float


def batch_domains(count: int = 256, seed: int = SEED_BASE + 5, nmin: int = 64, nmax: int = 512):
    """Independent square Taylor-Green domains: N ~ U{nmin..nmax}, theta ~ U[0.25, 0.4],
    nu ~ U[0.002, 0.02], u0 ~ U[0.02, 0.1]."""
    g = rng(seed)
    ns = g.integers(nmin, nmax + 1, size=count)
    thetas = g.uniform(0.25, 0.4, size=count)
    nus = g.uniform(0.002, 0.02, size=count)
    u0s = g.uniform(0.02, 0.1, size=count)
    return [Domain(int(n), float(t), float(v), float(u)) for n, t, v, u in zip(ns, thetas, nus, u0s)]
