"""Exact solution of the isothermal Euler Riemann problem (p = theta rho) and the measures that
compare a shocktube run with it: the checker of the isothermal shocktube of Sec. 5.2.

TEST INFRASTRUCTURE ONLY: tests/ use it. The product package never imports it, and it imports
nothing from the product package. Pinned by tests/test_riemann_cpu.py (Rankine-Hugoniot jumps, the
rarefaction's Riemann invariant, closed forms of the symmetric problems, conservation of the
integrals of rho and rho u).

Reading (the paper does not print the solution it compares with): the two-wave solution of the
isothermal Euler equations, each wave a shock (density rises across it) or a rarefaction, with the
middle state found by Newton's method on the sum of the two wave curves.
"""
from __future__ import annotations

import math

import numpy as np


def _wave_curve(rho, rho_k, c):
    """Velocity jump across a left/right wave from rho_k to rho, and its derivative: a shock
    (rho > rho_k), c (rho - rho_k) / sqrt(rho rho_k), or a rarefaction, c ln(rho / rho_k)."""
    if rho > rho_k:
        s = math.sqrt(rho * rho_k)
        return c * (rho - rho_k) / s, c * (rho + rho_k) / (2.0 * rho * s)
    return c * math.log(rho / rho_k), c / rho


def isothermal_riemann(rho_l: float, rho_r: float, theta: float, u_l: float = 0.0, u_r: float = 0.0):
    """Middle state (rho*, u*) of the isothermal Euler Riemann problem with p = theta rho: the root of
    f_L(rho*) + f_R(rho*) + u_r - u_l = 0 (f_K the wave curve of side K), by Newton's method, and
    u* = u_l - f_L(rho*)."""
    c = math.sqrt(theta)
    rho = math.sqrt(rho_l * rho_r)
    for _ in range(100):
        fl, dl = _wave_curve(rho, rho_l, c)
        fr, dr = _wave_curve(rho, rho_r, c)
        step = (fl + fr + u_r - u_l) / (dl + dr)
        rho = max(rho - step, 0.5 * rho)
        if abs(step) <= 1e-15 * rho:
            break
    return rho, u_l - _wave_curve(rho, rho_l, c)[0]


def isothermal_riemann_sample(rho_l: float, rho_r: float, theta: float, xi, u_l: float = 0.0, u_r: float = 0.0):
    """Exact (rho, u) of the isothermal Riemann problem at similarity coordinates xi = (x - x0) / t."""
    c = math.sqrt(theta)
    rs, us = isothermal_riemann(rho_l, rho_r, theta, u_l, u_r)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    for k, z in np.ndenumerate(xi):
        if z <= us:  # left of the contact: left state, left wave, or star
            if rs > rho_l:  # left shock, speed from mass conservation
                sl = u_l - c * math.sqrt(rs / rho_l)
                rho[k], u[k] = (rho_l, u_l) if z < sl else (rs, us)
            elif z < u_l - c:
                rho[k], u[k] = rho_l, u_l
            elif z > us - c:
                rho[k], u[k] = rs, us
            else:  # inside the left rarefaction: u - c = xi, u + c ln rho constant
                u[k] = z + c
                rho[k] = rho_l * math.exp((u_l - u[k]) / c)
        else:
            if rs > rho_r:
                sr = u_r + c * math.sqrt(rs / rho_r)
                rho[k], u[k] = (rho_r, u_r) if z > sr else (rs, us)
            elif z > u_r + c:
                rho[k], u[k] = rho_r, u_r
            elif z < us + c:
                rho[k], u[k] = rs, us
            else:  # inside the right rarefaction: u + c = xi, u - c ln rho constant
                u[k] = z - c
                rho[k] = rho_r * math.exp((u[k] - u_r) / c)
    return rho, u


def shocktube_measures(run: dict) -> dict:
    """Compare a shocktube run with the exact solution. `run` holds the fluid nodes' x, rho and
    u_x, the jump position x0 (between the two initial states), the step count, theta and the two
    initial densities (as returned by experiments.shocktube_run). Returns the exact fields at the
    nodes and: mean |rho - rho_exact| (l1_rho) and |u - u_exact| (l1_ux), the mean density and
    velocity over the middle state's interior (plateau_rho, plateau_ux) against rho*, u*
    (rho_star, u_star), and the total variation of rho above the exact (monotone) profile's
    (tv_excess: oscillations), and the run's finite flag; no comparison measures when the run is
    not finite."""
    theta, steps, x0 = run["theta"], run["steps"], run["x0"]
    rho_l, rho_r = run["rho_l"], run["rho_r"]
    x, r, u = run["x"], run["rho"], run["ux"]
    exact_rho, exact_u = isothermal_riemann_sample(rho_l, rho_r, theta, (x - x0) / steps)
    rs, us = isothermal_riemann(rho_l, rho_r, theta)
    out = {"rho_exact": exact_rho, "ux_exact": exact_u, "rho_star": rs, "u_star": us, "finite": run["finite"]}
    if not run["finite"]:
        return out
    c = math.sqrt(theta)
    # interior of the middle state: between the rarefaction tail and the shock, 10 nodes in
    lo, hi = x0 + (us - c) * steps + 10, x0 + c * math.sqrt(rs / rho_r) * steps - 10
    mid = (x > lo) & (x < hi)
    out.update({"l1_rho": float(np.mean(np.abs(r - exact_rho))), "l1_ux": float(np.mean(np.abs(u - exact_u))),
                "plateau_rho": float(r[mid].mean()), "plateau_ux": float(u[mid].mean()),
                "tv_excess": float(np.abs(np.diff(r)).sum() - np.abs(np.diff(exact_rho)).sum())})
    return out
