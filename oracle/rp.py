"""Rayleigh-Plesset radius history of a spherical gas bubble, Eq. (4.1).

TEST INFRASTRUCTURE: part of the CPU oracle. It is the reference the time-stepped
boundary-element bubble is compared with in Section 4.1.

Reading of Eq. (4.1): the printed right-hand side lacks the factor 1/rho; the equation is
read as
    a a'' + (3/2) a'^2 = (1/rho) [ p_g0 (a0/a)^(3 kappa) - p_inf(t) - 2 sigma / a ],
with p_g0 = p0 + 2 sigma / a0 (Eq. (2.8)) and p_inf(t) = p0 - Pa sin(omega t) (Eq. (2.6)),
a(0) = a0, a'(0) = 0 unless a different start is given.

Everything is dimensionless: lengths by a0, pressures by p0, time by a0 sqrt(rho / p0),
so rho = 1, p0 = 1, and sigma' = sigma / (p0 a0).
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp


def rp_rhs(t, y, sigma, kappa, pa, omega):
    a, adot = y
    pg0 = 1.0 + 2.0 * sigma
    pinf = 1.0 - pa * np.sin(omega * t)
    rhs = pg0 * a ** (-3.0 * kappa) - pinf - 2.0 * sigma / a
    return [adot, (rhs - 1.5 * adot * adot) / a]


def rayleigh_plesset(t_eval, sigma, kappa, pa, omega, a0=1.0, adot0=0.0, rtol=1e-11, atol=1e-13):
    """Integrate Eq. (4.1) with an error-controlled Runge-Kutta (DOP853) solver and return
    (a(t), a'(t)) at the requested times."""
    t_eval = np.asarray(t_eval, dtype=np.float64)
    sol = solve_ivp(rp_rhs, (0.0, float(t_eval[-1])), [a0, adot0], method="DOP853",
                    t_eval=t_eval, rtol=rtol, atol=atol, args=(sigma, kappa, pa, omega))
    if not sol.success:
        raise RuntimeError(sol.message)
    return sol.y[0], sol.y[1]


def rp_energy(a, adot, sigma, kappa):
    """Conserved energy of the unforced (pa = 0) equation, per unit rho, for kappa != 1:
    kinetic 2 pi a^3 a'^2 plus the work against p_inf = 1, the surface tension and the
    polytropic gas."""
    pg0 = 1.0 + 2.0 * sigma
    kin = 2.0 * np.pi * a ** 3 * adot ** 2
    pot = (4.0 * np.pi / 3.0) * a ** 3 + 4.0 * np.pi * sigma * a ** 2 \
        - 4.0 * np.pi * pg0 * a ** (3.0 - 3.0 * kappa) / (3.0 - 3.0 * kappa)
    return kin + pot
