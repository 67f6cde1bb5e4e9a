"""Linear QSA theory of the paper (Eqs. 1-7), FP64 / multiprecision.  TEST INFRASTRUCTURE ONLY.

Normalised units (k_p = omega_p = c = 1).  Sign convention of the build: psi = -Psi of the
paper (Eq. 2), so a density perturbation of the beam, rho_b1, drives
    (d_xi^2 + 1) n_p1 = rho_b1                       (Eq. 1)
    (lap - 1) psi1 = n_p1  ->  psi^ = -n_p^/(k^2 + 1)  (Eq. 2 with Psi = -psi)
and each beam species responds with d_tau^2 n_bs1 = (Z_s alpha_s/(gamma_b M_s)) lap psi1
(Eq. 3 without the gamma_b^-2 d_xi^2 term), which gives Eq. 5:
    [(d_xi^2 + 1) d_tau^2 - Gamma^2] psi^ = 0,
    Gamma^2 = sum_s omega_bs^2 k^2/(k^2 + 1),  omega_bs^2 = Z_s^2 alpha_s/(gamma_b M_s)  (Eq. 5).

Exact solution used as the growth-rate reference (a reading: the paper solves Eq. 5
numerically for its Fig. 1e).  For a cold beam whose density perturbation rho^_b0 is uniform
in xi from the front xi = 0, with zero data ahead of the front, the Laplace transform in xi
(variable s) gives
    psi~(s, tau) = -rho^_b0 cosh(Gamma tau / sqrt(s^2 + 1)) / ((k^2 + 1) s (s^2 + 1)),
so psi^(xi, tau) = -rho^_b0/(k^2+1) * sum_n (Gamma tau)^(2n)/(2n)! h_{n+1}(xi),
    h_m(xi) = L^-1[1/(s (s^2+1)^m)] = sum_i (-1)^i C(m+i-1, i) xi^(2(m+i)) / (2(m+i))!,
evaluated in multiprecision arithmetic (the series alternates).  h_1 = 1 - cos xi is the
step-on wake of Eq. 1.
"""
from __future__ import annotations

import math

import mpmath
import numpy as np


def omega_b2(species):
    """sum_s omega_bs^2 with omega_bs = Z_s sqrt(alpha_s/(gamma_b M_s)) (QSA section)."""
    return sum(s.Z ** 2 * s.alpha / (s.gamma_b * s.M) for s in species)


def growth_rate(k, species):
    """Gamma of Eq. 5 for transverse wavenumber |k| (units of k_p)."""
    return math.sqrt(omega_b2(species) * k * k / (k * k + 1.0))


def gamma_otsi(Gamma):
    """Temporal OTSI rate quoted after Eq. 6: sqrt(3)/2^(4/3) Gamma^(2/3)."""
    return math.sqrt(3.0) / 2.0 ** (4.0 / 3.0) * Gamma ** (2.0 / 3.0)


def exponent_rear(Gamma_tau, xi):
    """Growth exponent of Eq. 6 (far from the front): (3 sqrt 3 / 4)(Gamma tau)^(2/3) xi^(1/3)."""
    return 3.0 * math.sqrt(3.0) / 4.0 * Gamma_tau ** (2.0 / 3.0) * xi ** (1.0 / 3.0)


def exponent_front(Gamma_tau, xi):
    """Growth exponent of Eq. 7 (near the front): 2 sqrt(Gamma tau xi) (1 - xi/(4 Gamma tau))."""
    return 2.0 * math.sqrt(Gamma_tau * xi) * (1.0 - xi / (4.0 * Gamma_tau))


def transition_xi(Gamma_tau):
    """Front/rear boundary quoted with Eqs. 6-7: xi = 2 Gamma tau / sqrt(27)."""
    return 2.0 * Gamma_tau / math.sqrt(27.0)


def local_rate_front(Gamma, xi, tau):
    """Spatiotemporal CFI rate from the blazar paragraph: sqrt(Gamma xi / tau)."""
    return math.sqrt(Gamma * xi / tau)


def local_rate_rear(Gamma, xi, tau):
    """Spatiotemporal OTSI rate from the blazar paragraph: (sqrt 3/2) Gamma^(2/3) (xi/tau)^(1/3)."""
    return math.sqrt(3.0) / 2.0 * Gamma ** (2.0 / 3.0) * (xi / tau) ** (1.0 / 3.0)


def _h(m, xi, tol):
    """h_m(xi) = L^-1[1/(s (s^2+1)^m)] by its power series (mpmath)."""
    xi = mpmath.mpf(xi)
    total = mpmath.mpf(0)
    i = 0
    while True:
        term = (-1) ** i * mpmath.binomial(m + i - 1, i) * xi ** (2 * (m + i)) \
            / mpmath.factorial(2 * (m + i))
        total += term
        if i > 4 and abs(term) < tol:
            return total
        i += 1


def psi_series(xi, Gamma_tau, rho_b0=1.0, k=1.0, dps=60, tol=1e-45):
    """psi^(xi, tau) of Eq. 5 for a uniform step seed rho^_b0 (see module docstring)."""
    with mpmath.workdps(dps):
        gt2 = mpmath.mpf(Gamma_tau) ** 2
        total = mpmath.mpf(0)
        n = 0
        while True:
            term = gt2 ** n / mpmath.factorial(2 * n) * _h(n + 1, xi, tol)
            total += term
            if n > 3 and abs(term) < tol * (1 + abs(total)):
                break
            n += 1
        return float(-rho_b0 / (k * k + 1.0) * total)


def march_eq5(xi_grid, tau_end, n_tau, Gamma, rho_b0=1.0, k=1.0):
    """Independent numerical solution of Eq. 5: RK4 in tau on (psi, d_tau psi) with
    d_tau^2 psi = V, (d_xi^2 + 1) V = Gamma^2 psi, V(0) = V'(0) = 0, evaluated as
    V(xi) = Gamma^2 int_0^xi sin(xi - xi') psi(xi') dxi' (trapezoid rule on xi_grid).
    Initial data: psi(xi, 0) = -rho_b0 (1 - cos xi)/(k^2+1), d_tau psi = 0 (cold beam)."""
    xi_grid = np.asarray(xi_grid, dtype=np.float64)
    dx = np.diff(xi_grid)
    s, c = np.sin(xi_grid), np.cos(xi_grid)

    def V(psi):
        # sin(xi - xi') = sin xi cos xi' - cos xi sin xi'
        a = np.concatenate([[0.0], np.cumsum(0.5 * dx * (c[1:] * psi[1:] + c[:-1] * psi[:-1]))])
        b = np.concatenate([[0.0], np.cumsum(0.5 * dx * (s[1:] * psi[1:] + s[:-1] * psi[:-1]))])
        return Gamma ** 2 * (s * a - c * b)

    psi = -rho_b0 * (1.0 - c) / (k * k + 1.0)
    dpsi = np.zeros_like(psi)
    h = tau_end / n_tau
    for _ in range(n_tau):
        k1p, k1v = dpsi, V(psi)
        k2p, k2v = dpsi + 0.5 * h * k1v, V(psi + 0.5 * h * k1p)
        k3p, k3v = dpsi + 0.5 * h * k2v, V(psi + 0.5 * h * k2p)
        k4p, k4v = dpsi + h * k3v, V(psi + h * k3p)
        psi = psi + h / 6.0 * (k1p + 2 * k2p + 2 * k3p + k4p)
        dpsi = dpsi + h / 6.0 * (k1v + 2 * k2v + 2 * k3v + k4v)
    return psi


def wake_1d(xi_grid, n_b, rtol=1e-12):
    """Nonlinear 1D wake of a uniform electron beam of density n_b (current -n_b) starting at
    xi = 0, from the k = 0 equations: psi'' = [(1+psi)^-2 - 1]/2 + n_b, psi(0) = psi'(0) = 0.
    Returns psi and E_z = psi' on xi_grid (high-order Runge-Kutta, scipy)."""
    from scipy.integrate import solve_ivp

    def rhs(_, y):
        return [y[1], 0.5 * ((1.0 + y[0]) ** -2 - 1.0) + n_b]

    sol = solve_ivp(rhs, [0.0, float(xi_grid[-1])], [0.0, 0.0], t_eval=xi_grid, rtol=rtol,
                    atol=1e-15, method="DOP853")
    return sol.y[0], sol.y[1]
