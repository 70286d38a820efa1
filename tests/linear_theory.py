"""Closed-form linear theory used to pin the oracle (test helper).

Two independent predictions of how a small sinusoidal perturbation
h = h0 + eps cos(k x) of a flat film evolves:

* ``scheme_growth_rate``: the exact linearisation of one step of the lattice
  Boltzmann scheme of Section II (and of the labelled second-order-forcing
  alternative, ``forcing=1``) (Eq. LBE with the equilibria, the force of
  Eq. force and the stencils of Eqs. derivative / n_laplace) for a mode that
  is uniform in y.  Grouping the nine populations by c_x in {-1, 0, +1} makes
  the linearised step a 3 x 3 matrix; its dominant eigenvalue mu gives the
  growth rate ln|mu| per step.  The derivation is done by hand here, from
  the scheme's definition, not from the oracle's code:
    group sums of the equilibria about (h0, u = 0):
      A0_eq = h - g h^2 / 2           -> (1 - g h0) h'
      A+_eq = g h^2 / 4 + h u / 2     -> (g h0 / 2) h' + q' / 2
      A-_eq = g h^2 / 4 - h u / 2     -> (g h0 / 2) h' - q' / 2
    source 3 w_l c_l . F summed per group: +F/2, 0, -F/2
    force   F' = -lambda q' - i h0 sin(k) P h',  lambda = nu alpha(h0) / h0
    film pressure p' = P h', P = 2 gamma (1 - cos k) - s gamma kappa f'(h0)
    streaming multiplies A+ by exp(-i k) and A- by exp(+i k).
* ``lubrication_growth_rate``: the continuum result of linearising the
  quasi-steady Eq. (hydro2) (friction-dominated, inertia dropped) including
  the longitudinal viscous terms; with no disjoining pressure and delta = 0
  and k h0 -> 0 it is Eq. (RTgrowth).
"""
from __future__ import annotations

import math

import numpy as np


def alpha(h: float, delta: float) -> float:
    """Eq. (alphafric)."""
    return 6.0 * h / (2.0 * h * h + 6.0 * delta * h + 3.0 * delta * delta)


def fdisj_prime(h: float, n: int, m: int, hstar: float) -> float:
    """d/dh of (hstar/h)^n - (hstar/h)^m."""
    r = hstar / h
    return (-n * r ** n + m * r ** m) / h


def kappa(theta: float, n: int, m: int, hstar: float) -> float:
    return (1.0 - math.cos(theta)) * (n - 1) * (m - 1) / ((n - m) * hstar)


def pressure_symbol(k, gamma, kap=0.0, fprime=0.0, pi_sign=1):
    """p' / h' for the lattice Laplacian of a mode along x."""
    return 2.0 * gamma * (1.0 - math.cos(k)) - pi_sign * gamma * kap * fprime


def scheme_growth_rate(k, h0, g, gamma, tau, delta, kap=0.0, fprime=0.0, pi_sign=1, forcing=0):
    """forcing = 0: Eq. (LBE) as printed, u' = q'/h0 and the source 3 w_l c_l.F.
    forcing = 1: the second-order alternative, h0 u' = (q' + F_ext'/2) /
    (1 + lambda/2) (the friction -lambda h0 u' taken at that velocity) and
    the source scaled by (1 - omega/2) (its u.F terms are second order)."""
    omega = 1.0 / tau
    nu = (tau - 0.5) / 3.0
    lam = nu * alpha(h0, delta) / h0
    P = pressure_symbol(k, gamma, kap, fprime, pi_sign)
    s = math.sin(k)
    # order: (A-, A0, A+);  h' = A- + A0 + A+,  q' = A+ - A-
    Hrow = np.array([1.0, 1.0, 1.0], complex)
    Qrow = np.array([-1.0, 0.0, 1.0], complex)
    Fext = -1j * h0 * s * P * Hrow          # film-pressure force, linearised
    if forcing == 0:
        Urow = Qrow                          # h0 u'
        scale = 1.0
    else:
        Urow = (Qrow + 0.5 * Fext) / (1.0 + 0.5 * lam)
        scale = 1.0 - 0.5 * omega
    Eq = np.array([g * h0 / 2.0 * Hrow - 0.5 * Urow,
                   (1.0 - g * h0) * Hrow,
                   g * h0 / 2.0 * Hrow + 0.5 * Urow])
    Frow = -lam * Urow + Fext
    Src = scale * np.array([-0.5 * Frow, 0.0 * Frow, 0.5 * Frow])
    post = (1.0 - omega) * np.eye(3) + omega * Eq + Src
    stream = np.diag([np.exp(1j * k), 1.0, np.exp(-1j * k)])
    mu = np.linalg.eigvals(stream @ post)
    return math.log(np.max(np.abs(mu)))


def lubrication_growth_rate(k, h0, g, gamma, tau, delta, kap=0.0, fprime=0.0,
                            pi_sign=1, viscous=True):
    """sigma = -k^2 h0 (g + gamma k^2 - s gamma kappa f'(h0)) / (lambda + 3 nu k^2)."""
    nu = (tau - 0.5) / 3.0
    lam = nu * alpha(h0, delta) / h0
    P = gamma * k * k - pi_sign * gamma * kap * fprime
    damp = lam + (3.0 * nu * k * k if viscous else 0.0)
    return -k * k * h0 * (g + P) / damp


def rt_growth_rate(k, h0, g_abs, gamma, mu):
    """Eq. (RTgrowth): rho g h0^3 / (3 mu) (k^2 - l_cap^2 k^4), rho = 1."""
    lcap2 = gamma / g_abs
    return g_abs * h0 ** 3 / (3.0 * mu) * (k * k - lcap2 * k ** 4)
