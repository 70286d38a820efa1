"""Seeded synthetic workloads shaped like the paper's simulations.

This module only draws inputs: initial film heights h0(x, y), wettability
fields theta(x, y) in radians and the physical parameters of each run.  It
holds none of the method's arithmetic, so both the CUDA library's tests and
the CPU oracle may take their inputs from it.  All arrays are float64,
shape (ny, nx), x fastest; randomness comes from numpy.random.default_rng(seed).

Workloads (paper sections in brackets):
  rayleigh_taylor      128^2 hanging film with one sinusoidal mode [Sec. III A]
  sessile_drop         512^2 spherical-cap drop on a precursor film [Sec. III B]
  patterned_dewetting  2048^2 noisy film on a striped + patched substrate [Sec. III D]
  sliding_drops        64 uneven domains, drop under a tangential force [Sec. III C]
  inverse_design       512^2 noisy film, noisy theta and an 8-drop target
Parameters that the paper does not state for a workload take gamma = 0.01,
h_* = 0.07, (n, m) = (3, 2), tau = 1, g = 0 and slip length delta = 1.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULTS = dict(tau=1.0, gamma=0.01, g=0.0, delta=1.0, hstar=0.07,
                n_exp=3, m_exp=2, pi_sign=1, gx_body=0.0, gy_body=0.0)


def _params(nx, ny, **over):
    p = dict(DEFAULTS)
    p.update(over)
    p["nx"], p["ny"] = int(nx), int(ny)
    return p


def rayleigh_taylor(n: int = 128, ny: int | None = None, amp: float = 1e-3,
                    mode: int = 1, g: float = -1e-4, gamma: float = 0.01,
                    seed: int = 0):
    """Flat film h0 = 1 hanging under gravity (g < 0) plus one sinusoidal mode
    of amplitude ``amp`` and wavenumber 2 pi mode / n along x with a seeded
    phase.  No disjoining pressure (theta = 0), no-slip friction (delta = 0)."""
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    phase = rng.uniform(0.0, 2.0 * math.pi)
    x = np.arange(n, dtype=np.float64)
    row = 1.0 + amp * np.sin(2.0 * math.pi * mode * x / n + phase)
    h0 = np.ascontiguousarray(np.broadcast_to(row, (ny, n)))
    theta = np.zeros((ny, n))
    p = _params(n, ny, g=g, gamma=gamma, delta=0.0)
    p["phase"] = phase
    p["mode"] = mode
    return h0, theta, p


def spherical_cap(nx: int, ny: int, cx: float, cy: float, rb: float, hd: float,
                  hstar: float) -> np.ndarray:
    """Spherical cap of base radius rb and apex height hd centred at (cx, cy),
    on a precursor film hstar: h = max(hstar, sqrt(R^2 - r^2) - (R - hd)) with
    R = (rb^2 + hd^2) / (2 hd) (periodic distance)."""
    R = (rb * rb + hd * hd) / (2.0 * hd)
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    dx = np.abs(x[None, :] - cx)
    dx = np.minimum(dx, nx - dx)
    dy = np.abs(y[:, None] - cy)
    dy = np.minimum(dy, ny - dy)
    r2 = dx * dx + dy * dy
    cap = np.sqrt(np.maximum(R * R - r2, 0.0)) - (R - hd)
    return np.ascontiguousarray(np.maximum(cap, hstar))


def sessile_drop(n: int = 512, rb: float = 120.0, hd: float = 20.0,
                 theta_deg: float = 20.0, delta: float = 1.0, hstar: float = 0.07,
                 seed: int = 0):
    """Spherical-cap drop (base radius rb, apex height hd) in the middle of an
    n x n periodic domain on a precursor film; uniform contact angle."""
    h0 = spherical_cap(n, n, n / 2.0, n / 2.0, rb, hd, hstar)
    theta = np.full((n, n), math.radians(theta_deg))
    p = _params(n, n, delta=delta, hstar=hstar)
    p.update(rb=rb, hd=hd, theta_deg=theta_deg)
    return h0, theta, p


def patterned_theta(nx: int, ny: int, period: int = 256, lo_deg: float = 10.0,
                    hi_deg: float = 40.0, n_patches: int = 32, rmin: float = 16.0,
                    rmax: float = 64.0, rng=None) -> np.ndarray:
    """Stripes along x (first half of each period at lo_deg, second half at
    hi_deg) plus n_patches seeded discs at lo_deg (periodic distance)."""
    rng = np.random.default_rng(0) if rng is None else rng
    x = np.arange(nx)
    stripe = np.where((x % period) < period // 2, lo_deg, hi_deg).astype(np.float64)
    th = np.ascontiguousarray(np.broadcast_to(stripe, (ny, nx)))
    xs = np.arange(nx, dtype=np.float64)
    ys = np.arange(ny, dtype=np.float64)
    for _ in range(n_patches):
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        r = rng.uniform(rmin, rmax)
        dx = np.abs(xs[None, :] - cx)
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(ys[:, None] - cy)
        dy = np.minimum(dy, ny - dy)
        th[dx * dx + dy * dy <= r * r] = lo_deg
    return np.radians(th)


def patterned_dewetting(n: int = 2048, ny: int | None = None, noise: float = 1e-2,
                        period: int = 256, n_patches: int = 32, seed: int = 0):
    """Film h0 = 1 + U(-noise, noise) on a chemically patterned substrate:
    stripes of period ``period`` (10 and 40 degrees) plus seeded discs at 10
    degrees with radii U[16, 64] (scaled down on small domains)."""
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    h0 = 1.0 + rng.uniform(-noise, noise, size=(ny, n))
    scale = min(1.0, min(n, ny) / 2048.0 * 4.0)
    theta = patterned_theta(n, ny, period=max(2, min(period, n)), n_patches=n_patches,
                            rmin=max(1.0, 16.0 * scale), rmax=max(2.0, 64.0 * scale),
                            rng=rng)
    p = _params(n, ny)
    return np.ascontiguousarray(h0), theta, p


def sliding_drops(count: int = 64, theta_deg: float = 40.0, bo_min: float = 0.05,
                  bo_max: float = 1.0, seed: int = 0, lx_range=(256, 1024)):
    """``count`` independent domains of uneven size (Lx a multiple of 64 in
    lx_range, Ly = Lx / 2), each with a spherical-cap drop of seeded base
    radius U[40, 80] (capped at 0.4 Ly) and contact angle theta_deg, driven
    along x by a tangential body acceleration set by a Bond number; the Bond
    numbers are log-spaced over [bo_min, bo_max].  Returns a list of
    (h0, theta, params)."""
    rng = np.random.default_rng(seed)
    bos = np.logspace(math.log10(bo_min), math.log10(bo_max), count)
    th = math.radians(theta_deg)
    out = []
    for i in range(count):
        lx = int(rng.integers(lx_range[0] // 64, lx_range[1] // 64 + 1)) * 64
        ly = lx // 2
        rb = float(rng.uniform(40.0, 80.0))
        rb = min(rb, 0.4 * ly)
        R = rb / math.sin(th)
        hd = R * (1.0 - math.cos(th))
        hstar = DEFAULTS["hstar"]
        h0 = spherical_cap(lx, ly, lx / 2.0, ly / 2.0, rb, hd, hstar)
        vol = math.pi / 3.0 * R ** 3 * (2.0 + math.cos(th)) * (1.0 - math.cos(th)) ** 2
        # Bo = (3V / 4 pi)^(2/3) rho g sin(alpha) / gamma, rho = 1
        gpar = bos[i] * DEFAULTS["gamma"] / (3.0 * vol / (4.0 * math.pi)) ** (2.0 / 3.0)
        p = _params(lx, ly, delta=1.0, gx_body=gpar)
        p.update(bond=float(bos[i]), rb=rb, volume=vol)
        out.append((h0, np.full((ly, lx), th), p))
    return out


def inverse_design(n: int = 512, noise: float = 1e-2, theta0_deg: float = 30.0,
                   theta_sd_deg: float = 5.0, n_drops: int = 8, seed: int = 0):
    """Noisy flat film, noisy initial wettability and a target film shaped as
    n_drops seeded Gaussian bumps of the same mean height."""
    rng = np.random.default_rng(seed)
    h0 = 1.0 + rng.uniform(-noise, noise, size=(n, n))
    theta = np.radians(theta0_deg + theta_sd_deg * rng.standard_normal((n, n)))
    x = np.arange(n, dtype=np.float64)
    tgt = np.zeros((n, n))
    for _ in range(n_drops):
        cx, cy = rng.uniform(0, n), rng.uniform(0, n)
        s = rng.uniform(n / 32.0, n / 16.0)
        dx = np.abs(x[None, :] - cx)
        dx = np.minimum(dx, n - dx)
        dy = np.abs(x[:, None] - cy)
        dy = np.minimum(dy, n - dy)
        tgt += np.exp(-(dx * dx + dy * dy) / (2.0 * s * s))
    tgt = tgt * (h0.mean() * n * n / tgt.sum())
    p = _params(n, n)
    return np.ascontiguousarray(h0), theta, np.ascontiguousarray(tgt), p


def small_random(nx: int, ny: int, seed: int = 0, amp: float = 0.05,
                 theta_lo_deg: float = 10.0, theta_hi_deg: float = 40.0, **over):
    """Small generic case for parity tests: h0 = 1 + U(-amp, amp), theta
    uniform in [theta_lo, theta_hi] degrees per node."""
    rng = np.random.default_rng(seed)
    h0 = 1.0 + rng.uniform(-amp, amp, size=(ny, nx))
    theta = np.radians(rng.uniform(theta_lo_deg, theta_hi_deg, size=(ny, nx)))
    return np.ascontiguousarray(h0), theta, _params(nx, ny, **over)
