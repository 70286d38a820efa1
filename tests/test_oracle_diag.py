"""Pins of the oracle's film diagnostics and appendix term norms against
closed forms (no GPU).

States are built as f_l = f_eq_l(h, u) (Eq. equilibria, g = 0), whose moments
are h and h u exactly (the constraints pinned in test_oracle_pins), so each
diagnostic can be predicted from the chosen h and u fields alone:
  - the stencils of Eqs. (derivative) and (n_laplace) act on e^{i k x} as
    i sin(k) and 2 (cos k - 1) (a one-dimensional wave; the diagonal terms
    fold in), so every term of the appendix balance has a closed form for a
    single Fourier mode;
  - Fourier sums of a single mode are exact discrete orthogonality;
  - the circular first moments of a bump centred at (x0, y0) point at x0, y0;
  - a spherical cap satisfies tan(theta / 2) = h_d / r (Sec. III B geometry).
"""
import math

import numpy as np
import pytest

import oracle as O


def state(h, ux, uy):
    ny, nx = h.shape
    f = np.empty((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f[:, y, x] = O.feq(0.0, h[y, x], ux[y, x], uy[y, x])
    return f


def cfg(nx, ny, **kw):
    d = dict(nx=nx, ny=ny, tau=0.8, gamma=0.01, g=0.0, delta=1.0, hstar=0.07, n_exp=3, m_exp=2)
    d.update(kw)
    return O.Config(**d)


def test_fourier_sums_of_a_single_mode():
    nx, ny, a = 24, 16, 0.3
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    phase = 2 * np.pi * (3 * X / nx + 2 * Y / ny)
    h = 1.0 + a * np.cos(phase + 0.4)
    f = state(h, np.zeros_like(h), np.zeros_like(h))
    d = O.film_diagnostics(cfg(nx, ny), f, 0.5, mode=(3, 2))
    N = nx * ny
    # sum h e^{i phi} = a N / 2 e^{-0.4 i}
    assert abs(d[10] - a * N / 2 * math.cos(0.4)) < 1e-10
    assert abs(d[11] + a * N / 2 * math.sin(0.4)) < 1e-10
    assert abs(d[0] - N) < 1e-10
    # another mode sees nothing
    d2 = O.film_diagnostics(cfg(nx, ny), f, 0.5, mode=(1, 0))
    assert abs(d2[10]) < 1e-10 and abs(d2[11]) < 1e-10


def test_wetted_sums_centre_and_apex():
    nx, ny = 40, 30
    x0, y0 = 31.0, 6.0
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    dx = (X - x0 + nx / 2) % nx - nx / 2
    dy = (Y - y0 + ny / 2) % ny - ny / 2
    h = 0.07 + np.maximum(0.0, 2.0 - (dx ** 2 + dy ** 2) / 20.0)
    u = 1e-3
    f = state(h, np.full_like(h, u), np.zeros_like(h))
    d = O.film_diagnostics(cfg(nx, ny), f, 0.1)
    w = h > 0.1
    assert d[4] == w.sum()
    assert abs(d[1] - h[w].sum()) < 1e-11
    assert abs(d[2] - u * h[w].sum()) < 1e-12 and abs(d[3]) < 1e-12
    assert d[5] == pytest.approx(2.07, abs=1e-12)
    cx = (math.atan2(d[7], d[6]) / (2 * math.pi)) % 1.0 * nx
    cy = (math.atan2(d[9], d[8]) / (2 * math.pi)) % 1.0 * ny
    assert cx == pytest.approx(x0, abs=1e-9) and cy == pytest.approx(y0, abs=1e-9)


def test_term_norm_pressure_of_a_capillary_wave():
    """kappa = 0, u = 0, h = 1 + a cos(kx): p = -2 gamma (cos k - 1) a cos(kx),
    -h d_x p = -2 gamma a (cos k - 1) sin k (1 + a cos kx) sin kx, whose mean
    square is (2 gamma a (cos k - 1) sin k)^2 (1/2 + a^2/8)."""
    nx, ny, a, m = 32, 4, 0.2, 3
    k = 2 * np.pi * m / nx
    X, _ = np.meshgrid(np.arange(nx), np.arange(ny))
    h = 1.0 + a * np.cos(k * X)
    c = cfg(nx, ny)
    f = state(h, np.zeros_like(h), np.zeros_like(h))
    tn = O.term_norms(c, np.zeros((ny, nx)), f)
    expect = abs(2 * c.gamma * a * (math.cos(k) - 1) * math.sin(k)) * math.sqrt(0.5 + a * a / 8)
    assert tn[0] == pytest.approx(expect, rel=1e-10)
    assert tn[1] < 1e-15 and tn[2] < 1e-15


def test_term_norms_friction_and_dissipation_of_shear_and_compression():
    nx, ny, b, m = 16, 32, 1e-3, 2
    c = cfg(nx, ny)
    nu = (c.tau - 0.5) / 3
    al = 6.0 / (2.0 + 6.0 * c.delta + 3.0 * c.delta ** 2)  # Eq. (alphafric) at h = 1
    # shear u_x = b cos(k y): div j = 0, lap j_x = 2 (cos k - 1) j_x
    k = 2 * np.pi * m / ny
    _, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    h = np.ones((ny, nx))
    f = state(h, b * np.cos(k * Y), np.zeros_like(h))
    tn = O.term_norms(c, np.zeros((ny, nx)), f)
    assert tn[0] < 1e-15
    assert tn[1] == pytest.approx(nu * al * b / math.sqrt(2), rel=1e-9)
    assert tn[2] == pytest.approx(nu * 2 * (1 - math.cos(k)) * b / math.sqrt(2), rel=1e-9)
    # compression u_x = b cos(k x): d_x div j = -sin^2(k) j_x as well
    k = 2 * np.pi * m / nx
    X, _ = np.meshgrid(np.arange(nx), np.arange(ny))
    f = state(h, b * np.cos(k * X), np.zeros_like(h))
    tn = O.term_norms(c, np.zeros((ny, nx)), f)
    sym = 2 * (math.cos(k) - 1) - 2 * math.sin(k) ** 2
    assert tn[2] == pytest.approx(nu * abs(sym) * b / math.sqrt(2), rel=1e-9)


@pytest.mark.parametrize("r,hd", [(30.0, 10.0), (12.0, 3.0), (5.0, 9.0)])
def test_drop_geometry_matches_cap_identity(r, hd):
    rr, R, th = O.drop_geometry(math.pi * r * r, hd + 0.07, 0.07)
    assert rr == pytest.approx(r, rel=1e-14)
    assert R == pytest.approx((r * r + hd * hd) / (2 * hd), rel=1e-14)
    assert math.tan(th / 2) == pytest.approx(hd / r, rel=1e-12)
