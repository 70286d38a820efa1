"""FP64 CPU oracle of the thin-film D2Q9 lattice Boltzmann method.

Test infrastructure only.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The oracle shares no
code with the CUDA library, and the library never imports it.

The arithmetic lives in ``tflbm_oracle.c`` (plain C, double precision, built
with ``-ffp-contract=off``).  This module compiles it with gcc on first use
and wraps it with ctypes on numpy float64 arrays.  Populations are stored as
``f[l, y, x]`` (shape ``(9, ny, nx)``); fields are ``(ny, nx)`` with x fastest.
The method follows Section II of Zitz et al., arXiv:1810.07642: Eqs. (speeds),
(equilibria), (LBE), (force), (pfilm), (disjoiningP), (forcefric),
(alphafric), (derivative) and (n_laplace).  The readings of the garbled or
silent points are listed in the header of ``tflbm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tflbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in tflbm_oracle.c (same field order)."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("n_exp", ctypes.c_int32), ("m_exp", ctypes.c_int32),
        ("pi_sign", ctypes.c_int32), ("forcing", ctypes.c_int32),
        ("tau", ctypes.c_double), ("gamma", ctypes.c_double),
        ("g", ctypes.c_double), ("delta", ctypes.c_double),
        ("hstar", ctypes.c_double), ("gx_body", ctypes.c_double),
        ("gy_body", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)
_P = ctypes.POINTER(Params)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_lattice.argtypes = [_I, _I, _D]
        L.orc_feq.argtypes = [ctypes.c_double] * 4 + [_D]
        L.orc_laplacian.argtypes = [ctypes.c_int32, ctypes.c_int32, _D, _D]
        L.orc_gradient.argtypes = [ctypes.c_int32, ctypes.c_int32, _D, _D, _D]
        L.orc_kappa.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_double]
        L.orc_kappa.restype = ctypes.c_double
        L.orc_kappa_field.argtypes = [_P, _D, _D]
        L.orc_fdisj.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_double]
        L.orc_fdisj.restype = ctypes.c_double
        L.orc_alpha.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_alpha.restype = ctypes.c_double
        L.orc_moments.argtypes = [_P, _D, _D, _D, _D]
        L.orc_pressure_force.argtypes = [_P, _D, _D, _D, _D, _D]
        L.orc_init.argtypes = [_P, _D, _D]
        L.orc_step.argtypes = [_P, _D, _D, ctypes.c_int64]
        L.orc_mass.argtypes = [_P, _D]
        L.orc_mass.restype = ctypes.c_double
        L.orc_adjoint_step.argtypes = [_P, _D, _D, _D, _D, _D]
        L.orc_adjoint_init.argtypes = [_P, _D, _D, _D]
        L.orc_num_threads.restype = ctypes.c_int32
        L.orc_set_num_threads.argtypes = [ctypes.c_int32]
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


@dataclass
class Config:
    """Physical parameters of one run (lattice units, dx = dt = 1)."""
    nx: int
    ny: int
    tau: float = 1.0
    gamma: float = 0.01
    g: float = 0.0
    delta: float = 1.0
    hstar: float = 0.07
    n_exp: int = 3
    m_exp: int = 2
    pi_sign: int = 1
    gx_body: float = 0.0
    gy_body: float = 0.0
    # 0: Eq. (LBE) as printed (u = sum c f / h before collision, source
    # 3 w_l c_l.F); 1: the labelled second-order-forcing alternative (see the
    # header of tflbm_oracle.c), forward step only
    forcing: int = 0
    extra: dict = field(default_factory=dict)

    def cparams(self) -> Params:
        return Params(self.nx, self.ny, self.n_exp, self.m_exp, self.pi_sign, self.forcing,
                      self.tau, self.gamma, self.g, self.delta, self.hstar,
                      self.gx_body, self.gy_body)


def lattice():
    """Velocities c_l (Eq. speeds) and weights w_l as (cx, cy, w)."""
    cx = np.zeros(9, np.int32)
    cy = np.zeros(9, np.int32)
    w = np.zeros(9)
    lib().orc_lattice(cx.ctypes.data_as(_I), cy.ctypes.data_as(_I), _ptr(w))
    return cx, cy, w


def feq(g: float, h: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(g, h, ux, uy, _ptr(out))
    return out


def laplacian(phi: np.ndarray) -> np.ndarray:
    phi = np.ascontiguousarray(phi, np.float64)
    out = np.empty_like(phi)
    lib().orc_laplacian(phi.shape[1], phi.shape[0], _ptr(phi), _ptr(out))
    return out


def gradient(phi: np.ndarray):
    phi = np.ascontiguousarray(phi, np.float64)
    gx = np.empty_like(phi)
    gy = np.empty_like(phi)
    lib().orc_gradient(phi.shape[1], phi.shape[0], _ptr(phi), _ptr(gx), _ptr(gy))
    return gx, gy


def kappa(theta: float, n: int, m: int, hstar: float) -> float:
    return lib().orc_kappa(theta, n, m, hstar)


def kappa_field(cfg: Config, theta) -> np.ndarray:
    theta = np.broadcast_to(np.asarray(theta, np.float64), (cfg.ny, cfg.nx))
    theta = np.ascontiguousarray(theta)
    out = np.empty_like(theta)
    p = cfg.cparams()
    lib().orc_kappa_field(ctypes.byref(p), _ptr(theta), _ptr(out))
    return out


def fdisj(h: float, n: int, m: int, hstar: float) -> float:
    return lib().orc_fdisj(h, n, m, hstar)


def alpha(h: float, delta: float) -> float:
    return lib().orc_alpha(h, delta)


def init(cfg: Config, h0: np.ndarray) -> np.ndarray:
    """Post-streaming populations at t = 0: f_l = f_eq_l(h0, u = 0)."""
    h0 = np.ascontiguousarray(h0, np.float64)
    assert h0.shape == (cfg.ny, cfg.nx)
    f = np.empty((9, cfg.ny, cfg.nx))
    p = cfg.cparams()
    lib().orc_init(ctypes.byref(p), _ptr(h0), _ptr(f))
    return f


def step(cfg: Config, kap: np.ndarray, f: np.ndarray, nsteps: int) -> np.ndarray:
    """Advance f (modified in place and returned) by nsteps of Eq. (LBE)."""
    assert f.shape == (9, cfg.ny, cfg.nx) and f.dtype == np.float64 and f.flags.c_contiguous
    kap = np.ascontiguousarray(np.broadcast_to(np.asarray(kap, np.float64), (cfg.ny, cfg.nx)))
    p = cfg.cparams()
    lib().orc_step(ctypes.byref(p), _ptr(kap), _ptr(f), int(nsteps))
    return f


def moments(cfg: Config, f: np.ndarray):
    """(h, ux, uy) of the post-streaming populations f."""
    h = np.empty((cfg.ny, cfg.nx))
    ux = np.empty_like(h)
    uy = np.empty_like(h)
    p = cfg.cparams()
    lib().orc_moments(ctypes.byref(p), _ptr(f), _ptr(h), _ptr(ux), _ptr(uy))
    return h, ux, uy


def pressure_force(cfg: Config, kap: np.ndarray, f: np.ndarray):
    """(p_film, Fx, Fy) of the post-streaming populations f."""
    kap = np.ascontiguousarray(np.broadcast_to(np.asarray(kap, np.float64), (cfg.ny, cfg.nx)))
    pf = np.empty((cfg.ny, cfg.nx))
    fx = np.empty_like(pf)
    fy = np.empty_like(pf)
    p = cfg.cparams()
    lib().orc_pressure_force(ctypes.byref(p), _ptr(kap), _ptr(f), _ptr(pf), _ptr(fx), _ptr(fy))
    return pf, fx, fy


def mass(cfg: Config, f: np.ndarray) -> float:
    p = cfg.cparams()
    return lib().orc_mass(ctypes.byref(p), _ptr(f))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def adjoint_step(cfg: Config, kap: np.ndarray, f_t: np.ndarray, a_next: np.ndarray,
                 grad_kappa: np.ndarray):
    """dL/df(t) from dL/df(t+1) for the step taken from the post-streaming
    state f_t; adds the step's contribution to grad_kappa (in place)."""
    kap = np.ascontiguousarray(np.broadcast_to(np.asarray(kap, np.float64), (cfg.ny, cfg.nx)))
    if cfg.forcing != 0:
        raise ValueError("the oracle adjoint differentiates Eq. (LBE) as printed (forcing = 0) only")
    f_t = np.ascontiguousarray(f_t, np.float64)
    a_next = np.ascontiguousarray(a_next, np.float64)
    assert grad_kappa.flags.c_contiguous and grad_kappa.dtype == np.float64
    a = np.empty_like(a_next)
    p = cfg.cparams()
    lib().orc_adjoint_step(ctypes.byref(p), _ptr(kap), _ptr(f_t), _ptr(a_next), _ptr(a),
                           _ptr(grad_kappa))
    return a


def adjoint_init(cfg: Config, h0: np.ndarray, a0: np.ndarray) -> np.ndarray:
    """dL/dh0 from dL/df(0), for f(0) = f_eq(h0, 0)."""
    h0 = np.ascontiguousarray(h0, np.float64)
    out = np.empty_like(h0)
    p = cfg.cparams()
    lib().orc_adjoint_init(ctypes.byref(p), _ptr(h0), _ptr(np.ascontiguousarray(a0)), _ptr(out))
    return out


def dkappa_dtheta(cfg: Config, theta) -> np.ndarray:
    """d kappa / d theta of Eq. (disjoiningP): sin(theta) (n-1)(m-1)/((n-m) h_*)."""
    c = (cfg.n_exp - 1) * (cfg.m_exp - 1) / ((cfg.n_exp - cfg.m_exp) * cfg.hstar)
    return np.sin(np.asarray(theta, np.float64)) * c


def loss_gradient(cfg: Config, h0: np.ndarray, theta, nsteps: int, seed):
    """Reverse-mode gradient of a loss of the final post-streaming state.

    seed(f_T) -> (L, dL/df_T).  Keeps every intermediate state (small cases
    only).  Returns (L, dL/dtheta, dL/dh0, dL/dkappa)."""
    theta = np.ascontiguousarray(np.broadcast_to(np.asarray(theta, np.float64), (cfg.ny, cfg.nx)))
    kap = kappa_field(cfg, theta)
    states = [init(cfg, h0)]
    for _ in range(nsteps):
        states.append(step(cfg, kap, states[-1].copy(), 1))
    L, a = seed(states[-1])
    gk = np.zeros((cfg.ny, cfg.nx))
    for t in range(nsteps - 1, -1, -1):
        a = adjoint_step(cfg, kap, states[t], a, gk)
    gh0 = adjoint_init(cfg, h0, a)
    return L, gk * dkappa_dtheta(cfg, theta), gh0, gk


def run(cfg: Config, h0: np.ndarray, theta, nsteps: int):
    """Convenience: init from h0, advance nsteps, return (f, h, ux, uy)."""
    kap = kappa_field(cfg, theta)
    f = init(cfg, h0)
    step(cfg, kap, f, nsteps)
    h, ux, uy = moments(cfg, f)
    return f, h, ux, uy


# ---------------------------------------------------------------- diagnostics
# Plain definitions of the film diagnostics of Section III and the appendix,
# evaluated on a post-streaming state f (test infrastructure, like the rest).

DIAG_FIELDS = ("mass", "wet_mass", "wet_jx", "wet_jy", "wet_area", "h_max",
               "wet_cos_x", "wet_sin_x", "wet_cos_y", "wet_sin_y", "mode_cos", "mode_sin")


def film_diagnostics(cfg: Config, f: np.ndarray, h_wet: float, mode=(1, 0)) -> np.ndarray:
    """Film diagnostics of the state f, in the order of DIAG_FIELDS:
    sum of h over the lattice; over the wetted nodes W = {h > h_wet} the sums
    of h, of j = sum_l c_l f_l (two components) and of 1; the largest h; the
    circular first moments of the wetted film, sum_W h cos(2 pi x / nx),
    sum_W h sin(2 pi x / nx) and the same in y (the drop's position on the
    periodic lattice is their angle); and the Fourier sums of h over the
    whole lattice at the wave vector 2 pi (mx / nx, my / ny) (a single-mode
    amplitude, Sec. III A, is 2 |sum| / (nx ny)).  Section II gives h and j
    as the zeroth and first moments."""
    cx, cy, _ = lattice()
    h = f.sum(axis=0)
    jx = np.tensordot(cx.astype(np.float64), f, axes=1)
    jy = np.tensordot(cy.astype(np.float64), f, axes=1)
    w = h > h_wet
    ny, nx = h.shape
    ax = 2 * np.pi * np.arange(nx) / nx
    ay = 2 * np.pi * np.arange(ny) / ny
    hw = np.where(w, h, 0.0)
    mx, my = mode
    ph = 2 * np.pi * (mx * np.arange(nx)[None, :] / nx + my * np.arange(ny)[:, None] / ny)
    return np.array([
        h.sum(), hw.sum(), jx[w].sum(), jy[w].sum(), float(w.sum()), h.max(),
        (hw * np.cos(ax)[None, :]).sum(), (hw * np.sin(ax)[None, :]).sum(),
        (hw * np.cos(ay)[:, None]).sum(), (hw * np.sin(ay)[:, None]).sum(),
        (h * np.cos(ph)).sum(), (h * np.sin(ph)).sum()])


def term_norms(cfg: Config, kap: np.ndarray, f: np.ndarray) -> np.ndarray:
    """L2 norms, ||phi||_2 = (sum phi^2 / (nx ny))^(1/2) (appendix, Eq.
    magnitude), of the x-components of the three momentum terms the appendix
    compares: the film-pressure term -h d_x p, the friction -nu alpha(h) u_x
    (Eqs. forcefric, alphafric) and the longitudinal dissipation
    nu lap(h u_x) + 2 nu d_x(div(h u)).  p is the film pressure of Eq.
    (pfilm); d_x and div use the gradient stencil of Eq. (derivative) and lap
    the Laplacian of Eq. (n_laplace), each a pinned oracle routine."""
    h, ux, uy = moments(cfg, f)
    p, _, _ = pressure_force(cfg, kap, f)
    nu = (cfg.tau - 0.5) / 3.0
    a = np.vectorize(lambda hh: alpha(hh, cfg.delta))(h)
    jx, jy = h * ux, h * uy
    div = gradient(jx)[0] + gradient(jy)[1]
    terms = (-h * gradient(p)[0], -nu * a * ux, nu * laplacian(jx) + 2 * nu * gradient(div)[0])
    return np.array([np.sqrt((t ** 2).mean()) for t in terms])


def drop_geometry(wet_area: float, h_apex: float, hstar: float):
    """Contact radius, cap radius and contact angle of a spherical-cap drop
    (Sec. III B): r = sqrt(A / pi) from the wetted area, apex height
    h_d = h_max - h_*, R = (r^2 + h_d^2) / (2 h_d) and theta = arcsin(r / R)
    (pi - arcsin when h_d > r)."""
    r = np.sqrt(wet_area / np.pi)
    hd = h_apex - hstar
    R = (r * r + hd * hd) / (2 * hd)
    th = np.arcsin(np.clip(r / R, -1.0, 1.0))
    return r, R, (np.pi - th) if hd > r else th
