"""Derived film diagnostics from the device reductions of tf_lbm_diagnostics.

The reductions (sums over the lattice and over the wetted nodes) run on the
GPU; what is left here is a handful of scalar formulas per film:

- contact radius, cap radius and apparent contact angle of a spherical-cap
  drop (Sec. III B): r = sqrt(A / pi), h_d = h_max - h_*,
  R = (r^2 + h_d^2) / (2 h_d), theta = 2 atan(h_d / r) (the same angle as
  arcsin(r / R) for a cap, and well defined past 90 degrees);
- the drop's centre on the periodic lattice from the circular first moments;
- sliding velocity U = sum_W j_x / sum_W h and capillary number
  Ca = nu U / gamma with rho = 1 (Sec. III C);
- amplitude of a single Fourier mode of h (Sec. III A):
  2 |sum h e^{i phi}| / (nx ny).
"""
from __future__ import annotations

import math

import numpy as np

from ._lib import DIAG_FIELDS

_IX = {k: i for i, k in enumerate(DIAG_FIELDS)}


def as_dict(row) -> dict:
    """One tf_lbm_diag row (any array-like of 12 numbers) as a dict."""
    row = np.asarray(row, dtype=np.float64).reshape(-1)
    return {k: float(row[i]) for k, i in _IX.items()}


def drop(row, hstar: float, nx: int, ny: int, tau: float, gamma: float) -> dict:
    """Geometry and motion of the drop described by one diagnostics row."""
    d = as_dict(row)
    r = math.sqrt(d["wet_area"] / math.pi)
    hd = d["h_max"] - hstar
    theta = 2.0 * math.atan2(hd, r) if r > 0 else float("nan")
    cap_r = (r * r + hd * hd) / (2.0 * hd) if hd > 0 else float("inf")
    cx = (math.atan2(d["wet_sin_x"], d["wet_cos_x"]) / (2 * math.pi)) % 1.0 * nx
    cy = (math.atan2(d["wet_sin_y"], d["wet_cos_y"]) / (2 * math.pi)) % 1.0 * ny
    ux = d["wet_jx"] / d["wet_mass"] if d["wet_mass"] > 0 else 0.0
    uy = d["wet_jy"] / d["wet_mass"] if d["wet_mass"] > 0 else 0.0
    nu = (tau - 0.5) / 3.0
    return {"contact_radius": r, "apex": hd, "cap_radius": cap_r, "theta": theta,
            "centre_x": cx, "centre_y": cy, "ux": ux, "uy": uy, "ca": nu * ux / gamma}


def mode_amplitude(row, nx: int, ny: int) -> float:
    """Amplitude of the Fourier mode the row was reduced at."""
    d = as_dict(row)
    return 2.0 * math.hypot(d["mode_cos"], d["mode_sin"]) / (nx * ny)
