"""Physics of the paper's small workloads measured on the GPU with the device
diagnostics, against the hand-linearised scheme and the oracle.

- Rayleigh-Taylor (config 1, Sec. III A): 128^2 hanging film, g = -1e-4,
  2000 steps.  The growth rate of the seeded mode, fitted from its Fourier
  amplitude (tf_lbm_diagnostics, mode (1, 0)) over steps 100..2000, must lie
  within 5% of the dominant eigenvalue of the linearised step
  (tests/linear_theory.py); a mode above k_c must decay at its own rate; the
  perturbation dh = h - h0 must match the oracle's (FP64 1e-6, FP32 10%:
  see the test).  The growth over 2000 steps is only ~0.07% of the
  amplitude, far below the 1e-5 tolerance on h, which is why the rate is
  fitted from the mode sum.
- Sessile drop (config 2, Sec. III B): 512^2, r_b = 120, h_d = 20, theta =
  20 deg, delta in {1, 2}, 50k steps FP32.  The apparent angle from the
  wetted area and apex (threshold h* + 0.01 h_d) must relax into
  [19.15, 20] deg +- 1 deg: the small-slope first integral of the film
  equation gives tan(theta_app) = 2 sin(theta / 2), i.e. 19.15 deg at 20 deg.
"""
import math
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1810_07642_gb300 import inputs
from paper_1810_07642_gb300 import diagnostics as D
from paper_1810_07642_gb300.film import ThinFilm

sys.path.insert(0, os.path.dirname(__file__))
import linear_theory as LT  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1810_07642_gb300 import build
    build.build()
    O.set_num_threads(os.cpu_count() or 1)
    assert torch.cuda.is_available()


def cfg_of(p):
    return O.Config(**{k: v for k, v in p.items() if k in O.Config.__dataclass_fields__})


def fitted_rate(sim, mode, steps=2000, every=100, skip=100):
    ts, la = [], []
    for t in range(0, steps + 1, every):
        if t:
            sim.step(every)
        if t >= skip:
            row = sim.diagnostics(0.0, mode=(mode, 0)).cpu().numpy()
            ts.append(t)
            la.append(math.log(D.mode_amplitude(row, sim.nx, sim.ny)))
    return np.polyfit(ts, la, 1)[0]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("mode", [1, 8])
def test_rayleigh_taylor_growth_rate(dtype, mode):
    h0, th, p = inputs.rayleigh_taylor(128, mode=mode, g=-1e-4)
    sim = ThinFilm(p, h0, th, dtype=dtype)
    sig = fitted_rate(sim, mode)
    k = 2 * math.pi * mode / 128
    ref = LT.scheme_growth_rate(k, 1.0, -1e-4, 0.01, 1.0, 0.0)
    assert (sig > 0) == (mode == 1)
    assert abs(sig - ref) <= 0.05 * abs(ref), (sig, ref)
    if mode == 1:
        # The perturbation itself against the oracle, both started from the
        # h0 the run was given (rounded to FP32 in FP32).  FP64: 1e-6 of
        # max |dh|.  FP32
        # cannot reach that: every step rounds the stored f_0 - href (up to
        # 2e-3 here) to 2^-24, ~1e-10, and the exact residual of that rounding
        # is carried to the neighbours in f_1 and f_5 (mass stays exact);
        # after 2000 steps these local displacements (measured 3e-8) are 6% of
        # dh ~ 5e-7, while the mode sum above averages them out.
        h32 = h0 if dtype == "f64" else h0.astype(np.float32).astype(np.float64)
        cfg = cfg_of(p)
        f = O.init(cfg, h32)
        O.step(cfg, O.kappa_field(cfg, th), f, 2000)
        dh_o = f.sum(0) - h32
        # h from the exported state (FP64 sums of the stored values): an
        # FP32 h near 1 would round dh ~ 5e-7 to 2^-24
        dh_g = sim.get_state().sum(0).cpu().numpy() - h32
        tol = 1e-6 if dtype == "f64" else 0.1
        assert np.abs(dh_g - dh_o).max() <= tol * np.abs(dh_o).max()
    sim.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rayleigh_taylor_second_order_forcing_matches_eq_rtgrowth(dtype):
    """Config 1 with the second-order-forcing reading (forcing = 1): the
    seeded mode's growth rate on the GPU lies within 5% of Eq. (RTgrowth),
    3.658e-7 per step (Sec. III A), and within 1% of that reading's own
    linearisation; the printed reading's rate is 0.67 of it (test above)."""
    h0, th, p = inputs.rayleigh_taylor(128, mode=1, g=-1e-4)
    p = dict(p, forcing=1)
    sim = ThinFilm(p, h0, th, dtype=dtype)
    sig = fitted_rate(sim, 1)
    sim.close()
    k = 2 * math.pi / 128
    eq = LT.rt_growth_rate(k, 1.0, 1e-4, 0.01, 1.0 / 6.0)
    lin = LT.scheme_growth_rate(k, 1.0, -1e-4, 0.01, 1.0, 0.0, forcing=1)
    assert abs(sig / eq - 1) <= 0.05, (sig, eq)
    assert abs(sig / lin - 1) <= 0.01, (sig, lin)


@pytest.mark.parametrize("delta", [1.0, 2.0])
def test_sessile_drop_relaxes_to_the_equilibrium_angle(delta):
    h0, th, p = inputs.sessile_drop(512, rb=120.0, hd=20.0, theta_deg=20.0, delta=delta)
    p = dict(p, theta_uniform=math.radians(20.0))
    sim = ThinFilm(p, h0, None, dtype="f32")
    m0 = sim.mass()
    sim.step(50000)
    assert sim.check() == 0
    hd = sim.diagnostics(p["hstar"]).cpu().numpy()[5] - p["hstar"]
    row = sim.diagnostics(p["hstar"] + 0.01 * hd).cpu().numpy()
    g = D.drop(row, p["hstar"], 512, 512, p["tau"], p["gamma"])
    theta = math.degrees(g["theta"])
    assert 19.15 - 1.0 <= theta <= 20.0 + 1.0, theta
    assert abs(sim.mass() - m0) <= 1e-6 * m0
    sim.close()
