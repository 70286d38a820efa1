"""Pins of the oracle's hand-derived adjoint against central finite
differences of the oracle's forward step (FP64).  The adjoint is the exact
derivative of the discrete scheme, so the two must agree to the truncation
and rounding error of the difference quotient (~1e-8 relative here)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1810_07642_gb300 import inputs


def cfg_of(p, **over):
    d = {k: v for k, v in p.items() if k in O.Config.__dataclass_fields__}
    d.update(over)
    return O.Config(**d)


def _forward_loss(cfg, h0, theta, nsteps, r):
    f = O.init(cfg, h0)
    O.step(cfg, O.kappa_field(cfg, theta), f, nsteps)
    return float((r * f).sum())


CASES = [
    dict(tau=1.0, g=0.0, delta=1.0, gx_body=0.0, pi_sign=1),
    dict(tau=0.8, g=3e-3, delta=0.4, gx_body=2e-4, gy_body=-1e-4, pi_sign=1),
    dict(tau=1.3, g=-2e-3, delta=2.0, pi_sign=-1, n_exp=9, m_exp=3),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_adjoint_matches_central_differences(case):
    nx, ny, T = 7, 6, 5
    h0, th, p = inputs.small_random(nx, ny, seed=case + 20, amp=0.3)
    p.update(CASES[case])
    cfg = cfg_of(p)
    rng = np.random.default_rng(case)
    r = rng.standard_normal((9, ny, nx))  # a random linear functional of f(T)
    L, gth, gh0, gk = O.loss_gradient(cfg, h0, th, T, lambda f: (float((r * f).sum()), r.copy()))
    assert abs(L - _forward_loss(cfg, h0, th, T, r)) < 1e-12 * abs(L)
    scale = max(np.abs(gth).max(), np.abs(gh0).max())
    for _ in range(6):
        y, x = rng.integers(0, ny), rng.integers(0, nx)
        for which, grad in (("theta", gth), ("h0", gh0)):
            eps = 1e-6
            hp, hm, tp, tm = h0.copy(), h0.copy(), th.copy(), th.copy()
            if which == "theta":
                tp[y, x] += eps
                tm[y, x] -= eps
            else:
                hp[y, x] += eps
                hm[y, x] -= eps
            fd = (_forward_loss(cfg, hp, tp, T, r) - _forward_loss(cfg, hm, tm, T, r)) / (2 * eps)
            assert abs(fd - grad[y, x]) <= 1e-7 * scale + 1e-9 * abs(fd), (which, y, x, fd, grad[y, x])


def test_adjoint_of_height_loss_on_drop():
    """L = 1/2 sum (h_T - target)^2 on a small drop (the shape loss of the
    inverse-design workload): dL/df_l(T) = h_T - target for every l."""
    h0, th, p = inputs.sessile_drop(16, rb=5.0, hd=1.5, theta_deg=25.0, delta=1.0)
    th = th + np.radians(5) * np.random.default_rng(3).standard_normal(th.shape)
    cfg = cfg_of(p)
    tgt = np.random.default_rng(4).uniform(0.05, 1.5, h0.shape)

    def seed(f):
        h = f.sum(0)
        return 0.5 * float(((h - tgt) ** 2).sum()), np.broadcast_to(h - tgt, f.shape).copy()

    T = 8
    L, gth, gh0, _ = O.loss_gradient(cfg, h0, th, T, seed)

    def loss(h0_, th_):
        f = O.init(cfg, h0_)
        O.step(cfg, O.kappa_field(cfg, th_), f, T)
        return 0.5 * float(((f.sum(0) - tgt) ** 2).sum())

    rng = np.random.default_rng(5)
    scale = np.abs(gth).max()
    for _ in range(8):
        y, x = rng.integers(0, 16), rng.integers(0, 16)
        eps = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[y, x] += eps
        tm[y, x] -= eps
        fd = (loss(h0, tp) - loss(h0, tm)) / (2 * eps)
        assert abs(fd - gth[y, x]) <= 1e-6 * scale, (y, x, fd, gth[y, x])
