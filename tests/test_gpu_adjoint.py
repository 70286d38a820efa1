"""GPU adjoint (tf_lbm_adjoint_step, gradient tape, autograd Function)
against the FP64 oracle adjoint and against central finite differences.

Tolerances: one adjoint step in FP64 agrees with the oracle to 1e-10
relative (summation order only); in FP32 to 1e-4 of the largest entry (the
adjoint mixes terms of very different size, e.g. 1/h^2 in the equilibrium
derivatives).  Whole gradients through the tape in FP64 agree with the oracle
driver to 1e-9 and with central differences of the GPU FP64 forward to 1e-4,
the bound the inverse-design workload asks for.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1810_07642_gb300 import _lib as L
from paper_1810_07642_gb300 import inputs
from paper_1810_07642_gb300.adjoint import evolve
from paper_1810_07642_gb300.film import FilmBatch, ThinFilm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1810_07642_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def cfg_of(p, **over):
    d = {k: v for k, v in p.items() if k in O.Config.__dataclass_fields__}
    d.update(over)
    return O.Config(**d)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 1e-4)])
@pytest.mark.parametrize("case", [dict(tau=1.0, g=0.0), dict(tau=0.8, g=2e-3, gx_body=1e-4, delta=0.5),
                                  dict(tau=1.2, g=-1e-3, pi_sign=-1, n_exp=9, m_exp=3)])
def test_adjoint_step_matches_oracle(dtype, tol, case):
    nx, ny = 37, 29
    h0, th, p = inputs.small_random(nx, ny, seed=3, amp=0.2)
    p.update(case)
    cfg = cfg_of(p)
    kap = O.kappa_field(cfg, th)
    f = O.init(cfg, h0)
    O.step(cfg, kap, f, 7)
    a_next = np.random.default_rng(1).standard_normal((9, ny, nx))
    gk_o = np.zeros((ny, nx))
    a_o = O.adjoint_step(cfg, kap, f, a_next, gk_o)

    sim = ThinFilm(p, h0, th, dtype=dtype)
    td = sim.tdtype
    ft = torch.as_tensor(f, dtype=td, device="cuda").contiguous()
    an = torch.as_tensor(a_next, dtype=td, device="cuda").contiguous()
    at = torch.empty_like(an)
    gk = torch.zeros((ny, nx), dtype=td, device="cuda")
    L.tf_lbm_adjoint_step(sim.handle, ft.data_ptr(), an.data_ptr(), at.data_ptr(), gk.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    a_g = at.double().cpu().numpy()
    gk_g = gk.double().cpu().numpy()
    assert np.abs(a_g - a_o).max() <= tol * np.abs(a_o).max()
    assert np.abs(gk_g - gk_o).max() <= tol * np.abs(gk_o).max()


def _oracle_grads(p, h0, th, T, tgt):
    cfg = cfg_of(p)

    def seed(f):
        h = f.sum(0)
        return 0.5 * float(((h - tgt) ** 2).sum()), np.broadcast_to(h - tgt, f.shape).copy()

    return O.loss_gradient(cfg, h0, th, T, seed)


@pytest.mark.parametrize("every", [7, 0, 100])
def test_tape_gradient_matches_oracle_fp64(every):
    """Checkpoint segments of 7 (with a partial last one), sqrt(T), and one
    segment for the whole run all give the oracle's gradient."""
    h0, th, p = inputs.small_random(40, 32, seed=5, amp=0.1)
    p.update(tau=0.9, g=1e-3, delta=0.8)
    T = 30
    tgt = np.random.default_rng(2).uniform(0.9, 1.1, h0.shape)
    L_o, gth_o, gh0_o, _ = _oracle_grads(p, h0, th, T, tgt)
    theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    hh = torch.tensor(h0, dtype=torch.float64, device="cuda", requires_grad=True)
    h_t = evolve(theta, hh, p, T, dtype="f64", every=every)
    tg = torch.tensor(tgt, device="cuda")
    loss = 0.5 * ((h_t - tg) ** 2).sum()
    loss.backward()
    assert abs(loss.item() - L_o) <= 1e-11 * abs(L_o)
    gth = theta.grad.cpu().numpy()
    gh0 = hh.grad.cpu().numpy()
    assert np.abs(gth - gth_o).max() <= 1e-9 * np.abs(gth_o).max()
    assert np.abs(gh0 - gh0_o).max() <= 1e-9 * np.abs(gh0_o).max()


def test_gradient_matches_central_differences_inverse_design():
    """The inverse-design workload shape (noisy film, noisy theta, 8-drop
    target, L2 loss), reduced to 128^2 and 300 steps: dL/dtheta from the FP64
    tape against central differences (step 1e-4 rad) of the GPU FP64 forward
    on 16 random theta pixels, within 1e-4 relative."""
    h0, th, tgt, p = inputs.inverse_design(128, seed=1)
    T = 300
    theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    hh = torch.tensor(h0, dtype=torch.float64, device="cuda")
    tg = torch.tensor(tgt, device="cuda")
    loss = 0.5 * ((evolve(theta, hh, p, T, dtype="f64") - tg) ** 2).sum()
    loss.backward()
    g = theta.grad.cpu().numpy()

    def L_of(th_):
        sim = ThinFilm(p, h0, th_, dtype="f64")
        sim.step(T)
        h = sim.h()
        return 0.5 * float(((h - tg) ** 2).sum().item())

    rng = np.random.default_rng(7)
    eps = 1e-4
    floor = 1e-3 * np.abs(g).max()  # pixels whose gradient is ~0 are judged against this
    worst = 0.0
    for _ in range(16):
        y, x = int(rng.integers(0, 128)), int(rng.integers(0, 128))
        tp, tm = th.copy(), th.copy()
        tp[y, x] += eps
        tm[y, x] -= eps
        fd = (L_of(tp) - L_of(tm)) / (2 * eps)
        worst = max(worst, abs(fd - g[y, x]) / max(abs(g[y, x]), floor))
    assert worst <= 1e-4, worst


def test_gradient_matches_central_differences_inverse_design_512():
    """Config 5 at its own size and horizon: 512^2 inverse design (noisy flat
    film, theta = 30 deg + 5 deg noise, 8-drop target, L2 loss), T = 20000
    steps, sqrt(T) checkpoints.  dL/dtheta of the FP64 tape against central
    differences (step 1e-4 rad) of the GPU FP64 forward on 16 seeded theta
    pixels, within 1e-4.  The loss is about 5.5e5 while L+ - L- is about
    1e-5 of it, so the difference is summed as 1/2 sum (h+ - h-)(h+ + h- -
    2 target), which equals L+ - L- without cancelling two large sums; so
    summed, the check is well conditioned at this horizon (agreement of about
    1e-7 on this film).  The 32 perturbed forward runs go through one batch."""
    n, T = 512, 20000
    h0, th, tgt, p = inputs.inverse_design(n, seed=0)
    theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    hh = torch.tensor(h0, dtype=torch.float64, device="cuda")
    tg = torch.tensor(tgt, device="cuda")
    loss = 0.5 * ((evolve(theta, hh, p, T, dtype="f64") - tg) ** 2).sum()
    loss.backward()
    g = theta.grad.cpu().numpy()

    rng = np.random.default_rng(11)
    eps = 1e-4
    pix = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(16)]
    films = []
    for y, x in pix:
        for sgn in (1, -1):
            t_ = th.copy()
            t_[y, x] += sgn * eps
            films.append(ThinFilm(p, h0, t_, dtype="f64"))
    with FilmBatch(films) as B:
        B.step(T)
    floor = 1e-3 * np.abs(g).max()
    worst = 0.0
    for i, (y, x) in enumerate(pix):
        hp, hm = films[2 * i].h(), films[2 * i + 1].h()
        fd = 0.5 * float(((hp - hm) * (hp + hm - 2 * tg)).sum().item()) / (2 * eps)
        worst = max(worst, abs(fd - g[y, x]) / max(abs(g[y, x]), floor))
    for f in films:
        f.close()
    assert worst <= 1e-4, worst


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-3), ("f16", 2e-2), ("bf16", 2e-2)])
def test_reduced_precision_tape_gradient_matches_oracle(dtype, tol):
    """dL/dtheta and dL/dh0 of the FP32 and 16-bit-storage tapes, element by
    element, against the FP64 oracle's reverse sweep (inverse-design shape,
    64^2, 200 steps, sqrt(T) checkpoints).  The FP32 tape differentiates the
    FP32 scheme on its own trajectory: the gap is FP32 rounding carried
    through 200 steps forward and back (bound 1e-3 of the largest entry).
    With 16-bit storage the trajectory itself differs from FP64 by the 16-bit
    roundings of the moving populations (2^-12 FP16, 2^-9 BF16 relative),
    hence 2e-2."""
    h0, th, tgt, p = inputs.inverse_design(64, seed=4)
    T = 200
    L_o, gth_o, gh0_o, _ = _oracle_grads(p, h0, th, T, tgt)
    theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    hh = torch.tensor(h0, dtype=torch.float64, device="cuda", requires_grad=True)
    tg = torch.tensor(tgt, device="cuda")
    loss = 0.5 * ((evolve(theta, hh, p, T, dtype=dtype).double() - tg) ** 2).sum()
    loss.backward()
    gth = theta.grad.cpu().numpy()
    gh0 = hh.grad.cpu().numpy()
    assert np.abs(gth - gth_o).max() <= tol * np.abs(gth_o).max()
    assert np.abs(gh0 - gh0_o).max() <= tol * np.abs(gh0_o).max()
    assert abs(loss.item() - L_o) <= tol * abs(L_o)


def test_fp32_gradient_close_to_fp64():
    h0, th, tgt, p = inputs.inverse_design(64, seed=2)
    T = 200
    grads = {}
    for dt in ("f32", "f64"):
        theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
        hh = torch.tensor(h0, dtype=torch.float64, device="cuda", requires_grad=True)
        tg = torch.tensor(tgt, device="cuda")
        loss = 0.5 * ((evolve(theta, hh, p, T, dtype=dt).double() - tg) ** 2).sum()
        loss.backward()
        grads[dt] = (theta.grad.cpu().numpy(), hh.grad.cpu().numpy())
    for k in range(2):
        a, b = grads["f32"][k], grads["f64"][k]
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max()


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_16bit_storage_gradient_close_to_fp64(dtype):
    """With 16-bit population storage the tape differentiates the FP32 scheme
    along the stored trajectory; its gradient stays within 2e-2 of the FP64
    gradient (the trajectories themselves differ by the 16-bit rounding)."""
    h0, th, tgt, p = inputs.inverse_design(64, seed=4)
    T = 200
    grads = {}
    for dt in (dtype, "f64"):
        theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
        hh = torch.tensor(h0, dtype=torch.float64, device="cuda")
        tg = torch.tensor(tgt, device="cuda")
        loss = 0.5 * ((evolve(theta, hh, p, T, dtype=dt).double() - tg) ** 2).sum()
        loss.backward()
        grads[dt] = theta.grad.cpu().numpy()
    a, b = grads[dtype], grads["f64"]
    assert np.abs(a - b).max() <= 2e-2 * np.abs(b).max()


@pytest.mark.parametrize("case", range(6))
def test_tape_gradient_random_configurations(case):
    """Seeded random lattices and parameters (tau, g, delta, (n, m), pi_sign,
    body force), 25 steps with checkpoints every 4: the FP64 tape gradient
    against the oracle's."""
    rng = np.random.default_rng(3000 + case)
    nx, ny = int(rng.integers(9, 48)), int(rng.integers(9, 48))
    h0, th, p = inputs.small_random(nx, ny, seed=4000 + case, amp=0.08)
    nm = [(3, 2), (9, 3), (4, 3)][case % 3]
    p.update(tau=float(rng.uniform(0.6, 1.4)), g=float(rng.uniform(-5e-4, 5e-4)),
             delta=float(rng.uniform(0.5, 2.0)), n_exp=nm[0], m_exp=nm[1],
             pi_sign=1 if case < 5 else -1, gx_body=float(rng.uniform(-1e-4, 1e-4)))
    T = 25
    tgt = rng.uniform(0.9, 1.1, h0.shape)
    L_o, gth_o, gh0_o, _ = _oracle_grads(p, h0, th, T, tgt)
    theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    hh = torch.tensor(h0, dtype=torch.float64, device="cuda", requires_grad=True)
    loss = 0.5 * ((evolve(theta, hh, p, T, dtype="f64", every=4) - torch.tensor(tgt, device="cuda")) ** 2).sum()
    loss.backward()
    assert abs(loss.item() - L_o) <= 1e-11 * abs(L_o)
    assert np.abs(theta.grad.cpu().numpy() - gth_o).max() <= 1e-9 * np.abs(gth_o).max()
    assert np.abs(hh.grad.cpu().numpy() - gh0_o).max() <= 1e-9 * np.abs(gh0_o).max()


def test_adjoint_rejects_second_order_forcing():
    """The hand-written adjoint differentiates Eq. (LBE) as printed; the
    second-order-forcing reading is refused, not silently differentiated
    as the other scheme."""
    h0, th, p = inputs.small_random(16, 12, seed=1)
    sim = ThinFilm(dict(p, forcing=1), h0, th, dtype="f64")
    f = sim.get_state()
    a = torch.zeros_like(f)
    gk = torch.zeros((12, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(L.TfLbmError) as e:
        L.tf_lbm_adjoint_step(sim.handle, f.data_ptr(), a.data_ptr(), torch.empty_like(f).data_ptr(),
                              gk.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == L.TF_LBM_ERR_UNSUPPORTED
    with pytest.raises(L.TfLbmError) as e:
        L.tf_lbm_tape_create(sim.handle, sim.h0_dev.data_ptr(), sim.theta_dev.data_ptr(), 10, 0)
    assert e.value.code == L.TF_LBM_ERR_UNSUPPORTED
    sim.close()
