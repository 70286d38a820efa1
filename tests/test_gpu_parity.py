"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (relative L-infinity on h, max|h_gpu - h_oracle| / max|h_oracle|):
  FP32 storage and arithmetic: 1e-5 after 1000 steps; relative mass drift 1e-6.
  FP64: 1e-11 (only summation order and fused multiply-adds differ).
The FP32 bound comes from the arithmetic: every step rounds each population
to 2^-24 relative; the film dynamics are diffusive (friction-dominated), so
per-step errors of ~1e-7 do not amplify and accumulate at most like a random
walk, ~sqrt(1000) x 1e-7 = 3e-6 after 1000 steps.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1810_07642_gb300 import inputs
from paper_1810_07642_gb300 import _lib as L
from paper_1810_07642_gb300.film import ThinFilm

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-11, "f16": 1e-3, "bf16": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1810_07642_gb300 import build
    build.build()
    O.set_num_threads(os.cpu_count() or 1)
    assert torch.cuda.is_available()
    yield


def cfg_of(p, **over):
    d = {k: v for k, v in p.items() if k in O.Config.__dataclass_fields__}
    d.update(over)
    return O.Config(**d)


def rel_linf(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).max() / np.abs(b).max()


def run_both(h0, theta, p, steps, dtype="f32", launch=None, theta_uniform=None):
    cfg = cfg_of(p)
    th_o = theta if theta_uniform is None else theta_uniform
    kap = O.kappa_field(cfg, th_o)
    f = O.init(cfg, h0)
    m0 = O.mass(cfg, f)
    O.step(cfg, kap, f, steps)
    ho, uxo, uyo = O.moments(cfg, f)
    pp = dict(p)
    if theta_uniform is not None:
        pp["theta_uniform"] = theta_uniform
    sim = ThinFilm(pp, h0, None if theta_uniform is not None else theta, dtype=dtype)
    if launch:
        sim.set_launch(**launch)
    gm0 = sim.mass()
    sim.step(steps)
    mom = sim.moments()
    gm1 = sim.mass()
    torch.cuda.synchronize()
    out = {k: v.double().cpu().numpy() for k, v in mom.items()}
    sim.close()
    return dict(ho=ho, uxo=uxo, uyo=uyo, mo=m0, h=out["h"], ux=out["ux"], uy=out["uy"],
                gm0=gm0, gm1=gm1)


# ------------------------------------------------------------ small cases

SMALL = [(37, 29), (130, 70), (200, 33), (64, 64), (5, 7), (3, 3), (1, 1), (2, 9)]


@pytest.mark.parametrize("nx,ny", SMALL)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_parity_random_film_patterned(nx, ny, dtype):
    h0, th, p = inputs.small_random(nx, ny, seed=nx * 1000 + ny, amp=0.05)
    p.update(tau=0.9, g=2e-4, gx_body=2e-5, gy_body=-1e-5, delta=1.0)
    r = run_both(h0, th, p, 100, dtype)
    assert rel_linf(r["h"], r["ho"]) <= TOL[dtype]
    scale = max(np.abs(r["uxo"]).max(), np.abs(r["uyo"]).max(), 1e-12)
    assert np.abs(r["ux"] - r["uxo"]).max() <= 1e2 * TOL[dtype] * scale + 1e-12
    assert np.abs(r["uy"] - r["uyo"]).max() <= 1e2 * TOL[dtype] * scale + 1e-12


@pytest.mark.parametrize("tau", [1.0, 0.7, 1.6])
def test_parity_uniform_theta_tau(tau):
    h0, th, p = inputs.small_random(96, 80, seed=3, amp=0.1)
    p.update(tau=tau, delta=0.5)
    r = run_both(h0, th, p, 200, "f32", theta_uniform=math.radians(25))
    assert rel_linf(r["h"], r["ho"]) <= TOL["f32"]


def test_parity_rayleigh_taylor_128_fp32_and_fp64():
    """128 x 128 hanging film (g = -1e-4, delta = 0, kappa = 0), 1000 steps."""
    h0, th, p = inputs.rayleigh_taylor(128)
    for dtype in ("f32", "f64"):
        r = run_both(h0, th, p, 1000, dtype)
        assert rel_linf(r["h"], r["ho"]) <= TOL[dtype]
        # the perturbation itself (h - 1 ~ 1e-3) must match too
        dh, dho = r["h"] - 1.0, r["ho"] - 1.0
        assert np.abs(dh - dho).max() <= (1e-3 if dtype == "f32" else 1e-9) * np.abs(dho).max()
        assert abs(r["gm1"] - r["mo"]) <= 1e-6 * r["mo"]


def test_parity_sessile_drop_256_fp32():
    """Spherical-cap drop on a precursor film (theta = 20 deg, delta = 1)."""
    h0, th, p = inputs.sessile_drop(256, rb=60.0, hd=10.0)
    r = run_both(h0, th, p, 1000, "f32", theta_uniform=math.radians(20))
    assert rel_linf(r["h"], r["ho"]) <= TOL["f32"]
    assert abs(r["gm1"] - r["gm0"]) <= 1e-6 * r["gm0"]
    assert abs(r["gm0"] - r["mo"]) <= 1e-6 * r["mo"]


def test_parity_patterned_dewetting_256_fp32():
    h0, th, p = inputs.patterned_dewetting(256, seed=1)
    r = run_both(h0, th, p, 1000, "f32")
    assert rel_linf(r["h"], r["ho"]) <= TOL["f32"]
    assert abs(r["gm1"] - r["gm0"]) <= 1e-6 * r["gm0"]


@pytest.mark.parametrize("shape", [dict(block_x=64, rows=1, pipeline=1), dict(block_x=64, rows=5, pipeline=1),
                                   dict(block_x=64, rows=7, graph_chunk=4, pipeline=1),
                                   dict(block_x=128, rows=64, pipeline=1), dict(block_x=256, rows=17, pipeline=1),
                                   dict(block_x=128, rows=3, graph_chunk=4, pipeline=1),
                                   dict(block_x=64, rows=9, pipeline=0),
                                   dict(block_x=128, rows=33, pipeline=0),
                                   dict(block_x=64, rows=1, pipeline=2),
                                   dict(block_x=128, rows=29, pipeline=2, graph_chunk=4)])
def test_launch_shape_does_not_change_results(shape):
    """Every node does the same arithmetic in the same order whatever the band
    height or graph chunking, so with the same CTA width and load pipeline
    results are bitwise identical.  Another CTA width or pipeline is another
    kernel instantiation, in which the compiler may fuse multiply-adds
    differently: there results agree to rounding (1e-6 relative after 23
    steps)."""
    h0, th, p = inputs.small_random(304, 141, seed=9, amp=0.05)
    ref = ThinFilm(p, h0, th)
    ref.set_launch(block_x=64, rows=64, graph_chunk=0, pipeline=1)
    ref.step(23)
    other = ThinFilm(p, h0, th)
    other.set_launch(**shape)
    other.step(23)
    a, b = ref.get_state(), other.get_state()
    torch.cuda.synchronize()
    d = (a - b).abs()
    if shape["block_x"] == 64 and shape["pipeline"] == 1:
        assert torch.equal(a, b), (d.max().item(), (d > 0).sum().item())
    else:
        assert d.max().item() <= 1e-6 * a.abs().max().item()


@pytest.mark.parametrize("dtype", ["f32", "f64", "f16"])
@pytest.mark.parametrize("nx,ny", [(37, 29), (130, 70), (3, 3)])
def test_parity_per_thread_load_pipeline(dtype, nx, ny):
    """The per-thread-load kernel (pipeline 1, the default) against the oracle."""
    h0, th, p = inputs.small_random(nx, ny, seed=nx + ny, amp=0.05)
    p.update(tau=0.9, g=2e-4, gx_body=2e-5, delta=1.0)
    r = run_both(h0, th, p, 100, dtype, launch=dict(pipeline=1))
    assert rel_linf(r["h"], r["ho"]) <= TOL[dtype]


# ------------------------------------------------- 16-bit population storage

@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("case", ["rt128", "drop256", "pattern256", "random"])
def test_parity_16bit_storage(dtype, case):
    """Moving populations in FP16 / BF16, arithmetic in FP32: relative Linf
    on h within 1e-3 of the FP64 oracle after 1000 steps, and the total
    volume conserved to 1e-6 (the 16-bit roundings are folded into the FP32
    rest population)."""
    if case == "rt128":
        h0, th, p = inputs.rayleigh_taylor(128)
        r = run_both(h0, th, p, 1000, dtype)
    elif case == "drop256":
        h0, th, p = inputs.sessile_drop(256, rb=60.0, hd=10.0)
        r = run_both(h0, th, p, 1000, dtype, theta_uniform=math.radians(20))
    elif case == "pattern256":
        h0, th, p = inputs.patterned_dewetting(256, seed=1)
        r = run_both(h0, th, p, 1000, dtype)
    else:
        h0, th, p = inputs.small_random(130, 70, seed=12, amp=0.05)
        p.update(tau=0.9, g=2e-4, gx_body=2e-5, gy_body=-1e-5)
        r = run_both(h0, th, p, 300, dtype)
    err = rel_linf(r["h"], r["ho"])
    assert err <= TOL[dtype], err
    assert abs(r["gm1"] - r["gm0"]) <= 1e-6 * r["gm0"], abs(r["gm1"] - r["gm0"]) / r["gm0"]


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_16bit_state_roundtrip_and_shape_invariance(dtype):
    h0, th, p = inputs.small_random(300, 141, seed=9, amp=0.05)
    a = ThinFilm(p, h0, th, dtype=dtype)
    a.set_launch(block_x=64, rows=64, graph_chunk=0)
    a.step(17)
    s = a.get_state()
    b = ThinFilm(p, h0, th, dtype=dtype)
    b.set_launch(block_x=64, rows=5, graph_chunk=4)
    b.set_state(s)
    a.step(9)
    b.step(9)
    assert torch.equal(a.get_state(), b.get_state())


# ------------------------------------------------------- full-size sampled

def _window(f, y, x, rad):
    ny, nx = f.shape[1:]
    ys = (np.arange(y - rad, y + rad + 1)) % ny
    xs = (np.arange(x - rad, x + rad + 1)) % nx
    return np.ascontiguousarray(f[:, ys][:, :, xs])


def test_full_size_patterned_2048_sampled_against_oracle():
    """2048 x 2048 patterned dewetting in the default launch shape.  After k
    steps the population at a node depends only on the state within radius 3k
    (pull: radius 1, grad p: +1, lap h: +1, h: +1), so the oracle can advance
    a (6k+1)^2 window cut from the GPU state and compare its centre."""
    h0, th, p = inputs.patterned_dewetting(2048, seed=0)
    sim = ThinFilm(p, h0, th)
    sim.step(50)  # develop some dynamics first
    f0 = sim.get_state().double().cpu().numpy()
    k = 3
    sim.step(k)
    f1 = sim.get_state().double().cpu().numpy()
    assert sim.check() == 0
    sim.close()
    rng = np.random.default_rng(0)
    bx = 128
    pts = [(0, 0), (2047, 2047), (0, 2047), (2047, 0), (63, bx - 1), (64, bx), (1000, 1023)]
    pts += [(int(y), int(x)) for y, x in zip(rng.integers(0, 2048, 57), rng.integers(0, 2048, 57))]
    rad = 3 * k
    worst = 0.0
    cfg = cfg_of(p, nx=2 * rad + 1, ny=2 * rad + 1)
    for (y, x) in pts:
        fw = _window(f0, y, x, rad)
        thw = th[(np.arange(y - rad, y + rad + 1) % 2048)][:, (np.arange(x - rad, x + rad + 1) % 2048)]
        O.step(cfg, O.kappa_field(cfg, thw), fw, k)
        got = f1[:, y, x]
        worst = max(worst, np.abs(fw[:, rad, rad] - got).max() / np.abs(fw[:, rad, rad]).max())
    assert worst <= 1e-5, worst


def test_full_size_patterned_2048_1000_steps_every_storage_type():
    """Config 3's own lattice (2048 x 2048 chemically patterned dewetting,
    Sec. III D shape) for 1000 steps in FP32, FP16 and BF16 storage in the
    default launch shapes, against the whole FP64 oracle run (about a
    minute on the host cores): relative Linf on h within the storage type's
    tolerance and relative mass drift within 1e-6."""
    h0, th, p = inputs.patterned_dewetting(2048, seed=0)
    cfg = cfg_of(p)
    f = O.init(cfg, h0)
    O.step(cfg, O.kappa_field(cfg, th), f, 1000)
    ho = f.sum(0)
    for dtype in ("f32", "f16", "bf16"):
        sim = ThinFilm(p, h0, th, dtype=dtype)
        m0 = sim.mass()
        sim.step(1000)
        h = sim.h().double().cpu().numpy()
        drift = abs(sim.mass() - m0) / m0
        assert sim.check() == 0
        sim.close()
        err = rel_linf(h, ho)
        assert err <= TOL[dtype], (dtype, err)
        assert drift <= 1e-6, (dtype, drift)


def test_full_size_mass_conservation_and_check():
    h0, th, p = inputs.patterned_dewetting(2048, seed=2)
    sim = ThinFilm(p, h0, th)
    m0 = sim.mass()
    ref = float(np.asarray(h0, np.float32).astype(np.float64).sum())
    assert abs(m0 - ref) <= 1e-6 * ref
    sim.step(300)
    m1 = sim.mass()
    assert abs(m1 - m0) <= 1e-6 * m0
    assert sim.check() == 0
    sim.close()


# ------------------------------------------------------------ API behaviour

def test_initial_moments_are_h0_at_rest():
    h0, th, p = inputs.small_random(50, 40, seed=4, amp=0.2)
    sim = ThinFilm(p, h0, th, dtype="f64")
    m = sim.moments()
    assert torch.allclose(m["h"].cpu(), torch.as_tensor(h0), rtol=1e-15, atol=0)
    assert m["ux"].abs().max().item() < 1e-15 and m["uy"].abs().max().item() < 1e-15
    assert sim.time == 0


def test_flat_film_stays_flat_on_gpu():
    p = inputs._params(70, 50, g=-1e-4, tau=0.8)
    p["theta_uniform"] = 0.3
    sim = ThinFilm(p, np.full((50, 70), 1.3), None)
    sim.step(100)
    m = sim.moments()
    assert (m["h"].max() - m["h"].min()).item() == 0.0
    assert m["ux"].abs().max().item() == 0.0 and m["uy"].abs().max().item() == 0.0


@pytest.mark.parametrize("forcing", [0, 1])
def test_pressure_force_diagnostic_matches_oracle(forcing):
    h0, th, p = inputs.small_random(64, 48, seed=6, amp=0.1)
    p.update(gx_body=1e-5, delta=0.3, forcing=forcing)
    cfg = cfg_of(p)
    kap = O.kappa_field(cfg, th)
    f = O.init(cfg, h0)
    O.step(cfg, kap, f, 20)
    po, fxo, fyo = O.pressure_force(cfg, kap, f)
    sim = ThinFilm(p, h0, th, dtype="f64")
    sim.step(20)
    d = {k: v.cpu().numpy() for k, v in sim.pressure_force().items()}
    assert rel_linf(d["p"], po) < 1e-10
    assert np.abs(d["fx"] - fxo).max() < 1e-10 * np.abs(fxo).max()
    assert np.abs(d["fy"] - fyo).max() < 1e-10 * np.abs(fyo).max()


def test_state_roundtrip_resumes_bitwise():
    h0, th, p = inputs.small_random(90, 70, seed=8, amp=0.1)
    a = ThinFilm(p, h0, th)
    a.step(17)
    s = a.get_state()
    b = ThinFilm(p, h0, th)
    b.set_state(s)
    a.step(9)
    b.step(9)
    assert torch.equal(a.get_state(), b.get_state())


def test_bulk_copy_pipeline_needs_nx_multiple_of_8():
    h0, th, p = inputs.small_random(300, 20, seed=1)
    sim = ThinFilm(p, h0, th)
    assert p["tau"] == 1.0
    assert sim.launch["pipeline"] == 3  # FP32, tau = 1, nx even: two columns per thread
    assert ThinFilm(p, h0, th, dtype="f16").launch["pipeline"] == 3  # 16-bit, nx even: two columns
    assert ThinFilm(dict(p, tau=0.8), h0, th).launch["pipeline"] == 1  # tau != 1: one column
    assert ThinFilm(dict(p, tau=0.8), h0, th, dtype="f16").launch["pipeline"] == 1
    h1, t1, p1 = inputs.small_random(301, 20, seed=1)
    assert ThinFilm(p1, h1, t1).launch["pipeline"] == 1  # nx odd: one column
    with pytest.raises(L.TfLbmError):
        sim.set_launch(pipeline=0)
    h0, th, p = inputs.small_random(304, 20, seed=1)
    sim = ThinFilm(p, h0, th)
    sim.set_launch(pipeline=0)
    assert sim.launch["pipeline"] == 0


@pytest.mark.parametrize("dtype", ["f32", "f64", "f16", "bf16"])
@pytest.mark.parametrize("nx,ny", [(64, 48), (200, 33), (16, 9)])
def test_parity_bulk_copy_pipeline(dtype, nx, ny):
    """The bulk-copy (TMA) kernel against the oracle, including lattices whose
    strips wrap on both sides."""
    h0, th, p = inputs.small_random(nx, ny, seed=nx * 7 + ny, amp=0.05)
    p.update(tau=0.9 if dtype == "f64" else 1.0, g=2e-4, gx_body=2e-5, delta=1.0)
    r = run_both(h0, th, p, 100, dtype, launch=dict(pipeline=0))
    assert rel_linf(r["h"], r["ho"]) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f32", "f64", "f16", "bf16"])
@pytest.mark.parametrize("case", ["random", "pattern128"])
def test_parity_printed_pi_sign(dtype, case):
    """The printed sign of Eq. (pfilm), p = -gamma (lap h - Pi) (pi_sign =
    -1), element by element against the oracle in every storage type: a
    theta field on a thick noisy film (the printed sign destabilises only
    films near the precursor thickness), and patterned dewetting at 128^2."""
    if case == "random":
        h0, th, p = inputs.small_random(96, 80, seed=31, amp=0.05)
        p.update(tau=0.9, g=1e-4, gx_body=1e-5, delta=1.0, pi_sign=-1)
        steps = 300
    else:
        h0, th, p = inputs.patterned_dewetting(128, seed=5)
        p.update(pi_sign=-1)
        steps = 1000
    r = run_both(h0, th, p, steps, dtype)
    assert rel_linf(r["h"], r["ho"]) <= TOL[dtype]
    assert abs(r["gm1"] - r["gm0"]) <= 1e-6 * r["gm0"]


@pytest.mark.parametrize("block_x", [64, 128, 256])
@pytest.mark.parametrize("tau", [0.7, 1.6])
@pytest.mark.parametrize("nx,ny", [(37, 29), (300, 41), (130, 3)])
def test_parity_async_copy_pipeline_general_tau(block_x, tau, nx, ny):
    """FP32 async-copy kernel (pipeline 2) at tau != 1, where it keeps the
    pulled populations of the last four rows in a per-thread shared ring
    beside the copy ring, for every CTA width, against the oracle."""
    h0, th, p = inputs.small_random(nx, ny, seed=nx + 5 * ny, amp=0.05)
    p.update(tau=tau, g=2e-4, gx_body=2e-5, gy_body=-1e-5, delta=1.0)
    r = run_both(h0, th, p, 200, "f32", launch=dict(pipeline=2, block_x=block_x, rows=7))
    assert rel_linf(r["h"], r["ho"]) <= TOL["f32"]


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("nx,ny", [(37, 29), (130, 70), (3, 3), (2, 1), (200, 2)])
@pytest.mark.parametrize("rows", [1, 2, 16])
def test_parity_async_copy_pipeline(dtype, nx, ny, rows):
    """The async-copy kernel (pipeline 2) against the oracle, including bands
    of one and two rows, where the three-stage ring wraps every step."""
    h0, th, p = inputs.small_random(nx, ny, seed=nx * 3 + ny, amp=0.05)
    p.update(tau=0.9 if dtype == "f64" else 1.0, g=2e-4, gx_body=2e-5, delta=1.0)
    r = run_both(h0, th, p, 100, dtype, launch=dict(pipeline=2, rows=rows))
    assert rel_linf(r["h"], r["ho"]) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("tau", [1.0, 0.75])
@pytest.mark.parametrize("theta_field", [True, False])
@pytest.mark.parametrize("nx,ny,block_x", [(16, 9, 64), (64, 48, 64), (200, 33, 128), (304, 41, 256),
                                           (520, 70, 128), (2, 5, 64), (6, 1, 128)])
def test_parity_two_column_pipeline(dtype, tau, theta_field, nx, ny, block_x):
    """The two-column kernel (pipeline 3: aligned pair loads, lane shuffles
    for the values that cross a pair boundary) against the oracle, at both
    relaxation kernels, with and without a theta field, every storage type it
    takes and CTA widths of 64, 128 and 256 columns, including lattices
    narrower than one CTA (strips wrap on both sides), one row, and several
    strips with a ragged last one."""
    h0, th, p = inputs.small_random(nx, ny, seed=nx * 11 + ny, amp=0.05)
    p.update(tau=tau, g=2e-4, gx_body=2e-5, gy_body=-1e-5, delta=1.0)
    r = run_both(h0, th, p, 100, dtype, launch=dict(pipeline=3, block_x=block_x, rows=7),
                 theta_uniform=None if theta_field else math.radians(20.0))
    assert rel_linf(r["h"], r["ho"]) <= TOL[dtype]
    assert abs(r["gm1"] - r["gm0"]) <= 1e-6 * r["gm0"]


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_two_column_band_heights_agree_bitwise(dtype):
    """With the same CTA width, every node of the two-column kernel runs the
    same instruction sequence whatever the band height or graph chunking, so
    the states are identical bit for bit."""
    h0, th, p = inputs.small_random(304, 141, seed=19, amp=0.05)
    p.update(tau=0.9, gx_body=1e-5)
    states = []
    for rows, chunk in ((13, 0), (1, 0), (64, 4), (141, 0)):
        sim = ThinFilm(p, h0, th, dtype=dtype)
        sim.set_launch(pipeline=3, block_x=128, rows=rows, graph_chunk=chunk)
        sim.step(25)
        states.append(sim.get_state())
        sim.close()
    for st in states[1:]:
        assert torch.equal(states[0], st)


@pytest.mark.parametrize("pipeline,dtype", [(0, "f32"), (0, "f16"), (0, "bf16"), (0, "f64")])
def test_bulk_copy_wait_limit_reports_timeout(pipeline, dtype):
    """A bulk-copy step kernel that gives up waiting for its own row copies
    sets TF_LBM_STATUS_TIMEOUT, stops issuing, waits (bounded) for the copies
    it has issued and returns.  A limit of 0 polls makes every wait give up
    at once, deterministically, while every issued copy still lands.  The
    context stays usable: a fresh run with the default limit then matches
    the oracle."""
    h0, th, p = inputs.small_random(64, 48, seed=2, amp=0.05)
    sim = ThinFilm(p, h0, th, dtype=dtype)
    sim.set_launch(pipeline=pipeline, graph_chunk=0)
    assert sim.check() == 0
    L.tf_lbm_set_wait_limit(sim.handle, 0)
    sim.step(3)
    assert sim.check() & L.TF_LBM_STATUS_TIMEOUT
    L.tf_lbm_set_wait_limit(sim.handle, -1)
    sim.close()
    r = run_both(h0, th, p, 50, dtype, launch=dict(pipeline=pipeline))
    assert rel_linf(r["h"], r["ho"]) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f32", "f64", "f16", "bf16"])
@pytest.mark.parametrize("pipeline", [0, 1, 2, 3])
@pytest.mark.parametrize("tau", [1.0, 0.75])
def test_parity_second_order_forcing(dtype, pipeline, tau):
    """The labelled second-order-forcing reading (forcing = 1: u = (j +
    F/2)/h with implicit friction, source (1 - omega/2) w_l [3 (c_l - u) +
    9 (c_l.u) c_l].F) against the oracle's, in every storage type and step
    pipeline that applies, both relaxation kernels, body forces, a theta
    field and gravity in the equilibria."""
    if pipeline == 2 and dtype in ("f16", "bf16"):
        pytest.skip("the async-copy pipeline takes full-width storage only")
    if pipeline == 3 and dtype == "f64":
        pytest.skip("the two-column pipeline computes in FP32")
    h0, th, p = inputs.small_random(96, 40, seed=77, amp=0.05)
    p.update(tau=tau, g=2e-4, gx_body=2e-5, gy_body=-1e-5, delta=0.5, forcing=1)
    r = run_both(h0, th, p, 200, dtype, launch=dict(pipeline=pipeline, rows=9))
    assert rel_linf(r["h"], r["ho"]) <= TOL[dtype]
    assert abs(r["gm1"] - r["gm0"]) <= 1e-6 * r["gm0"]


def test_second_order_forcing_differs_from_printed_scheme():
    """The two readings are different schemes: on the same film their
    states part after a few steps (a guard against the option being
    ignored)."""
    h0, th, p = inputs.small_random(64, 32, seed=3, amp=0.1)
    p.update(gx_body=1e-4, delta=0.5)
    a = ThinFilm(dict(p, forcing=0), h0, th, dtype="f64")
    b = ThinFilm(dict(p, forcing=1), h0, th, dtype="f64")
    a.step(20)
    b.step(20)
    d = (a.h() - b.h()).abs().max().item()
    assert d > 1e-8


def test_async_copy_pipeline_needs_full_width_storage():
    h0, th, p = inputs.small_random(16, 16, seed=1)
    sim = ThinFilm(p, h0, th, dtype="f16")
    with pytest.raises(L.TfLbmError) as e:
        sim.set_launch(pipeline=2)
    assert "FP32 or FP64" in str(e.value)


def test_invalid_arguments_are_rejected():
    from paper_1810_07642_gb300.film import make_params
    h0 = torch.ones((8, 8), device="cuda")
    base = dict(inputs._params(8, 8))
    for bad in (dict(tau=0.5), dict(hstar=0.0), dict(n_exp=2, m_exp=2), dict(pi_sign=0),
                dict(delta=-1.0), dict(nx=0), dict(ny=-3), dict(gamma=float("nan"))):
        q = dict(base, **bad)
        with pytest.raises(L.TfLbmError) as e:
            L.tf_lbm_init(make_params(**q), h0.data_ptr(), None, 0)
        assert e.value.code == L.TF_LBM_ERR_ARG
        assert "invalid parameter" in str(e.value)
    prm = make_params(8, 8)
    hh = np.ones((8, 8), np.float32)
    with pytest.raises(L.TfLbmError) as e:
        L.tf_lbm_init(prm, hh.ctypes.data, None, 0)  # host pointer
    assert e.value.code == L.TF_LBM_ERR_ARG and "device" in str(e.value)
    sim = ThinFilm(base, h0)
    with pytest.raises(L.TfLbmError):
        sim.step(-1)
    with pytest.raises(L.TfLbmError):
        sim.set_launch(block_x=96)
    with pytest.raises(L.TfLbmError):
        sim.set_launch(graph_chunk=3)


def test_check_reports_nonfinite_and_nonpositive():
    p = inputs._params(16, 16)
    h0 = np.ones((16, 16))
    h0[3, 4] = np.nan
    assert ThinFilm(p, h0).check() & L.TF_LBM_STATUS_NONFINITE
    h0 = np.ones((16, 16))
    h0[5, 5] = 0.0
    assert ThinFilm(p, h0).check() & L.TF_LBM_STATUS_NONPOSITIVE
    assert ThinFilm(p, np.ones((16, 16))).check() == 0


def test_no_slip_precursor_diverges_and_is_reported():
    """With delta = 0 the explicit friction factor 1 - nu alpha / h is about
    -100 on the h* = 0.07 precursor, so the sessile-drop run diverges; the
    library must report it rather than hide it."""
    h0, th, p = inputs.sessile_drop(128, rb=30.0, hd=5.0, delta=0.0)
    p["theta_uniform"] = math.radians(20)
    sim = ThinFilm(p, h0, None)
    status = 0
    for _ in range(50):
        sim.step(20)
        status = sim.check()
        if status:
            break
    assert status & (L.TF_LBM_STATUS_NONFINITE | L.TF_LBM_STATUS_NONPOSITIVE)


def test_lattice_beyond_32bit_offsets_is_unsupported():
    from paper_1810_07642_gb300.film import make_params
    h0 = torch.ones(16, device="cuda")  # never read: the size check comes first
    with pytest.raises(L.TfLbmError) as e:
        L.tf_lbm_init(make_params(16384, 16384), h0.data_ptr(), None, 0)
    assert e.value.code == L.TF_LBM_ERR_UNSUPPORTED and "2^31" in str(e.value)


def test_largest_lattice_tiles_the_oracle():
    """16000 x 14000 (9 ny pitch = 2.016e9 elements, just under the 2^31
    offset limit; 16 GB of FP32 populations).  h0 is periodic with a 64 x 56
    period that divides the lattice, so the solution is the tiling of the
    solution on one 64 x 56 period: sampled nodes all over the lattice,
    including the last rows and columns, must match the oracle run on that
    period."""
    nx, ny, px, py, steps = 16000, 14000, 64, 56, 10
    hp, _, p = inputs.small_random(px, py, seed=21, amp=0.05)
    p = dict(p, nx=nx, ny=ny, theta_uniform=math.radians(25.0), tau=0.9, gx_body=1e-5)
    h0 = torch.as_tensor(hp, device="cuda").repeat(ny // py, nx // px)
    sim = ThinFilm(p, h0, None, dtype="f32")
    del h0
    m0 = sim.mass()
    sim.step(steps)
    h = sim.h()
    assert sim.check() == 0
    assert abs(sim.mass() - m0) <= 1e-6 * m0
    cfg = cfg_of(dict(p, nx=px, ny=py))
    f = O.init(cfg, hp.astype(np.float32).astype(np.float64))
    O.step(cfg, O.kappa_field(cfg, p["theta_uniform"]), f, steps)
    ho = f.sum(0)
    rng = np.random.default_rng(5)
    ys = np.concatenate([rng.integers(0, ny, 200), [0, ny - 1, ny - 1]])
    xs = np.concatenate([rng.integers(0, nx, 200), [nx - 1, 0, nx - 1]])
    got = h[torch.as_tensor(ys, device="cuda"), torch.as_tensor(xs, device="cuda")].double().cpu().numpy()
    want = ho[ys % py, xs % px]
    assert np.abs(got - want).max() <= 1e-5 * np.abs(ho).max()
    sim.close()


@pytest.mark.parametrize("case", range(24))
def test_parity_random_configurations(case):
    """Seeded random lattices (1..90 x 1..90) and parameters (tau, gamma, g,
    delta, h*, (n, m), pi_sign, body force, theta field or uniform angle,
    storage type), 60 steps, against the oracle."""
    rng = np.random.default_rng(1000 + case)
    nx, ny = int(rng.integers(1, 91)), int(rng.integers(1, 91))
    dtype = ["f32", "f64", "f16", "bf16"][case % 4]
    nm = [(3, 2), (9, 3), (4, 3)][int(rng.integers(0, 3))]
    h0, th, p = inputs.small_random(nx, ny, seed=2000 + case, amp=float(rng.uniform(0.0, 0.1)))
    p.update(tau=float(rng.uniform(0.6, 1.5)), gamma=float(rng.uniform(0.005, 0.02)),
             g=float(rng.uniform(-5e-4, 5e-4)), delta=float(rng.uniform(0.5, 2.0)),
             hstar=float(rng.uniform(0.05, 0.1)), n_exp=nm[0], m_exp=nm[1],
             gx_body=float(rng.uniform(-1e-4, 1e-4)), gy_body=float(rng.uniform(-1e-4, 1e-4)))
    uniform = bool(rng.integers(0, 2))
    th_u = float(np.radians(rng.uniform(5, 45))) if uniform else None
    p["pi_sign"] = int(rng.choice([1, -1]))
    r = run_both(h0, th, p, 60, dtype, theta_uniform=th_u)
    assert rel_linf(r["h"], r["ho"]) <= TOL[dtype], (nx, ny, dtype, p)
    if dtype in ("f32", "f64"):
        assert abs(r["gm1"] - r["gm0"]) <= 1e-6 * r["gm0"]
