"""GPU batches of uneven domains (tf_lbm_batch_*), the launch-shape
autotuners and the on-device film diagnostics, against the FP64 oracle and
against the single-domain path.

Tolerances are those of the single-domain parity tests (relative L-infinity
on h after the stated steps: FP32 1e-5, FP64 1e-11, FP16/BF16 storage 1e-3):
a batched step runs the same per-node arithmetic as the single-domain step.
Launch shapes that share the CTA width (band height, work queue on or off)
give bit-identical states, since every node is computed by the same
instruction sequence whichever CTA owns it.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1810_07642_gb300 import _lib as L
from paper_1810_07642_gb300 import inputs
from paper_1810_07642_gb300.film import FilmBatch, ThinFilm

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-11, "f16": 1e-3, "bf16": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1810_07642_gb300 import build
    build.build()
    O.set_num_threads(os.cpu_count() or 1)
    assert torch.cuda.is_available()


def cfg_of(p):
    return O.Config(**{k: v for k, v in p.items() if k in O.Config.__dataclass_fields__})


def oracle_h(h0, theta, p, steps):
    cfg = cfg_of(p)
    kap = O.kappa_field(cfg, theta if theta is not None else p["theta_uniform"])
    f = O.init(cfg, h0)
    O.step(cfg, kap, f, steps)
    return O.moments(cfg, f)[0]


def rel_linf(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max())


def uneven_specs(tau=(1.0, 1.0, 1.0, 1.0), even=False):
    """Four uneven domains: patterned theta fields and uniform angles mixed,
    one narrower than a CTA, one smaller than the stencil (even: every nx
    even, as the two-column kernel needs)."""
    out = []
    sizes = [(38, 29), (130, 70), (64, 32), (6, 7)] if even else [(37, 29), (130, 70), (64, 32), (5, 7)]
    for i, (nx, ny) in enumerate(sizes):
        h0, th, p = inputs.small_random(nx, ny, seed=10 + i, amp=0.1)
        p["tau"] = tau[i]
        p["g"] = 1e-3 * (i - 1)
        if i % 2 == 1:  # uniform angle, no theta field
            p["theta_uniform"] = np.radians(25.0 + 5 * i)
            th = None
        out.append((h0, th, p))
    return out


def make_films(specs, dtype):
    return [ThinFilm(p, h0, th, dtype=dtype) for h0, th, p in specs]


def host_h(film):
    return film.h().double().cpu().numpy()


@pytest.mark.parametrize("dtype", ["f32", "f64", "f16", "bf16"])
@pytest.mark.parametrize("taus", [(1.0, 1.0, 1.0, 1.0), (0.8, 1.0, 1.3, 0.6)])
@pytest.mark.parametrize("even", [False, True])
def test_batch_parity_with_oracle(dtype, taus, even):
    """Odd widths take the one-column kernel; even widths the two-column one
    (its default for 16-bit storage and for FP32 at tau = 1, asked for
    explicitly otherwise)."""
    specs = uneven_specs(taus, even=even)
    films = make_films(specs, dtype)
    m0 = [f.mass() for f in films]
    with FilmBatch(films) as B:
        if even and dtype != "f64":
            B.set_launch(pipeline=3)
        assert B.launch["pipeline"] == (3 if even and dtype != "f64" else 1)
        B.step(1000)
        torch.cuda.synchronize()
        for (h0, th, p), f, m in zip(specs, films, m0):
            assert f.time == 1000
            ho = oracle_h(h0, th, p, 1000)
            assert rel_linf(host_h(f), ho) <= TOL[dtype], (p["nx"], p["ny"])
            if dtype in ("f32", "f64"):
                assert abs(f.mass() - m) / m <= 1e-6
    for f in films:
        f.close()


# Sliding drops: BF16 keeps 8 significant bits against FP16's 11, so its
# unit roundoff (2^-9) is 8 times FP16's (2^-12); on drops that slide, every
# step's rounding of the momentum-carrying populations moves the contact
# lines, and the error on h scales with that roundoff.  The BF16 bound for
# moving contact lines is therefore the FP16 bound times 8.
TOL_SLIDING = {"f32": 1e-5, "f16": 1e-3, "bf16": 8e-3}


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_sliding_drop_sweep_parity(dtype):
    """The sliding-drop sweep reduced to four domains (192x96 and 256x128,
    drops of apex 14-19 on the h* precursor, Bo from 0.05 to 1), batched,
    1000 steps: moving contact lines are where rounding grows fastest."""
    specs = [(h0, None, dict(p, theta_uniform=float(th[0, 0])))
             for h0, th, p in inputs.sliding_drops(count=4, seed=1, lx_range=(128, 256))]
    films = make_films(specs, dtype)
    m0 = [f.mass() for f in films]
    with FilmBatch(films) as B:
        B.step(1000)
        for (h0, th, p), f, m in zip(specs, films, m0):
            ho = oracle_h(h0, th, p, 1000)
            assert rel_linf(host_h(f), ho) <= TOL_SLIDING[dtype], (p["nx"], p["bond"])
            assert abs(f.mass() - m) / m <= 1e-6
    for f in films:
        f.close()


@pytest.mark.parametrize("dtype", ["f32", "f16"])
@pytest.mark.parametrize("pipeline", [1, 3])
def test_batch_matches_single_domain_path(dtype, pipeline):
    """A batched step and a single-domain step with the same pipeline, CTA
    width and band height agree to rounding.  The two kernels may contract
    different multiply-adds; with 16-bit storage such a difference can flip
    the rounding of a stored deviation (2^-11 relative), hence the looser
    bound."""
    specs = uneven_specs(even=pipeline == 3)
    singles = make_films(specs, dtype)
    batched = make_films(specs, dtype)
    for f in singles:
        f.set_launch(block_x=64, rows=16, graph_chunk=0, pipeline=pipeline)
        f.step(200)
    with FilmBatch(batched) as B:
        B.set_launch(block_x=64, rows=16, graph_chunk=0, queue=0, pipeline=pipeline)
        B.step(200)
        for a, b in zip(singles, batched):
            sa = a.get_state().cpu().numpy()
            sb = b.get_state().cpu().numpy()
            tol = 1e-6 if dtype == "f32" else 2e-5
            assert np.abs(sa - sb).max() <= tol * np.abs(sa).max()


@pytest.mark.parametrize("pipeline", [1, 3])
def test_batch_launch_shapes_are_bit_identical(pipeline):
    specs = uneven_specs((0.9, 0.9, 0.9, 0.9), even=pipeline == 3)
    ref = None
    for shape in [dict(block_x=64, rows=16, queue=0), dict(block_x=64, rows=5, queue=1),
                  dict(block_x=64, rows=200, queue=1), dict(block_x=64, rows=1, queue=0)]:
        films = make_films(specs, "f32")
        with FilmBatch(films) as B:
            B.set_launch(graph_chunk=4, pipeline=pipeline, **shape)
            B.step(50)
            states = [f.get_state().cpu().numpy() for f in films]
        if ref is None:
            ref = states
        else:
            for a, b in zip(ref, states):
                assert np.array_equal(a, b), shape
        for f in films:
            f.close()


def test_batch_with_single_steps_in_between_and_graphs():
    """Single-handle steps between batched ones (the handles' buffer order
    then differs from the batch's table) and graph chunks with a remainder."""
    specs = uneven_specs()
    films = make_films(specs, "f32")
    with FilmBatch(films) as B:
        B.set_launch(graph_chunk=4)
        B.step(3)
        films[1].step(1)
        B.step(10)  # two graph replays and two single launches
        films[2].step(3)
        B.step(5)
        torch.cuda.synchronize()
        expect = [18, 19, 21, 18]
        for (h0, th, p), f, t in zip(specs, films, expect):
            assert f.time == t
            assert rel_linf(host_h(f), oracle_h(h0, th, p, t)) <= TOL["f32"]


def test_batch_tuner_keeps_state_and_time():
    specs = uneven_specs()
    films = make_films(specs, "f32")
    with FilmBatch(films) as B:
        B.step(7)
        before = [f.get_state().cpu().numpy() for f in films]
        best = B.tune(trial_steps=4)
        assert best["block_x"] in (64, 128, 256) and best["rows"] >= 1 and best["queue"] in (0, 1)
        assert best["pipeline"] == 1  # odd widths: the one-column kernel only
        assert B.launch == best
        after = [f.get_state().cpu().numpy() for f in films]
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
        assert [f.time for f in films] == [7] * 4
        B.step(13)
        torch.cuda.synchronize()
        for (h0, th, p), f in zip(specs, films):
            assert rel_linf(host_h(f), oracle_h(h0, th, p, 20)) <= TOL["f32"]


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_single_tuner_keeps_state_and_time(dtype):
    h0, th, p = inputs.small_random(200, 120, seed=4)
    sim = ThinFilm(p, h0, th, dtype=dtype)
    sim.step(5)
    before = sim.get_state().cpu().numpy()
    best = sim.tune(trial_steps=4)
    assert best["block_x"] in (64, 128, 256) and best["pipeline"] in ((0, 1, 2, 3) if dtype == "f32" else (0, 1, 3))
    assert sim.launch == best
    assert np.array_equal(before, sim.get_state().cpu().numpy())
    assert sim.time == 5
    sim.step(95)
    torch.cuda.synchronize()
    assert rel_linf(host_h(sim), oracle_h(h0, th, p, 100)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16"])
def test_diagnostics_match_oracle_on_the_same_state(dtype):
    """Device diagnostics (single-handle and batched) against the oracle's
    plain definitions evaluated on the state the GPU exported."""
    films, cfgs = [], []
    for h0, th, p in inputs.sliding_drops(count=3, lx_range=(128, 256), seed=3):
        p = dict(p, theta_uniform=float(th[0, 0]))
        films.append(ThinFilm(p, h0, None, dtype=dtype))
        cfgs.append(cfg_of(p))
    h_wet = 2 * inputs.DEFAULTS["hstar"]
    # FP32 h per node carries ~1e-7 relative rounding (the oracle sums the
    # exported populations in double)
    tol = 1e-12 if dtype == "f64" else 1e-6
    with FilmBatch(films) as B:
        B.step(300)
        rows = B.diagnostics(h_wet, mode=(2, 1)).cpu().numpy()
        for f, c, row in zip(films, cfgs, rows):
            single = f.diagnostics(h_wet, mode=(2, 1)).cpu().numpy()
            ref = O.film_diagnostics(c, f.get_state().cpu().numpy(), h_wet, mode=(2, 1))
            scale = np.abs(ref).max()
            assert np.abs(single - row).max() <= 1e-12 * scale
            for k, name in enumerate(L.DIAG_FIELDS):
                if name == "wet_area":
                    assert abs(row[k] - ref[k]) <= (0 if dtype == "f64" else 2)
                else:  # sums judged against the largest sum of the row
                    assert abs(row[k] - ref[k]) <= tol * scale, (name, row[k], ref[k])
    # drops are pushed along +x, so their momentum points that way
    assert (rows[:, 2] > 0).all()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 2e-3)])
def test_term_norms_match_oracle_on_the_same_state(dtype, tol):
    """Appendix term balance (Eq. magnitude) on a sliding drop: device L2
    norms against the oracle's composition of its pinned stencils on the
    exported state.  In FP32 the dissipation term is a difference of
    near-equal neighbours of j, so it is compared to 2e-3 relative."""
    (h0, th, p), = inputs.sliding_drops(count=1, lx_range=(256, 256), seed=5)
    p = dict(p, theta_uniform=float(th[0, 0]), tau=0.8)
    sim = ThinFilm(p, h0, None, dtype=dtype)
    sim.step(400)
    tn = sim.term_norms().cpu().numpy()
    c = cfg_of(p)
    ref = O.term_norms(c, O.kappa_field(c, p["theta_uniform"]), sim.get_state().cpu().numpy())
    assert np.all(np.abs(tn - ref) <= tol * np.abs(ref)), (tn, ref)


def test_batch_rejects_bad_input():
    h0, th, p = inputs.small_random(16, 16, seed=1)
    a = ThinFilm(p, h0, th, dtype="f32")
    b = ThinFilm(p, h0, th, dtype="f64")
    with pytest.raises(L.TfLbmError) as e:
        L.tf_lbm_batch_create([a.handle, b.handle])
    assert e.value.code == L.TF_LBM_ERR_ARG and "dtype" in str(e.value)
    with pytest.raises(L.TfLbmError) as e:
        L.tf_lbm_batch_create([a.handle, a.handle])
    assert "twice" in str(e.value)
    with pytest.raises(L.TfLbmError):
        L.tf_lbm_batch_create([])
    with FilmBatch([a]) as B:
        for bad in [dict(block_x=96), dict(rows=0), dict(graph_chunk=3), dict(queue=2)]:
            kw = dict(B.launch)
            kw.update(bad)
            with pytest.raises(L.TfLbmError):
                L.tf_lbm_batch_set_launch(B.batch, kw["block_x"], kw["rows"], kw["graph_chunk"], kw["queue"])
        with pytest.raises(L.TfLbmError):
            B.step(-1)
        host = np.zeros(12)
        with pytest.raises(L.TfLbmError):
            L.tf_lbm_batch_diagnostics(B.batch, 0.1, 1, 0, host.ctypes.data)
        with pytest.raises(L.TfLbmError):
            L.tf_lbm_diagnostics(a.handle, 0.1, 1, 0, host.ctypes.data)
        with pytest.raises(L.TfLbmError):
            L.tf_lbm_term_norms(a.handle, host.ctypes.data)


def test_persistent_queue_with_more_items_than_resident_ctas():
    """One-row bands on eight 256 x 256 domains give ~10k items, several
    times the resident CTAs, so every persistent CTA takes many items from
    the counter (and the counter is reset between launches): the result is
    bit-identical to one CTA per item, and the batch matches the oracle."""
    specs = []
    for i in range(8):
        h0, th, p = inputs.small_random(256, 256, seed=40 + i, amp=0.05)
        specs.append((h0, th if i % 2 else None, dict(p, theta_uniform=np.radians(30.0))))
    states = {}
    for queue in (0, 1):
        films = make_films(specs, "f32")
        with FilmBatch(films) as B:
            B.set_launch(block_x=64, rows=1, graph_chunk=4, queue=queue)
            assert B.items > 4 * 16 * torch.cuda.get_device_properties(0).multi_processor_count
            B.step(10)
            states[queue] = [f.get_state().cpu().numpy() for f in films]
            if queue == 1:
                for (h0, th, p), f in zip(specs[:2], films[:2]):
                    assert rel_linf(host_h(f), oracle_h(h0, th, p, 10)) <= TOL["f32"]
        for f in films:
            f.close()
    for a, b in zip(states[0], states[1]):
        assert np.array_equal(a, b)
