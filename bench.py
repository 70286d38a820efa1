"""Benchmark of the fused thin-film D2Q9 step (MLUPS and fraction of HBM roofline).

Workload: chemically patterned dewetting, 2048 x 2048 periodic lattice, FP32
populations; h0 = 1 + U(-1e-2, 1e-2), theta(x) = stripes of period 256 at
10/40 degrees plus 32 seeded discs at 10 degrees (Section III D of the paper,
synthetic stand-in).  Its populations (2 x 151 MB) and kappa field (17 MB)
exceed the 129 MB L2, so no L2 flush is needed between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {tflbm,reference}]
                  [--workload {patterned,sweep,adjoint}] [--storage {f32,f16,bf16}]

One step = one time step of the whole lattice = one launch of the fused
kernel.  `value` is MLUPS = nodes x steps / time / 1e6 over all ranks (each
rank runs an independent replica: the method needs no exchange between
independent simulations).  `--impl reference` times the FP64 CPU oracle (the
plain restatement of the method used by the tests) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (D2Q9 thin-film step) and % of HBM roofline; adjoint/forward cost ratio"
N_SIDE = 2048
BYTES_PER_LU = 76  # FP32: 9 populations read + 9 written + kappa(x)
_CSRC = "paper_1810_07642_gb300/csrc/"
# committed ncu summary of the default step kernel of each storage form and
# the sources that kernel is compiled from (the summary's kernel_hash)
PROFILES = {
    "f32": ("k_step2_f32_patterned_2048.txt",
            [_CSRC + "tflbm_step.cuh", _CSRC + "tflbm_step2.cuh", _CSRC + "step2_f32.cu",
             _CSRC + "tflbm_internal.h"]),
    "f16": ("k_step2_f16_patterned_2048.txt",
            [_CSRC + "tflbm_step.cuh", _CSRC + "tflbm_step2.cuh", _CSRC + "step2_f16.cu",
             _CSRC + "tflbm_internal.h"]),
}
WORKLOAD = ("chemically patterned dewetting, 2048x2048 periodic D2Q9 thin film, FP32 "
            "populations; h0=1+U(-1e-2,1e-2); theta stripes period 256 (10/40 deg) + 32 "
            "seeded discs (10 deg); gamma=0.01, h*=0.07, (n,m)=(3,2), tau=1, delta=1, g=0")


def kernel_hash(storage: str = "f32") -> str:
    """Hash of the sources of the default step kernel for one storage form."""
    h = hashlib.sha256()
    for rel in PROFILES[storage][1]:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled_traffic(storage: str = "f32"):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary
    (lines "key: value"), if it was taken on the current kernel source."""
    if storage not in PROFILES:
        return None, None
    path = os.path.join(ROOT, "profiles", PROFILES[storage][0])
    if not os.path.exists(path):
        return None, None
    d = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                d[k.strip()] = v.strip()
    if d.get("kernel_hash") != kernel_hash(storage) or "dram_bytes_per_launch" not in d:
        return None, d
    return float(d["dram_bytes_per_launch"]), d


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(nodes: int, steps: int, world: int, t_max: float) -> float:
    """Whole-job MLUPS: every rank advanced its own replica of `nodes` nodes."""
    return world * nodes * steps / t_max / 1e6


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_cpu_baseline(budget_s: float = 15.0):
    """The FP64 oracle as it stands, on a bounded sample of the workload: whole
    2048^2 steps from the same h0 / theta, as many as fit the budget."""
    import oracle as O
    from paper_1810_07642_gb300 import inputs
    h0, th, p = inputs.patterned_dewetting(N_SIDE, seed=0)
    cfg = O.Config(**{k: v for k, v in p.items() if k in O.Config.__dataclass_fields__})
    kap = O.kappa_field(cfg, th)
    f = O.init(cfg, h0)
    t0 = time.perf_counter()
    O.step(cfg, kap, f, 1)
    t1 = time.perf_counter() - t0
    n = int(max(2, min(400, budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    O.step(cfg, kap, f, n)
    dt = time.perf_counter() - t0
    out = {"value": N_SIDE * N_SIDE * n / dt / 1e6, "unit": "MLUPS", "cores": O.num_threads(),
           "kind": "oracle",
           "sample": f"{n} full 2048x2048 steps of the FP64 oracle on the same inputs "
                     f"({dt:.1f} s, {O.num_threads()} OpenMP threads)"}
    # the same oracle on one thread, over a 2048 x 64 band of the workload
    threads = O.num_threads()
    try:
        O.set_num_threads(1)
        cfg.ny = 64
        kb = O.kappa_field(cfg, th[:64])
        fb = O.init(cfg, np.ascontiguousarray(h0[:64]))
        t0 = time.perf_counter()
        O.step(cfg, kb, fb, 1)
        t1 = time.perf_counter() - t0
        nb = int(max(2, min(200, 5.0 / max(t1, 1e-6))))
        t0 = time.perf_counter()
        O.step(cfg, kb, fb, nb)
        dt1 = time.perf_counter() - t0
        out["value_1_thread"] = N_SIDE * 64 * nb / dt1 / 1e6
        out["sample_1_thread"] = f"{nb} steps of a 2048x64 periodic band ({dt1:.1f} s, 1 thread)"
    finally:
        O.set_num_threads(threads)
    # smaller lattices of the paper's workloads (Rayleigh-Taylor 128^2, drop
    # 512^2), all threads and one thread, short runs
    by_size = {}
    for label, mk, steps_all, steps_one in (
            ("rayleigh_taylor_128", lambda: inputs.rayleigh_taylor(128, mode=1, g=-1e-4), 2000, 200),
            ("sessile_drop_512", lambda: inputs.sessile_drop(512), 200, 10)):
        hs, ths, ps = mk()
        c = O.Config(**{k: v for k, v in ps.items() if k in O.Config.__dataclass_fields__})
        ks = O.kappa_field(c, ths)
        rec = {}
        for nthr, nst in ((threads, steps_all), (1, steps_one)):
            O.set_num_threads(nthr)
            fs = O.init(c, hs)
            t0 = time.perf_counter()
            O.step(c, ks, fs, nst)
            rec[f"mlups_{nthr}_threads"] = c.nx * c.ny * nst / (time.perf_counter() - t0) / 1e6
        O.set_num_threads(threads)
        by_size[label] = rec
    out["by_size"] = by_size
    out["cpu"] = cpu_model()
    return out


def cpu_model() -> str:
    """CPU model of the host, from /proc/cpuinfo where it names one."""
    import platform
    try:
        with open("/proc/cpuinfo") as fh:
            info = fh.read().splitlines()
        for key in ("model name", "Model", "CPU part"):
            for line in info:
                if line.startswith(key):
                    return f"{platform.machine()}: {line.split(':', 1)[1].strip()}"
    except OSError:
        pass
    return platform.machine()


def storage_variants(steps: int = 2000, check_steps: int = 1000):
    """MLUPS of every storage form on the bench workload (default launch
    shapes, same timing rules), and the relative Linf error on h and the
    relative mass drift of every form against the FP64 oracle on the same
    2048^2 workload after `check_steps` steps (the oracle's whole run takes
    about a minute on the host cores)."""
    import torch
    import oracle as O
    from paper_1810_07642_gb300 import inputs
    from paper_1810_07642_gb300.film import ThinFilm
    out = {}
    h0, th, p = inputs.patterned_dewetting(N_SIDE, seed=0)
    for dt, bpl in (("f32", 76), ("f16", 44), ("bf16", 44), ("f64", 152)):
        sim = ThinFilm(p, h0, th, dtype=dt)
        sim.step(50)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        sim.step(steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[dt] = {"mlups": N_SIDE * N_SIDE / ms / 1e3, "bytes_per_lu": bpl,
                   "gbs": bpl * N_SIDE * N_SIDE / ms / 1e6, "launch": sim.launch}
        sim.close()
    cfg = O.Config(**{k: v for k, v in p.items() if k in O.Config.__dataclass_fields__})
    t0 = time.perf_counter()
    _, ho, _, _ = O.run(cfg, h0, th, check_steps)
    out["oracle_s"] = time.perf_counter() - t0
    for dt in ("f32", "f16", "bf16", "f64"):
        sim = ThinFilm(p, h0, th, dtype=dt)
        m0 = sim.mass()
        sim.step(check_steps)
        h = sim.h().double().cpu().numpy()
        out[dt][f"rel_linf_h_vs_oracle_2048_{check_steps}"] = float(np.abs(h - ho).max() / np.abs(ho).max())
        out[dt][f"mass_rel_drift_2048_{check_steps}"] = abs(sim.mass() - m0) / m0
        sim.close()
    out["f64"]["context"] = "the paper's FP64 code: 404.7 MLUPS at 2048^2 on a GTX 1080 Ti"
    out["speedup_f16_over_f32"] = out["f16"]["mlups"] / out["f32"]["mlups"]
    out["speedup_bf16_over_f32"] = out["bf16"]["mlups"] / out["f32"]["mlups"]
    return out


def adjoint_cost(n: int = 512, nsteps: int = 20000, repeats: int = 3):
    """Cost of one gradient of the inverse-design loss (checkpointed forward +
    backward with the hand-written adjoint) in units of a plain forward run,
    FP32, on the inverse-design workload (n^2, T = nsteps, sqrt(T)
    checkpoints).  Both are timed with CUDA events on the current stream,
    `repeats` times each; the median and the spread (max/min - 1) are
    reported."""
    import torch
    from paper_1810_07642_gb300 import inputs
    from paper_1810_07642_gb300.adjoint import evolve
    from paper_1810_07642_gb300.film import ThinFilm
    h0, th, tgt, p = inputs.inverse_design(n, seed=0)
    theta = torch.tensor(th, dtype=torch.float32, device="cuda", requires_grad=True)
    hh = torch.tensor(h0, dtype=torch.float32, device="cuda")
    tg = torch.tensor(tgt, dtype=torch.float32, device="cuda")

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def forward():
        sim = ThinFilm(p, h0, th)
        sim.step(nsteps)
        sim.h()
        sim.close()

    def gradient():
        theta.grad = None
        (0.5 * ((evolve(theta, hh, p, nsteps) - tg) ** 2).sum()).backward()

    # warm-up: first use of the kernels and of the graph capture paths
    (0.5 * ((evolve(theta, hh, p, 300) - tg) ** 2).sum()).backward()
    forward()
    t_fwd = sorted(timed(forward) for _ in range(repeats))
    t_grad = sorted(timed(gradient) for _ in range(repeats))
    med = lambda v: v[len(v) // 2]
    return {"workload": f"inverse design {n}x{n}, T={nsteps}, checkpoints every "
                        f"{int(math.ceil(math.sqrt(nsteps)))} steps, FP32",
            "timing": f"CUDA events, {repeats} runs each, median",
            "forward_s": med(t_fwd), "gradient_s": med(t_grad),
            "forward_spread": t_fwd[-1] / t_fwd[0] - 1, "gradient_spread": t_grad[-1] / t_grad[0] - 1,
            "gradient_over_forward": med(t_grad) / med(t_fwd)}


def batched_sweep(steps: int = 30000, timed: int = 400):
    """The batched sliding-drop sweep: 64 uneven domains (256x128 .. 1024x512,
    FP32, uniform theta = 40 deg, delta = 1, tangential body force from Bond
    numbers log-spaced over 0.05 .. 1).  MLUPS of one batched launch per step
    (default and autotuned shape) against the same domains stepped one after
    another by single-domain launches; the batched path's error against the
    FP64 oracle on four reduced domains; and the steady capillary number
    Ca = nu U / gamma against Bo after `steps` steps, U the wetted-region
    momentum over the wetted mass (h > 2 h*), reduced on the device."""
    import torch
    import oracle as O
    from paper_1810_07642_gb300 import inputs
    from paper_1810_07642_gb300.film import FilmBatch, ThinFilm

    def films_of(specs):
        return [ThinFilm(dict(p, theta_uniform=float(th[0, 0])), h0, None) for h0, th, p in specs]

    def mlups(fn, nodes, k):
        fn(4)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn(k)
        e1.record()
        torch.cuda.synchronize()
        return nodes * k / e0.elapsed_time(e1) / 1e3

    specs = inputs.sliding_drops(count=64, seed=0)
    films = films_of(specs)
    nodes = sum(f.nx * f.ny for f in films)

    def seq(k):
        for f in films:
            f.step(k)

    out = {"domains": len(films), "nodes": nodes}
    out["mlups_single_domain_launches"] = mlups(seq, nodes, timed)
    B = FilmBatch(films)
    out["default_launch"] = B.launch
    out["mlups_batched_default"] = mlups(B.step, nodes, timed)
    out["tuned_launch"] = B.tune(16)
    out["items"] = B.items
    out["mlups_batched_tuned"] = mlups(B.step, nodes, timed)
    out["speedup_batched_over_single_domain_launches"] = (out["mlups_batched_tuned"] /
                                                         out["mlups_single_domain_launches"])
    # the persistent work queue and graph replay, beside the tuned shape
    forms = {}
    for queue in (0, 1):
        for chunk in (0, 64):
            B.set_launch(queue=queue, graph_chunk=chunk)
            forms[f"queue{queue}_graph{chunk}"] = mlups(B.step, nodes, timed)
    out["mlups_forms_at_tuned_shape"] = forms
    # the one-column kernel in the shape its own tuning chose for this sweep
    # (64-column CTAs, 60-row bands, one CTA per item, no graph)
    B.set_launch(block_x=64, rows=60, queue=0, graph_chunk=0, pipeline=1)
    out["mlups_batched_one_column"] = mlups(B.step, nodes, timed)
    B.set_launch(**out["tuned_launch"])
    B.close()
    for f in films:
        f.close()
    # Ca vs Bo (the paper's sliding-drop study), fresh runs in the tuned shape;
    # U is read at two late times and a drop counts as terminal when it
    # changed by less than 3% between them
    films = films_of(specs)
    B = FilmBatch(films)
    B.set_launch(**out["tuned_launch"])
    h_wet = 2 * inputs.DEFAULTS["hstar"]
    nu = (specs[0][2]["tau"] - 0.5) / 3.0
    gamma = specs[0][2]["gamma"]
    bo = np.array([p["bond"] for _, _, p in specs])
    t_early = steps - steps // 6
    B.step(t_early)
    d = B.diagnostics(h_wet).cpu().numpy()
    ca_early = nu * (d[:, 2] / d[:, 1]) / gamma
    B.step(steps - t_early)
    d = B.diagnostics(h_wet).cpu().numpy()
    ca = nu * (d[:, 2] / d[:, 1]) / gamma
    terminal = np.abs(ca - ca_early) <= 0.03 * np.abs(ca)
    # sliding drops: terminal and moving (pinned drops keep a tiny residual U)
    sl = terminal & (ca > 0.05 * ca.max())
    rec = {"steps": steps, "early_steps": t_early, "bo": [round(float(x), 4) for x in bo],
           "ca": [float(f"{x:.4g}") for x in ca], "ca_early": [float(f"{x:.4g}") for x in ca_early],
           "terminal": [bool(x) for x in terminal], "terminal_count": int(terminal.sum()),
           "check_status_nonzero": int(sum(1 for f in films if f.check()))}
    if sl.sum() >= 3:
        slope, icpt = np.polyfit(bo[sl], ca[sl], 1)
        fit = slope * bo[sl] + icpt
        r2 = 1 - ((ca[sl] - fit) ** 2).sum() / ((ca[sl] - ca[sl].mean()) ** 2).sum()
        rec["fit_terminal_sliding_drops"] = {"slope": float(slope), "bo_c": float(-icpt / slope), "r2": float(r2),
                                             "count": int(sl.sum()),
                                             "bo_range": [float(bo[sl].min()), float(bo[sl].max())]}
    out["ca_vs_bo"] = rec
    B.close()
    for f in films:
        f.close()
    # accuracy of the batched path: four reduced sweep domains, 1000 steps,
    # every storage type
    small = inputs.sliding_drops(count=4, seed=1, lx_range=(128, 256))
    acc = {}
    refs = []
    for h0, th, p in small:
        cfg = O.Config(**{k: v for k, v in dict(p, theta_uniform=float(th[0, 0])).items()
                          if k in O.Config.__dataclass_fields__})
        refs.append(O.run(cfg, h0, th, 1000)[1])
    for dt in ("f32", "f16", "bf16"):
        sf = [ThinFilm(dict(p, theta_uniform=float(th[0, 0])), h0, None, dtype=dt) for h0, th, p in small]
        err = 0.0
        with FilmBatch(sf) as SB:
            SB.step(1000)
            for f, ho in zip(sf, refs):
                h = f.h().double().cpu().numpy()
                err = max(err, float(np.abs(h - ho).max() / np.abs(ho).max()))
        for f in sf:
            f.close()
        acc[dt] = err
    out["rel_linf_h_vs_oracle_4_domains_1000"] = acc
    return out


def small_workloads():
    """Configs 1 and 2, measured with the device diagnostics.

    Rayleigh-Taylor (128^2, g = -1e-4, 2000 steps, FP64 and FP32): growth
    rate of the seeded mode fitted from its Fourier amplitude over steps
    100..2000, beside Eq. (RTgrowth)'s continuum rate (the scheme's explicit
    friction lowers it, see the design notes), mass drift, and MLUPS of this
    L2-resident, launch-bound lattice (graph-replayed steps).
    Sessile drop (512^2, r_b = 120, h_d = 20, theta = 20 deg, 50k steps FP32,
    delta in {0, 1, 2}): contact radius every 2500 steps and the final
    apparent angle (threshold h* + 0.01 h_d); delta = 0 diverges (explicit
    friction on the precursor) and is reported with the step it was found."""
    import torch
    from paper_1810_07642_gb300 import diagnostics as D
    from paper_1810_07642_gb300 import inputs
    from paper_1810_07642_gb300.film import ThinFilm
    import oracle as O
    out = {"rayleigh_taylor": {}, "sessile_drop": {}}
    h0, th, p = inputs.rayleigh_taylor(128, mode=1, g=-1e-4)
    k = 2 * math.pi / 128
    nu = (p["tau"] - 0.5) / 3
    cont = (1e-4 / (3 * nu)) * (k * k - (p["gamma"] / 1e-4) * k ** 4)
    # the FP64 oracle under both readings of the forcing (Eq. LBE as printed,
    # and the labelled second-order alternative), same fit
    xs = np.exp(-1j * k * np.arange(128))
    for forcing in (0, 1):
        cfg = O.Config(**{kk: v for kk, v in p.items() if kk in O.Config.__dataclass_fields__})
        cfg.forcing = forcing
        kap = O.kappa_field(cfg, th)
        f = O.init(cfg, h0)
        ts, la = [], []
        for t in range(0, 2001, 100):
            if t:
                O.step(cfg, kap, f, 100)
            if t >= 100:
                hh = f.sum(0)
                ts.append(t)
                la.append(math.log(abs(((hh - hh.mean()) @ xs).mean())))
        out["rayleigh_taylor"][f"oracle_forcing_{forcing}"] = {
            "sigma_fit_per_step": float(np.polyfit(ts, la, 1)[0]), "sigma_eq_rtgrowth": cont,
            "reading": "Eq. (LBE) as printed" if forcing == 0 else "second-order forcing (labelled alternative)"}
    for dt in ("f64", "f32"):
        sim = ThinFilm(p, h0, th, dtype=dt)
        m0 = sim.mass()
        ts, la = [], []
        for t in range(0, 2001, 100):
            if t:
                sim.step(100)
            if t >= 100:
                ts.append(t)
                la.append(math.log(D.mode_amplitude(sim.diagnostics(0.0, mode=(1, 0)).cpu().numpy(),
                                                    128, 128)))
        sig = float(np.polyfit(ts, la, 1)[0])
        m1 = sim.mass()
        launch = sim.tune(16)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sim.step(128)
        e0.record()
        sim.step(4096)
        e1.record()
        torch.cuda.synchronize()
        out["rayleigh_taylor"][dt] = {"sigma_fit_per_step": sig, "sigma_eq_rtgrowth": cont,
                                      "mass_rel_drift_2000": abs(m1 - m0) / m0,
                                      "mlups_l2_resident_launch_bound": 128 * 128 * 4096 /
                                      e0.elapsed_time(e1) / 1e3, "tuned_launch": launch}
        sim.close()
    for delta in (0.0, 1.0, 2.0):
        h0, th, p = inputs.sessile_drop(512, rb=120.0, hd=20.0, theta_deg=20.0, delta=delta)
        p = dict(p, theta_uniform=math.radians(20.0))
        sim = ThinFilm(p, h0, None)
        launch = sim.tune(16)
        m0 = sim.mass()
        curve, status, t = [], 0, 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        while t < 50000:
            e0.record()
            sim.step(2500)
            e1.record()
            t += 2500
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            status = sim.check()
            if status:
                break
            hd = sim.diagnostics(p["hstar"]).cpu().numpy()[5] - p["hstar"]
            g = D.drop(sim.diagnostics(p["hstar"] + 0.01 * hd).cpu().numpy(), p["hstar"], 512, 512,
                       p["tau"], p["gamma"])
            curve.append([t, round(g["contact_radius"], 3), round(math.degrees(g["theta"]), 3)])
        rec = {"status": status, "steps": t, "mlups": 512 * 512 * t / ms / 1e3, "tuned_launch": launch}
        if status:
            rec["diverged_by_step"] = t
        else:
            rec["r_theta_every_2500"] = curve
            rec["theta_final_deg"] = curve[-1][2]
            rec["mass_rel_drift"] = abs(sim.mass() - m0) / m0
        out["sessile_drop"][f"delta_{delta:g}"] = rec
        sim.close()
    return out


def term_balance(times=(1000, 5000, 20000)):
    """The appendix's term balance (Eq. magnitude): L2 norms of the
    x-components of the film-pressure term -h d_x p, the friction
    -nu alpha(h) u_x and the longitudinal dissipation
    nu lap(h u_x) + 2 nu d_x(div(h u)) over time, reduced on the device, for
    a spreading drop (256^2, cap r_b = 60, h_d = 10, theta = 20 deg), a
    sliding drop (256x128, Bo = 0.5) and a dewetting film (512^2 patterned),
    FP32, tau = 1."""
    from paper_1810_07642_gb300 import inputs
    from paper_1810_07642_gb300.film import ThinFilm
    cases = {}
    h0, th, p = inputs.sessile_drop(256, rb=60.0, hd=10.0, theta_deg=20.0)
    cases["spreading_drop_256"] = (h0, None, dict(p, theta_uniform=math.radians(20.0)))
    (h0, th, p), = inputs.sliding_drops(count=1, bo_min=0.5, bo_max=0.5, lx_range=(256, 256), seed=2)
    cases["sliding_drop_256x128"] = (h0, None, dict(p, theta_uniform=float(th[0, 0])))
    h0, th, p = inputs.patterned_dewetting(512, seed=1)
    cases["dewetting_512"] = (h0, th, p)
    out = {}
    for name, (h0, th, p) in cases.items():
        sim = ThinFilm(p, h0, th)
        t, rows = 0, []
        for T in times:
            sim.step(T - t)
            t = T
            tn = sim.term_norms().cpu().numpy()
            rows.append({"t": T, "pressure": float(tn[0]), "friction": float(tn[1]),
                         "dissipation": float(tn[2])})
        out[name] = rows
        sim.close()
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, each step one oracle time step on a
    2048 x R periodic band of the workload, R sized to fit a few minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    from paper_1810_07642_gb300 import inputs
    h0, th, p = inputs.patterned_dewetting(N_SIDE, seed=0)
    total = args.steps + args.warmup

    def band(rows):
        cfg = O.Config(**{k: v for k, v in p.items() if k in O.Config.__dataclass_fields__})
        cfg.ny = rows
        kap = O.kappa_field(cfg, th[:rows])
        return cfg, kap, O.init(cfg, np.ascontiguousarray(h0[:rows]))

    cfg, kap, f = band(64)
    t0 = time.perf_counter()
    O.step(cfg, kap, f, 2)
    per_node = (time.perf_counter() - t0) / (2 * N_SIDE * 64)
    rows = int(max(2, min(N_SIDE, 150.0 / total / per_node / N_SIDE)))
    cfg, kap, f = band(rows)
    for _ in range(args.warmup):
        O.step(cfg, kap, f, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.step(cfg, kap, f, 1)
    dt = time.perf_counter() - t0
    value = N_SIDE * rows * args.steps / dt / 1e6
    sample = (f"each step: one FP64 oracle time step on a {N_SIDE}x{rows} periodic band of "
              f"the workload ({O.num_threads()} OpenMP threads)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_rows": rows},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_tflbm(args):
    import torch
    from paper_1810_07642_gb300 import build, inputs
    from paper_1810_07642_gb300.film import ThinFilm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        if world == 1 and args.gpus > 1:
            raise SystemExit("--gpus N > 1 must be launched with torch.distributed.run")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()

    h0, th, p = inputs.patterned_dewetting(N_SIDE, seed=rank)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = ThinFilm(p, h0, th, dtype=args.storage, stream=stream)
    if args.launch:
        bx, rows, pipe = (int(v) for v in args.launch.split(","))
        sim.set_launch(block_x=bx, rows=rows, pipeline=pipe)
    launch = sim.launch
    nodes = N_SIDE * N_SIDE

    def barrier():
        if dist:
            dist.barrier()

    # warm-up
    sim.step(args.warmup)
    stream.synchronize()
    m0 = sim.mass()

    # timed region: K steps issued by one library call (its C loop launches
    # the fused kernel once per step, back to back on `stream`)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    total_ms = ev0.elapsed_time(ev1)
    t_local = total_ms / 1e3
    t_max = max_over_ranks(t_local, dist, "cuda")
    m1 = sim.mass()
    status = sim.check()
    value = aggregate_mlups(nodes, args.steps, world, t_max)

    # dominant kernel: the fused step, one launch per step, launches back to
    # back, so its average duration is the timed region over K
    kern_s = t_local / args.steps
    bpl = BYTES_PER_LU if args.storage == "f32" else 44  # 16-bit: 2 x (4 + 8 x 2) + 4
    achieved = bpl * nodes / kern_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic, prof = profiled_traffic(args.storage)

    # end to end through the public API with host buffers (pinned)
    h_host = torch.from_numpy(np.asarray(h0, np.float32)).pin_memory()
    th_host = torch.from_numpy(np.asarray(th, np.float32)).pin_memory()
    out_host = torch.empty((N_SIDE, N_SIDE), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        hd = h_host.to("cuda", non_blocking=True)
        thd = th_host.to("cuda", non_blocking=True)
        sim2 = ThinFilm(p, hd, thd, dtype=args.storage, stream=stream)
        sim2.set_launch(**launch)
        sim2.step(args.steps)
        hres = sim2.moments(("h",))["h"]
        out_host.copy_(hres, non_blocking=True)
    stream.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    sim2.close()
    e2e = {"value": aggregate_mlups(nodes, args.steps, world, t_e2e), "unit": "MLUPS",
           "h2d_bytes_per_step": (h_host.numel() + th_host.numel()) * 4 / args.steps,
           "d2h_bytes_per_step": out_host.numel() * 4 / args.steps,
           "job": f"upload h0+theta, init, {args.steps} steps, download h (host wall clock)"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cpu = oracle_cpu_baseline() if world == 1 else None
    clocks = clk.summary()
    extras = {}
    if world == 1 and not args.skip_extras and args.storage == "f32":
        extras["storage"] = storage_variants()
        extras["adjoint"] = adjoint_cost()
        extras["batched_sweep"] = batched_sweep()
        extras["small_workloads"] = small_workloads()
        extras["term_balance"] = term_balance()
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": N_SIDE, "ny": N_SIDE, "replicas": world,
                   "l2": "inputs larger than L2 (302 MB populations + 17 MB kappa > 129 MB): no flush",
                   "launch": launch, "bytes_per_lu": bpl, "storage": args.storage},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "kernel": ("k_step2<" if launch["pipeline"] == 3 else "k_step<") +
                               {"f32": "float", "f16": "__half", "bf16": "__nv_bfloat16"}[args.storage] + ",...>",
                     "kernel_ms": kern_s * 1e3},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "mass_rel_drift": abs(m1 - m0) / m0,
        "check_status": status,
        "context": {"paper_gtx1080ti_fp64_2048": 404.7},
    }
    line.update(extras)
    if "adjoint" in extras:
        line["adjoint_forward_cost_ratio"] = extras["adjoint"]["gradient_over_forward"]
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_sweep(args):
    """--workload sweep: the batched sliding-drop sweep as the timed step (one
    batched launch per step over all 64 domains, autotuned shape)."""
    import torch
    from paper_1810_07642_gb300 import build, inputs
    from paper_1810_07642_gb300.film import FilmBatch, ThinFilm
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    specs = inputs.sliding_drops(count=64, seed=rank)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        films = [ThinFilm(dict(p, theta_uniform=float(th[0, 0])), h0, None, stream=stream)
                 for h0, th, p in specs]
        B = FilmBatch(films, stream=stream)
    nodes = sum(f.nx * f.ny for f in films)
    if args.batch_launch:
        v = [int(x) for x in args.batch_launch.split(",")]
        B.set_launch(block_x=v[0], rows=v[1], graph_chunk=v[2], queue=v[3],
                     pipeline=v[4] if len(v) > 4 else None)
        launch = B.launch
    else:
        launch = B.tune(16)
    B.step(args.warmup)
    stream.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        B.step(args.steps)
        ev1.record(stream)
        stream.synchronize()
    if dist:
        dist.barrier()
    t_local = ev0.elapsed_time(ev1) / 1e3
    t_max = max_over_ranks(t_local, dist, "cuda")
    value = aggregate_mlups(nodes, args.steps, world, t_max)
    bpl = 72  # FP32, uniform theta: 9 populations read + 9 written
    achieved = bpl * nodes / (t_local / args.steps) / 1e9
    peak, peak_kind = measured_peaks()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "batched sliding-drop sweep: 64 periodic domains 256x128.."
                                       "1024x512 (seeded), FP32, theta=40 deg, delta=1, Bo "
                                       "log-spaced 0.05..1", "nodes": nodes, "launch": launch,
                           "items": B.items,
                           "l2": "inputs larger than L2 (2.3 GB populations): no flush"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None,
                             "peak_kind": f"{peak_kind} copy bandwidth",
                             "kernel": "k_step_batch<float,float,...>"},
                "gpu_launches": args.steps, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    B.close()
    for f in films:
        f.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_adjoint(args):
    """--workload adjoint: gradients of the inverse-design loss as the timed
    step (512^2, FP32, T = --adjoint-steps, sqrt(T) checkpoints): each step is
    one checkpointed forward run plus the backward sweep of the hand-written
    adjoint.  value = lattice updates of the forward horizon per second of
    gradient (MLUPS-equivalent); the cost ratio against a plain forward run
    of the same horizon is reported beside it."""
    import torch
    from paper_1810_07642_gb300 import build, inputs
    from paper_1810_07642_gb300.adjoint import evolve
    from paper_1810_07642_gb300.film import ThinFilm
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    n, T = 512, args.adjoint_steps
    h0, th, tgt, p = inputs.inverse_design(n, seed=rank)
    theta = torch.tensor(th, dtype=torch.float32, device="cuda", requires_grad=True)
    hh = torch.tensor(h0, dtype=torch.float32, device="cuda")
    tg = torch.tensor(tgt, dtype=torch.float32, device="cuda")

    def gradient(nsteps):
        theta.grad = None
        (0.5 * ((evolve(theta, hh, p, nsteps) - tg) ** 2).sum()).backward()

    for _ in range(args.warmup):
        gradient(300)
    sim = ThinFilm(p, h0, th)
    sim.step(100)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.step(T)
    sim.h()
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    sim.close()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            gradient(T)
        torch.cuda.synchronize()
        t_local = time.perf_counter() - t0
    t_max = max_over_ranks(t_local, dist, "cuda")
    every = int(math.ceil(math.sqrt(T)))
    nck = (T + every - 1) // every
    if rank == 0:
        line = {"metric": METRIC, "value": aggregate_mlups(n * n, T * args.steps, world, t_max),
                "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"inverse design gradient: {n}x{n} periodic, FP32, flat film "
                                       f"with 1e-2 noise, theta 30 deg + 5 deg noise, 8-drop target, L2 "
                                       f"loss, T={T}, checkpoints every {int(math.ceil(math.sqrt(T)))} "
                                       f"steps", "l2": "L2-resident lattice (20 MB); timed on the host "
                                       "clock around whole gradients"},
                "adjoint_forward_cost_ratio": t_local / args.steps / t_fwd,
                "forward_s": t_fwd,
                # per gradient: T forward steps, T - nck recomputed steps, T adjoint
                # steps, the seed, the initial-state adjoint and the final moments
                "gpu_launches": args.steps * (3 * T - nck + 3), "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="tflbm", choices=["tflbm", "reference"])
    ap.add_argument("--workload", default="patterned", choices=["patterned", "sweep", "adjoint"],
                    help="patterned: the 2048^2 dewetting run (default); sweep: the batched "
                         "64-domain sliding-drop sweep as the timed step; adjoint: gradients of "
                         "the 512^2 inverse-design loss")
    ap.add_argument("--adjoint-steps", type=int, default=20000,
                    help="adjoint workload: time steps of the forward horizon")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="population storage of the patterned workload (arithmetic is FP32)")
    ap.add_argument("--launch", default="",
                    help="patterned workload: block_x,rows,pipeline of the fused step instead of "
                         "the library's default shape")
    ap.add_argument("--batch-launch", default="",
                    help="sweep workload: block_x,rows,graph_chunk,queue[,pipeline] instead of autotuning")
    ap.add_argument("--skip-extras", action="store_true",
                    help="skip the 16-bit storage, adjoint and batched-sweep measurements")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    return run_tflbm(args)


if __name__ == "__main__":
    sys.exit(main())
