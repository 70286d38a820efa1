"""Driver for the bounds-checked debug build (run by tests/test_gpu_bounds.py
in a child process whose TFLBM_LIBRARY names that build).

Runs the tiny and ragged lattices of the parity tests through every step
pipeline that applies, every storage type and both relaxation kernels, plus
one batch of uneven domains, and checks that no step kernel reported an
index outside its buffers (TF_LBM_STATUS_BOUNDS) and that the results still
match the FP64 oracle.  Exit status 0 on success; the failures are printed
otherwise.
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle as O  # noqa: E402
from paper_1810_07642_gb300 import _lib as L  # noqa: E402
from paper_1810_07642_gb300 import inputs  # noqa: E402
from paper_1810_07642_gb300.film import FilmBatch, ThinFilm  # noqa: E402

TOL = {"f32": 1e-5, "f64": 1e-11, "f16": 1e-3, "bf16": 1e-3}
SIZES = [(1, 1), (2, 1), (3, 3), (2, 9), (5, 7), (6, 1), (16, 9), (37, 29), (64, 48), (130, 70), (200, 33),
         (304, 13)]
STEPS = 30


def pipelines(nx, dtype):
    out = [1]
    if dtype in ("f32", "f64"):
        out.append(2)
    if nx % 8 == 0 and nx >= 16:
        out.append(0)
    if nx % 2 == 0 and dtype != "f64":
        out.append(3)
    return out


def run_batch(specs, dtype, pipe, failures):
    """Step a batch through both queue modes and compare every domain with
    the oracle; returns the number of domains checked."""
    films = [ThinFilm(p, h0, th, dtype=dtype) for h0, th, p in specs]
    with FilmBatch(films) as B:
        for queue in (0, 1):
            B.set_launch(block_x=64, rows=5, graph_chunk=0, queue=queue, pipeline=pipe)
            B.step(STEPS // 2)
    for f, (h0, th, p) in zip(films, specs):
        cfg = O.Config(**{k: v for k, v in p.items() if k in O.Config.__dataclass_fields__})
        ff = O.init(cfg, h0)
        O.step(cfg, O.kappa_field(cfg, th), ff, 2 * (STEPS // 2))
        ho = ff.sum(0)
        status = f.check()
        err = float(np.abs(f.h().double().cpu().numpy() - ho).max() / np.abs(ho).max())
        if status or not err <= TOL[dtype]:
            failures.append(("batch", pipe, f.nx, f.ny, dtype, status, err))
        f.close()
    return len(films)


def main():
    assert L.library_path() == os.environ.get("TFLBM_LIBRARY"), "not the checked build"
    failures, runs = [], 0
    for nx, ny in SIZES:
        h0, th, p = inputs.small_random(nx, ny, seed=nx * 31 + ny, amp=0.05)
        for tau in (1.0, 0.8):
            pp = dict(p, tau=tau, g=2e-4, gx_body=2e-5, delta=1.0)
            cfg = O.Config(**{k: v for k, v in pp.items() if k in O.Config.__dataclass_fields__})
            f = O.init(cfg, h0)
            O.step(cfg, O.kappa_field(cfg, th), f, STEPS)
            ho = f.sum(0)
            for dtype in ("f32", "f64", "f16", "bf16"):
                for pipe in pipelines(nx, dtype):
                    for bx in (64, 128, 256):
                        sim = ThinFilm(pp, h0, th, dtype=dtype)
                        sim.set_launch(block_x=bx, rows=5, graph_chunk=0, pipeline=pipe)
                        sim.step(STEPS)
                        status = sim.check()
                        h = sim.h().double().cpu().numpy()
                        sim.close()
                        runs += 1
                        err = float(np.abs(h - ho).max() / np.abs(ho).max())
                        if status or not err <= TOL[dtype]:
                            failures.append((nx, ny, tau, dtype, pipe, bx, status, err))
    # batches of uneven domains (one narrower than a CTA, one smaller than
    # the stencil): odd widths with the one-column kernel, even widths with
    # the two-column kernel
    for sizes, pipe in (([(37, 29), (130, 70), (64, 32), (5, 7)], 1),
                        ([(38, 29), (130, 70), (64, 32), (6, 7)], 3)):
        specs = []
        for i, (nx, ny) in enumerate(sizes):
            h0, th, p = inputs.small_random(nx, ny, seed=50 + i, amp=0.1)
            specs.append((h0, th, dict(p, tau=0.9)))
        for dtype in ("f32", "f16"):
            runs += run_batch(specs, dtype, pipe, failures)
    print(f"{runs} runs through the bounds-checked build, {len(failures)} failures")
    for x in failures[:50]:
        print("FAIL", x)
    return 1 if failures else 0


if __name__ == "__main__":
    torch.cuda.set_device(0)
    sys.exit(main())
