"""Differentiable thin-film evolution: torch.autograd.Function over the
library's gradient tape (checkpointed forward, hand-written adjoint kernels).

    h_T = evolve(theta, h0, params, nsteps)        # (ny, nx) tensors
    loss = ((h_T - target) ** 2).sum() / 2
    loss.backward()                                 # theta.grad, h0.grad

The adjoint is the exact derivative of the discrete step (Eqs. LBE,
equilibria, force, pfilm, disjoiningP, forcefric, alphafric, derivative,
n_laplace); dL/dtheta goes through kappa(theta) of Eq. (disjoiningP).  PyTorch
provides memory and autograd plumbing only; every step and every adjoint step
runs in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import _lib as L
from .film import ThinFilm


class _Tape:
    """Owns one library gradient tape and the simulation it runs on."""

    def __init__(self, sim: ThinFilm, nsteps: int, every: int):
        self.sim = sim
        self.tape = L.tf_lbm_tape_create(sim.handle, sim.h0_dev.data_ptr(),
                                         sim.theta_dev.data_ptr() if sim.theta_dev is not None else None,
                                         nsteps, every)

    def forward(self):
        L.tf_lbm_tape_forward(self.sim.handle, self.tape, self.sim._st)

    def backward(self, grad_h, want_theta, want_h0):
        sim = self.sim
        gh = grad_h.to(device=sim.device, dtype=sim.tdtype).contiguous()
        gth = torch.empty((sim.ny, sim.nx), dtype=sim.tdtype, device=sim.device) if want_theta else None
        gh0 = torch.empty((sim.ny, sim.nx), dtype=sim.tdtype, device=sim.device) if want_h0 else None
        L.tf_lbm_tape_backward(sim.handle, self.tape, gh.data_ptr(),
                               gth.data_ptr() if gth is not None else None,
                               gh0.data_ptr() if gh0 is not None else None, sim._st)
        return gth, gh0

    def close(self):
        if self.tape:
            L.tf_lbm_tape_destroy(self.tape)
            self.tape = None
        self.sim.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Evolve(torch.autograd.Function):
    """h_T = Evolve.apply(theta, h0, params, nsteps, dtype, every)."""

    @staticmethod
    def forward(ctx, theta, h0, params, nsteps, dtype="f32", every=0):
        sim = ThinFilm(params, h0.detach(), theta.detach() if theta is not None else None,
                       dtype=dtype, device=h0.device if h0.is_cuda else "cuda")
        tape = _Tape(sim, int(nsteps), int(every))
        tape.forward()
        h_t = sim.h()
        ctx.tape = tape
        ctx.in_dtypes = (theta.dtype if theta is not None else None, h0.dtype)
        return h_t

    @staticmethod
    def backward(ctx, grad_h):
        want_theta = ctx.needs_input_grad[0]
        want_h0 = ctx.needs_input_grad[1]
        gth, gh0 = ctx.tape.backward(grad_h, want_theta, want_h0)
        if gth is not None:
            gth = gth.to(ctx.in_dtypes[0])
        if gh0 is not None:
            gh0 = gh0.to(ctx.in_dtypes[1])
        ctx.tape.close()
        return gth, gh0, None, None, None, None


def evolve(theta, h0, params: dict, nsteps: int, dtype: str = "f32", every: int = 0):
    """Film height after nsteps steps, differentiable in theta and h0."""
    return Evolve.apply(theta, h0, params, nsteps, dtype, every)
