"""Torch-facing wrapper of libtflbm: one thin-film simulation on one GPU.

PyTorch only provides device memory and streams here; every step of the method
runs in the library's CUDA kernels (include/tflbm.h).
"""
from __future__ import annotations

import math

import torch

from . import _lib as L

# storage name -> (library dtype code, torch dtype of fields and inputs)
_DT = {"f32": (L.TF_LBM_F32, torch.float32), "f64": (L.TF_LBM_F64, torch.float64),
       "f16": (L.TF_LBM_F16, torch.float32), "bf16": (L.TF_LBM_BF16, torch.float32)}


def make_params(nx, ny, dtype="f32", tau=1.0, gamma=0.01, g=0.0, delta=1.0, hstar=0.07,
                n_exp=3, m_exp=2, pi_sign=1, gx_body=0.0, gy_body=0.0, theta_uniform=0.0,
                forcing=0, **_ignored) -> L.Params:
    code = _DT[dtype][0]
    return L.Params(int(nx), int(ny), code, int(n_exp), int(m_exp), int(pi_sign), int(forcing), float(tau),
                    float(gamma), float(g), float(delta), float(hstar), float(gx_body),
                    float(gy_body), float(theta_uniform))


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class ThinFilm:
    """A periodic nx x ny thin-film simulation (Section II of the paper).

    h0 and theta are (ny, nx) tensors (any device/dtype; copied to the GPU in
    the run's dtype).  theta=None uses ``theta_uniform`` (radians) everywhere.
    """

    def __init__(self, params: dict, h0, theta=None, dtype: str = "f32", stream=None,
                 device="cuda"):
        if dtype not in _DT:
            raise ValueError(f"dtype must be one of {list(_DT)}")
        self.dtype_name = dtype
        self.tdtype = _DT[dtype][1]
        self.device = torch.device(device)
        self.params = dict(params)
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self.cparams = make_params(dtype=dtype, **params)
        self.stream = stream
        h0 = torch.as_tensor(h0).to(device=self.device, dtype=self.tdtype).contiguous()
        if tuple(h0.shape) != (self.ny, self.nx):
            raise ValueError(f"h0 must have shape {(self.ny, self.nx)}")
        th = None
        if theta is not None:
            th = torch.as_tensor(theta).to(device=self.device, dtype=self.tdtype).contiguous()
            if tuple(th.shape) != (self.ny, self.nx):
                raise ValueError(f"theta must have shape {(self.ny, self.nx)}")
        st = _stream_ptr(stream)
        self.handle = L.tf_lbm_init(self.cparams, h0.data_ptr(),
                                    th.data_ptr() if th is not None else None, st)
        # the device copies of h0 and theta (kept for gradient tapes)
        self.h0_dev, self.theta_dev = h0, th
        self._keep = (h0, th)
        self._st = st

    # -- stepping and outputs -------------------------------------------------
    def step(self, nsteps: int = 1):
        L.tf_lbm_step(self.handle, nsteps, self._st)

    def _field(self):
        return torch.empty((self.ny, self.nx), dtype=self.tdtype, device=self.device)

    def moments(self, want=("h", "ux", "uy")):
        out = {k: self._field() for k in want}
        L.tf_lbm_moments(self.handle, *(out[k].data_ptr() if k in out else None
                                        for k in ("h", "ux", "uy")), self._st)
        return out

    def h(self):
        return self.moments(("h",))["h"]

    def pressure_force(self):
        out = {k: self._field() for k in ("p", "fx", "fy")}
        L.tf_lbm_pressure_force(self.handle, out["p"].data_ptr(), out["fx"].data_ptr(),
                                out["fy"].data_ptr(), self._st)
        return out

    def mass(self) -> float:
        return L.tf_lbm_mass(self.handle, self._st)

    def check(self) -> int:
        return L.tf_lbm_check(self.handle, self._st)

    def get_state(self):
        """Post-streaming populations f_l(x, t) as a float64 (9, ny, nx) tensor."""
        f = torch.empty((9, self.ny, self.nx), dtype=torch.float64, device=self.device)
        L.tf_lbm_get_state(self.handle, f.data_ptr(), self._st)
        return f

    def set_state(self, f):
        f = torch.as_tensor(f).to(device=self.device, dtype=torch.float64).contiguous()
        L.tf_lbm_set_state(self.handle, f.data_ptr(), self._st)
        self._keep = (f,)

    @property
    def time(self) -> int:
        return L.tf_lbm_time(self.handle)

    @property
    def launch(self):
        l = L.tf_lbm_get_launch(self.handle)
        return dict(block_x=l.block_x, rows=l.rows, graph_chunk=l.graph_chunk, pipeline=l.pipeline)

    def set_launch(self, block_x=None, rows=None, graph_chunk=None, pipeline=None):
        cur = self.launch
        L.tf_lbm_set_launch(self.handle, block_x or cur["block_x"], rows or cur["rows"],
                            cur["graph_chunk"] if graph_chunk is None else graph_chunk,
                            cur["pipeline"] if pipeline is None else pipeline)

    def tune(self, trial_steps: int = 16):
        """Time candidate launch shapes on this run's own state, keep the
        fastest and return it (the state and time are left as they were)."""
        l = L.tf_lbm_tune(self.handle, trial_steps, self._st)
        return dict(block_x=l.block_x, rows=l.rows, graph_chunk=l.graph_chunk, pipeline=l.pipeline)

    def diagnostics(self, h_wet: float, mode=(1, 0), out=None):
        """Film diagnostics of the current state: a float64 device tensor of
        the tf_lbm_diag fields (_lib.DIAG_FIELDS), no host synchronisation."""
        if out is None:
            out = torch.empty(len(L.DIAG_FIELDS), dtype=torch.float64, device=self.device)
        L.tf_lbm_diagnostics(self.handle, h_wet, mode[0], mode[1], out.data_ptr(), self._st)
        return out

    def term_norms(self, out=None):
        """L2 norms of the pressure, friction and dissipation terms (x
        components) of the paper's appendix, as a float64 device tensor."""
        if out is None:
            out = torch.empty(3, dtype=torch.float64, device=self.device)
        L.tf_lbm_term_norms(self.handle, out.data_ptr(), self._st)
        return out

    def close(self):
        if getattr(self, "handle", None):
            L.tf_lbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class FilmBatch:
    """Many independent ThinFilm runs of uneven sizes (one dtype) advanced by
    one batched launch per step (tf_lbm_batch_*).  The films stay usable on
    their own (state, moments, mass) and must outlive the batch."""

    def __init__(self, films, stream=None):
        self.films = list(films)
        if not self.films:
            raise ValueError("a batch needs at least one film")
        self._st = _stream_ptr(stream)
        self.device = self.films[0].device
        self.batch = L.tf_lbm_batch_create([f.handle for f in self.films], self._st)

    def step(self, nsteps: int = 1):
        L.tf_lbm_batch_step(self.batch, nsteps, self._st)

    @property
    def items(self) -> int:
        return L.tf_lbm_batch_items(self.batch)

    @property
    def launch(self):
        l = L.tf_lbm_batch_get_launch(self.batch)
        return dict(block_x=l.block_x, rows=l.rows, graph_chunk=l.graph_chunk, queue=l.queue,
                    pipeline=l.pipeline)

    def set_launch(self, block_x=None, rows=None, graph_chunk=None, queue=None, pipeline=None):
        cur = self.launch
        L.tf_lbm_batch_set_launch(self.batch, block_x or cur["block_x"], rows or cur["rows"],
                                  cur["graph_chunk"] if graph_chunk is None else graph_chunk,
                                  cur["queue"] if queue is None else queue,
                                  cur["pipeline"] if pipeline is None else pipeline)

    def tune(self, trial_steps: int = 16):
        l = L.tf_lbm_batch_tune(self.batch, trial_steps, self._st)
        return dict(block_x=l.block_x, rows=l.rows, graph_chunk=l.graph_chunk, queue=l.queue,
                    pipeline=l.pipeline)

    def diagnostics(self, h_wet: float, mode=(1, 0), out=None):
        """(count, 12) float64 device tensor of tf_lbm_diag rows, one per film."""
        if out is None:
            out = torch.empty((len(self.films), len(L.DIAG_FIELDS)), dtype=torch.float64,
                              device=self.device)
        L.tf_lbm_batch_diagnostics(self.batch, h_wet, mode[0], mode[1], out.data_ptr(), self._st)
        return out

    def close(self):
        if getattr(self, "batch", None):
            L.tf_lbm_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def theta_radians(deg) -> float:
    return math.radians(deg)
