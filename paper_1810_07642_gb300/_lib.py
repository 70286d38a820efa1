"""ctypes binding of libtflbm (include/tflbm.h), with the same names.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  If the library has not been built, every entry point raises;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

TF_LBM_F32, TF_LBM_F64, TF_LBM_F16, TF_LBM_BF16 = 0, 1, 2, 3
TF_LBM_OK = 0
TF_LBM_ERR_ARG, TF_LBM_ERR_CUDA, TF_LBM_ERR_NOMEM = -1, -2, -3
TF_LBM_ERR_NONFINITE, TF_LBM_ERR_UNSUPPORTED = -4, -5
TF_LBM_STATUS_NONFINITE, TF_LBM_STATUS_NONPOSITIVE, TF_LBM_STATUS_TIMEOUT = 1, 2, 4
TF_LBM_STATUS_BOUNDS = 8

EXPORTED = [
    "tf_lbm_init", "tf_lbm_step", "tf_lbm_moments", "tf_lbm_pressure_force", "tf_lbm_mass",
    "tf_lbm_check", "tf_lbm_get_state", "tf_lbm_set_state", "tf_lbm_time", "tf_lbm_get_launch",
    "tf_lbm_set_launch", "tf_lbm_destroy", "tf_lbm_last_error", "tf_lbm_version",
    "tf_lbm_sum_noalloc", "tf_lbm_adjoint_step", "tf_lbm_tape_create", "tf_lbm_tape_forward",
    "tf_lbm_tape_backward", "tf_lbm_tape_destroy", "tf_lbm_tune", "tf_lbm_diagnostics",
    "tf_lbm_batch_create", "tf_lbm_batch_step", "tf_lbm_batch_get_launch", "tf_lbm_batch_set_launch",
    "tf_lbm_batch_tune", "tf_lbm_batch_diagnostics", "tf_lbm_batch_items", "tf_lbm_batch_destroy",
    "tf_lbm_batch_last_error", "tf_lbm_term_norms", "tf_lbm_set_wait_limit",
]
# fields of tf_lbm_diag, in order
DIAG_FIELDS = ("mass", "wet_mass", "wet_jx", "wet_jy", "wet_area", "h_max",
               "wet_cos_x", "wet_sin_x", "wet_cos_y", "wet_sin_y", "mode_cos", "mode_sin")
TF_LBM_NOALLOC_MAX_ELEMS = 67108864


class TfLbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tflbm error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    """Mirror of tf_lbm_params."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dtype", ctypes.c_int32),
        ("n_exp", ctypes.c_int32), ("m_exp", ctypes.c_int32), ("pi_sign", ctypes.c_int32),
        ("forcing", ctypes.c_int32), ("tau", ctypes.c_double), ("gamma", ctypes.c_double), ("g", ctypes.c_double),
        ("delta", ctypes.c_double), ("hstar", ctypes.c_double), ("gx_body", ctypes.c_double),
        ("gy_body", ctypes.c_double), ("theta_uniform", ctypes.c_double),
    ]


class Launch(ctypes.Structure):
    """Mirror of tf_lbm_launch."""
    _fields_ = [("block_x", ctypes.c_int32), ("rows", ctypes.c_int32),
                ("graph_chunk", ctypes.c_int32), ("pipeline", ctypes.c_int32)]


class BatchLaunch(ctypes.Structure):
    """Mirror of tf_lbm_batch_launch."""
    _fields_ = [("block_x", ctypes.c_int32), ("rows", ctypes.c_int32),
                ("graph_chunk", ctypes.c_int32), ("queue", ctypes.c_int32),
                ("pipeline", ctypes.c_int32)]


_lib = None
_VP = ctypes.c_void_p


def library_path() -> str:
    """The library this process loads: the in-tree build, or the build named
    by the TFLBM_LIBRARY environment variable (e.g. the bounds-checked debug
    build, paper_1810_07642_gb300.build.LIB_CHECKED)."""
    return os.environ.get("TFLBM_LIBRARY") or _build.LIB


def lib():
    """Load the library (see library_path); raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libtflbm is not built ({path} missing): run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    L.tf_lbm_init.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(Params), _VP, _VP, _VP]
    L.tf_lbm_step.argtypes = [_VP, i64, _VP]
    L.tf_lbm_moments.argtypes = [_VP, _VP, _VP, _VP, _VP]
    L.tf_lbm_pressure_force.argtypes = [_VP, _VP, _VP, _VP, _VP]
    L.tf_lbm_mass.argtypes = [_VP, ctypes.POINTER(ctypes.c_double), _VP]
    L.tf_lbm_check.argtypes = [_VP, ctypes.POINTER(i32), _VP]
    L.tf_lbm_get_state.argtypes = [_VP, _VP, _VP]
    L.tf_lbm_set_state.argtypes = [_VP, _VP, _VP]
    L.tf_lbm_time.argtypes = [_VP]
    L.tf_lbm_time.restype = i64
    L.tf_lbm_get_launch.argtypes = [_VP, ctypes.POINTER(Launch)]
    L.tf_lbm_set_launch.argtypes = [_VP, ctypes.POINTER(Launch)]
    L.tf_lbm_set_wait_limit.argtypes = [_VP, i32]
    L.tf_lbm_destroy.argtypes = [_VP]
    L.tf_lbm_destroy.restype = None
    L.tf_lbm_last_error.argtypes = [_VP]
    L.tf_lbm_last_error.restype = ctypes.c_char_p
    L.tf_lbm_version.restype = i32
    L.tf_lbm_sum_noalloc.argtypes = [_VP, i64, _VP, _VP]
    L.tf_lbm_adjoint_step.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP]
    L.tf_lbm_tape_create.argtypes = [_VP, _VP, _VP, i64, i32, ctypes.POINTER(_VP)]
    L.tf_lbm_tape_forward.argtypes = [_VP, _VP]
    L.tf_lbm_tape_backward.argtypes = [_VP, _VP, _VP, _VP, _VP]
    L.tf_lbm_tape_destroy.argtypes = [_VP]
    L.tf_lbm_tape_destroy.restype = None
    L.tf_lbm_tune.argtypes = [_VP, i32, ctypes.POINTER(Launch), _VP]
    L.tf_lbm_diagnostics.argtypes = [_VP, ctypes.c_double, i32, i32, _VP, _VP]
    L.tf_lbm_term_norms.argtypes = [_VP, _VP, _VP]
    L.tf_lbm_batch_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(_VP), i32, _VP]
    L.tf_lbm_batch_step.argtypes = [_VP, i64, _VP]
    L.tf_lbm_batch_get_launch.argtypes = [_VP, ctypes.POINTER(BatchLaunch)]
    L.tf_lbm_batch_set_launch.argtypes = [_VP, ctypes.POINTER(BatchLaunch)]
    L.tf_lbm_batch_tune.argtypes = [_VP, i32, ctypes.POINTER(BatchLaunch), _VP]
    L.tf_lbm_batch_diagnostics.argtypes = [_VP, ctypes.c_double, i32, i32, _VP, _VP]
    L.tf_lbm_batch_items.argtypes = [_VP]
    L.tf_lbm_batch_items.restype = i32
    L.tf_lbm_batch_destroy.argtypes = [_VP]
    L.tf_lbm_batch_destroy.restype = None
    L.tf_lbm_batch_last_error.argtypes = [_VP]
    L.tf_lbm_batch_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int, handle=None):
    if rc != TF_LBM_OK:
        msg = lib().tf_lbm_last_error(handle).decode(errors="replace")
        raise TfLbmError(rc, msg)


# ---- thin wrappers, same names as the C entry points (pointers are ints) ----

def tf_lbm_init(params: Params, h0: int, theta: int | None, stream: int = 0) -> int:
    h = _VP()
    rc = lib().tf_lbm_init(ctypes.byref(h), ctypes.byref(params), _VP(h0), _VP(theta or 0),
                           _VP(stream))
    _check(rc, None)
    return h.value


def tf_lbm_step(handle: int, nsteps: int, stream: int = 0) -> None:
    _check(lib().tf_lbm_step(_VP(handle), int(nsteps), _VP(stream)), _VP(handle))


def tf_lbm_moments(handle: int, h: int | None, ux: int | None, uy: int | None, stream: int = 0) -> None:
    _check(lib().tf_lbm_moments(_VP(handle), _VP(h or 0), _VP(ux or 0), _VP(uy or 0),
                                _VP(stream)), _VP(handle))


def tf_lbm_pressure_force(handle: int, p: int | None, fx: int | None, fy: int | None,
                          stream: int = 0) -> None:
    _check(lib().tf_lbm_pressure_force(_VP(handle), _VP(p or 0), _VP(fx or 0), _VP(fy or 0),
                                       _VP(stream)), _VP(handle))


def tf_lbm_mass(handle: int, stream: int = 0) -> float:
    m = ctypes.c_double()
    _check(lib().tf_lbm_mass(_VP(handle), ctypes.byref(m), _VP(stream)), _VP(handle))
    return m.value


def tf_lbm_check(handle: int, stream: int = 0) -> int:
    s = ctypes.c_int32()
    _check(lib().tf_lbm_check(_VP(handle), ctypes.byref(s), _VP(stream)), _VP(handle))
    return s.value


def tf_lbm_get_state(handle: int, f: int, stream: int = 0) -> None:
    _check(lib().tf_lbm_get_state(_VP(handle), _VP(f), _VP(stream)), _VP(handle))


def tf_lbm_set_state(handle: int, f: int, stream: int = 0) -> None:
    _check(lib().tf_lbm_set_state(_VP(handle), _VP(f), _VP(stream)), _VP(handle))


def tf_lbm_time(handle: int) -> int:
    return int(lib().tf_lbm_time(_VP(handle)))


def tf_lbm_get_launch(handle: int) -> Launch:
    out = Launch()
    _check(lib().tf_lbm_get_launch(_VP(handle), ctypes.byref(out)), _VP(handle))
    return out


def tf_lbm_set_launch(handle: int, block_x: int, rows: int, graph_chunk: int,
                      pipeline: int = 0) -> None:
    L = Launch(block_x, rows, graph_chunk, pipeline)
    _check(lib().tf_lbm_set_launch(_VP(handle), ctypes.byref(L)), _VP(handle))


def tf_lbm_set_wait_limit(handle: int, polls: int) -> None:
    _check(lib().tf_lbm_set_wait_limit(_VP(handle), int(polls)), _VP(handle))


def tf_lbm_destroy(handle: int) -> None:
    lib().tf_lbm_destroy(_VP(handle))


def tf_lbm_last_error(handle: int | None = None) -> str:
    return lib().tf_lbm_last_error(_VP(handle or 0)).decode(errors="replace")


def tf_lbm_version() -> int:
    return int(lib().tf_lbm_version())


def tf_lbm_sum_noalloc(x: int, n: int, out: int, stream: int = 0) -> None:
    """Compensated sum of n device doubles at x into the device double at out,
    allocating nothing (for callers that may not allocate device memory)."""
    _check(lib().tf_lbm_sum_noalloc(_VP(x), int(n), _VP(out), _VP(stream)), None)


def tf_lbm_adjoint_step(handle: int, f_t: int, a_next: int, a_t: int, grad_kappa: int,
                        stream: int = 0) -> None:
    _check(lib().tf_lbm_adjoint_step(_VP(handle), _VP(f_t), _VP(a_next), _VP(a_t),
                                     _VP(grad_kappa), _VP(stream)), _VP(handle))


def tf_lbm_tape_create(handle: int, h0: int, theta: int | None, nsteps: int, every: int = 0) -> int:
    t = _VP()
    _check(lib().tf_lbm_tape_create(_VP(handle), _VP(h0), _VP(theta or 0), int(nsteps), int(every),
                                    ctypes.byref(t)), _VP(handle))
    return t.value


def tf_lbm_tape_forward(handle: int, tape: int, stream: int = 0) -> None:
    _check(lib().tf_lbm_tape_forward(_VP(tape), _VP(stream)), _VP(handle))


def tf_lbm_tape_backward(handle: int, tape: int, grad_h: int, grad_theta: int | None,
                         grad_h0: int | None, stream: int = 0) -> None:
    _check(lib().tf_lbm_tape_backward(_VP(tape), _VP(grad_h), _VP(grad_theta or 0),
                                      _VP(grad_h0 or 0), _VP(stream)), _VP(handle))


def tf_lbm_tape_destroy(tape: int) -> None:
    lib().tf_lbm_tape_destroy(_VP(tape))


def tf_lbm_tune(handle: int, trial_steps: int = 16, stream: int = 0) -> Launch:
    out = Launch()
    _check(lib().tf_lbm_tune(_VP(handle), int(trial_steps), ctypes.byref(out), _VP(stream)), _VP(handle))
    return out


def tf_lbm_diagnostics(handle: int, h_wet: float, mode_x: int, mode_y: int, out: int,
                       stream: int = 0) -> None:
    _check(lib().tf_lbm_diagnostics(_VP(handle), float(h_wet), int(mode_x), int(mode_y), _VP(out),
                                    _VP(stream)), _VP(handle))


def tf_lbm_term_norms(handle: int, out: int, stream: int = 0) -> None:
    _check(lib().tf_lbm_term_norms(_VP(handle), _VP(out), _VP(stream)), _VP(handle))


def _bcheck(rc: int, batch=None):
    if rc != TF_LBM_OK:
        msg = lib().tf_lbm_batch_last_error(batch).decode(errors="replace")
        raise TfLbmError(rc, msg)


def tf_lbm_batch_create(handles, stream: int = 0) -> int:
    arr = (_VP * len(handles))(*[_VP(h) for h in handles])
    b = _VP()
    _bcheck(lib().tf_lbm_batch_create(ctypes.byref(b), arr, len(handles), _VP(stream)), None)
    return b.value


def tf_lbm_batch_step(batch: int, nsteps: int, stream: int = 0) -> None:
    _bcheck(lib().tf_lbm_batch_step(_VP(batch), int(nsteps), _VP(stream)), _VP(batch))


def tf_lbm_batch_get_launch(batch: int) -> BatchLaunch:
    out = BatchLaunch()
    _bcheck(lib().tf_lbm_batch_get_launch(_VP(batch), ctypes.byref(out)), _VP(batch))
    return out


def tf_lbm_batch_set_launch(batch: int, block_x: int, rows: int, graph_chunk: int, queue: int = 0,
                            pipeline: int = 1) -> None:
    L = BatchLaunch(block_x, rows, graph_chunk, queue, pipeline)
    _bcheck(lib().tf_lbm_batch_set_launch(_VP(batch), ctypes.byref(L)), _VP(batch))


def tf_lbm_batch_tune(batch: int, trial_steps: int = 16, stream: int = 0) -> BatchLaunch:
    out = BatchLaunch()
    _bcheck(lib().tf_lbm_batch_tune(_VP(batch), int(trial_steps), ctypes.byref(out), _VP(stream)),
            _VP(batch))
    return out


def tf_lbm_batch_diagnostics(batch: int, h_wet: float, mode_x: int, mode_y: int, out: int,
                             stream: int = 0) -> None:
    _bcheck(lib().tf_lbm_batch_diagnostics(_VP(batch), float(h_wet), int(mode_x), int(mode_y), _VP(out),
                                           _VP(stream)), _VP(batch))


def tf_lbm_batch_items(batch: int) -> int:
    return int(lib().tf_lbm_batch_items(_VP(batch)))


def tf_lbm_batch_destroy(batch: int) -> None:
    lib().tf_lbm_batch_destroy(_VP(batch))


def tf_lbm_batch_last_error(batch: int | None = None) -> str:
    return lib().tf_lbm_batch_last_error(_VP(batch or 0)).decode(errors="replace")
