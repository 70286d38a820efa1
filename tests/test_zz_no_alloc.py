"""The allocation-free sum entry point, through the C ABI, against the
library's regular mass reduction.

tf_lbm_sum_noalloc exists for callers that cannot allocate device memory
(code inside an application that owns the device memory budget, loops that
cannot afford cudaMalloc's possible device-wide synchronisation).  Summing the
exported state must give the volume tf_lbm_mass reports, call after call,
although every call reuses the same fixed scratch array.  This file is
collected last so that a run stopping at its first failure has already run
every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1810_07642_gb300 import _lib as L
from paper_1810_07642_gb300 import inputs
from paper_1810_07642_gb300.film import ThinFilm

pytestmark = pytest.mark.gpu

TOL = 1e-11  # the FP64 parity tolerance of the GPU tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1810_07642_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _noalloc_sum(x: torch.Tensor) -> float:
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=x.device)
    L.tf_lbm_sum_noalloc(x.data_ptr(), x.numel(), out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    return float(out.item())


def test_noalloc_sum_matches_mass_on_two_calls_in_a_row():
    h0, th, p = inputs.patterned_dewetting(512, seed=3)
    sim = ThinFilm(p, h0, th)
    sim.step(20)
    first = _noalloc_sum(sim.get_state())
    m1 = sim.mass()
    # second call on a smaller array: it must not pick up the first call's
    # partial sums left in the shared scratch array
    small = ThinFilm(inputs._params(100, 37), np.full((37, 100), 0.5))
    second = _noalloc_sum(small.get_state())
    m2 = small.mass()
    assert abs(first - m1) <= TOL * abs(m1)
    assert abs(second - m2) <= TOL * abs(m2)
    assert abs(second - 0.5 * 100 * 37) <= TOL * 1850
    # and once more on the first state, after further steps
    sim.step(7)
    third = _noalloc_sum(sim.get_state())
    assert abs(third - sim.mass()) <= TOL * abs(third)


def test_noalloc_sum_limits_and_empty_input():
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.ones(8, dtype=torch.float64, device="cuda")
    with pytest.raises(L.TfLbmError) as e:
        L.tf_lbm_sum_noalloc(x.data_ptr(), L.TF_LBM_NOALLOC_MAX_ELEMS + 1, out.data_ptr(), 0)
    assert e.value.code == L.TF_LBM_ERR_ARG and "67108864" in str(e.value)
    with pytest.raises(L.TfLbmError):
        L.tf_lbm_sum_noalloc(x.data_ptr(), -1, out.data_ptr(), 0)
    out.fill_(7.0)
    L.tf_lbm_sum_noalloc(0, 0, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert out.item() == 0.0


def test_noalloc_sum_at_the_largest_accepted_size():
    """n = TF_LBM_NOALLOC_MAX_ELEMS exactly: every one of the 4096 blocks is
    full and the final kernel reduces the largest partial table.  A sum of
    ones is exact in double precision; a smaller call right after it must
    not see the large call's partials."""
    n = L.TF_LBM_NOALLOC_MAX_ELEMS
    x = torch.ones(n, dtype=torch.float64, device="cuda")  # 512 MB
    assert _noalloc_sum(x) == float(n)
    del x
    y = torch.full((1000,), 0.25, dtype=torch.float64, device="cuda")
    assert _noalloc_sum(y) == 250.0
