"""FP32-bulk CCZ4 against FP64 over 100 RK4 steps (the precision claim of the
FP32-bulk path), on the 96^3 workload: Minkowski + 1e-10 uniform noise, and
the A = 0.01 gauge wave.  The FP64 GPU path is the reference here (it matches
the oracle to 1e-12 per substep, tests/test_gpu_parity.py).

The per-field error is max |U32 - U64| over the grid divided by the field's
deviation scale max |U64 - U_flat| (U_flat = 1 for chi, gt_ii, alpha; 0
otherwise), floored at 1e-12 (noise data) or 1e-3 (gauge wave).  Bounds: the
noise data live at 1e-10 with float storage of their deviations (relative
precision 6e-8); 100 steps x 4 stages of rounding that grows through the
1/dx^2 stencils keep the relative error of every field below 1e-3.  The table
is printed (pytest -s).
"""
import numpy as np
import pytest
import torch

from paper_1806_04182_gb300 import build, capi, inputs
from paper_1806_04182_gb300.state import PatchState

pytestmark = pytest.mark.gpu
FLAT = (0, 1, 4, 6, 18)


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    build.build()
    return capi.lib()


def evolve(U0, dx, precision, steps, prm):
    n = (U0.shape[3], U0.shape[2], U0.shape[1])
    st = PatchState(capi.SF_Z4, n, dx, 0.25 * dx[0], precision=precision, prm=prm)
    st.upload(U0)
    st.step(steps)
    return st.fields().cpu().numpy()


def per_field_error(a, ref, floor):
    bg = np.zeros(25)
    bg[list(FLAT)] = 1.0
    errs = []
    for f in range(25):
        scale = max(np.abs(ref[f] - bg[f]).max(), floor)
        errs.append(np.abs(a[f] - ref[f]).max() / scale)
    return np.array(errs)


@pytest.mark.parametrize("precision", [capi.SF_FP32_BULK_DW, capi.SF_FP32_BULK])
def test_fp32_bulk_noise_100_steps(precision):
    n = (96, 96, 96)
    U0, dx = inputs.z4_minkowski_noise(n, seed=0, amp=1e-10)
    prm = capi.params()
    ref = evolve(U0, dx, capi.SF_FP64, 100, prm)
    got = evolve(U0, dx, precision, 100, prm)
    e = per_field_error(got, ref, 1e-12)
    print("\nnoise 96^3, 100 steps, precision", precision, ":",
          " ".join(f"{inputs.Z4_NAMES[f]}={e[f]:.2e}" for f in range(25)))
    assert np.all(np.isfinite(got))
    assert e.max() < 1e-3, e


def test_fp32_bulk_gauge_wave_100_steps():
    n = (96, 96, 96)
    U0, dx = inputs.z4_gauge_wave(n, amp=0.01)
    prm = capi.params(slicing=1, shift_frozen=1)
    ref = evolve(U0, dx, capi.SF_FP64, 100, prm)
    got = evolve(U0, dx, capi.SF_FP32_BULK_DW, 100, prm)
    e = per_field_error(got, ref, 1e-3)
    print("\ngauge wave 96^3, 100 steps:",
          " ".join(f"{inputs.Z4_NAMES[f]}={e[f]:.2e}" for f in range(25)))
    assert e.max() < 1e-3, e
