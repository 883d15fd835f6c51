"""Failure detection on the GPU without a fault: a bounded device wait that
runs out reports SF_ETIMEOUT through the status word, and the context stays
usable.

sf_selftest_wait_timeout launches one warp that waits, through the same
bounded mbarrier wait the TMA-staged CCZ4 kernel uses, on a barrier that
nothing ever completes.  The wait gives up after the given number of cycles;
nothing traps, faults or hangs.  Afterwards the TMA-staged kernel (whose own
waits use that code) runs one RK4 step and still matches the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1806_04182_gb300 import build, capi, inputs
from paper_1806_04182_gb300.state import PatchState

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    return capi.lib()


def test_wait_that_runs_out_reports_timeout_and_context_survives():
    capi.sf_get_device_status()  # clear
    capi.sf_selftest_wait_timeout(1_000_000)  # about half a millisecond
    assert capi.sf_get_device_status() == capi.SF_ETIMEOUT
    assert capi.sf_get_device_status() == capi.SF_OK  # cleared by the read

    # the TMA-staged kernel (padded float layout) still runs and is right
    n = (32, 96, 5)
    U0, dx = inputs.z4_perturbed(n, seed=4, amp=0.05)
    prm = capi.params()
    dt = 0.25 * min(dx)
    st = PatchState(capi.SF_Z4, n, dx, dt, precision=capi.SF_FP32_BULK_DW, prm=prm, x_pitch=104)
    st.upload(U0)
    st.step(1)
    got = st.fields().cpu().numpy().astype(np.float64)
    assert capi.sf_get_device_status() == capi.SF_OK
    G = oracle.ghosted(U0.copy())
    oracle.rk4_step(oracle.Z4, G, dx, dt, oracle.params())
    want = oracle.interior(G)
    eps32 = float(np.finfo(np.float32).eps)
    bound = 4 * 64 / 12 * eps32 * dt / min(dx) ** 2 / 1e-2
    for f in range(want.shape[0]):
        e = np.abs(got[f] - want[f]).max() / max(np.abs(want[f]).max(), 1e-2)
        assert e < bound, (f, e, bound)
