"""state.HostPipeline: RK steps of states held in host memory, with the
copies of neighbouring steps overlapping the stages.  Every step must give
exactly (bit for bit) what one PatchState.step gives from the same uploaded
state: the same kernels run on the same inputs, only the streams differ."""
import numpy as np
import pytest
import torch

from paper_1806_04182_gb300 import build, capi, inputs
from paper_1806_04182_gb300.state import HostPipeline, PatchState

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    return capi.lib()


@pytest.mark.parametrize("system,precision,pitch", [
    (capi.SF_Z4, capi.SF_FP32_BULK_DW, 24),   # 16-byte rows: the TMA-staged kernel
    (capi.SF_Z4, capi.SF_FP64, None),
    (capi.SF_WAVE, capi.SF_FP32_BULK, None),
])
def test_host_pipeline_equals_device_steps(system, precision, pitch):
    n = (17, 13, 9)
    data = (lambda q: inputs.z4_perturbed(n, seed=q, amp=0.04)) if system == capi.SF_Z4 else \
        (lambda q: inputs.wave_plane(n, seed=q))
    U = [data(q)[0] for q in range(5)]
    dx = data(0)[1]
    dt = 0.25 * min(dx)
    kw = dict(precision=precision, x_pitch=pitch)
    # reference: each input uploaded into a device state and stepped once
    ref = []
    st = PatchState(system, n, dx, dt, **kw)
    hosts_in = []
    for u in U:
        st.upload(u)
        hosts_in.append(st.A.cpu().pin_memory())
        st.step(1)
        ref.append(st.A.cpu())
    torch.cuda.synchronize()
    pipe = HostPipeline(system, n, dx, dt, **kw)
    outs = [torch.empty_like(h).pin_memory() for h in hosts_in]
    for h_in, h_out in zip(hosts_in, outs):
        pipe.step(h_in, h_out)
    pipe.synchronize()
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)
