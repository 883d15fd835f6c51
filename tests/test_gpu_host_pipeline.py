"""state.HostPipeline (the C-ABI call sf_step_host): RK steps of states held
in host memory, with the copies of neighbouring steps overlapping the
stages.  Every step must give exactly (bit for bit) what one PatchState.step
gives from the same uploaded state, and an evolution kept in host memory
what the same steps give on the device: the same kernels run on the same
inputs, only the streams differ."""
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


CASES = [
    (capi.SF_Z4, capi.SF_FP32_BULK_DW, 24, 0),   # 16-byte rows: the TMA-staged kernel
    (capi.SF_Z4, capi.SF_FP64, None, 0),
    (capi.SF_WAVE, capi.SF_FP32_BULK, None, 0),
]


def data_fn(system, n):
    if system == capi.SF_Z4:
        return lambda q: inputs.z4_perturbed(n, seed=q, amp=0.04)
    return lambda q: inputs.wave_plane(n, seed=q)


@pytest.mark.parametrize("system,precision,pitch,xo", CASES)
def test_host_pipeline_equals_device_steps(system, precision, pitch, xo):
    n = (17, 13, 9)
    data = data_fn(system, n)
    U = [data(q)[0] for q in range(5)]
    dx = data(0)[1]
    dt = 0.25 * min(dx)
    kw = dict(precision=precision, x_pitch=pitch, x_offset=xo)
    pipe = HostPipeline(system, n, dx, dt, **kw)
    # reference: each input uploaded into a device state and stepped once
    ref = []
    st = PatchState(system, n, dx, dt, **kw)
    hosts_in = []
    for u in U:
        st.upload(u)
        hosts_in.append(pipe.image(st.A).cpu().pin_memory())
        st.step(1)
        ref.append(pipe.image(st.A).cpu())
    torch.cuda.synchronize()
    outs = [torch.empty_like(h).pin_memory() for h in hosts_in]
    pipe.run(hosts_in, outs)
    pipe.synchronize()
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)


@pytest.mark.parametrize("system,precision,pitch,xo", CASES + [(capi.SF_Z4, capi.SF_FP32_BULK_DW, 104, 1)])
def test_host_evolution_equals_device_evolution(system, precision, pitch, xo):
    # one slot, the compensation carried over: ten steps fed back through one
    # pinned buffer equal ten device-resident steps bit for bit
    n = (32, 96, 3) if pitch == 104 else (17, 13, 9)
    U0, dx = data_fn(system, n)(0)
    dt = 0.25 * min(dx)
    kw = dict(precision=precision, x_pitch=pitch, x_offset=xo)
    st = PatchState(system, n, dx, dt, **kw)
    st.upload(U0)
    pipe = HostPipeline(system, n, dx, dt, slots=1, **kw)
    pipe.states[0].upload(U0)  # zero compensation, as st's
    h = pipe.image(st.A).cpu().pin_memory()
    st.step(10)
    pipe.run([h] * 10, [h] * 10, reset_kahan=False)
    pipe.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(h, pipe.image(st.A).cpu())
