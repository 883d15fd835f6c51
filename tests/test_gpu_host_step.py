"""sf_step_host: RK steps of states held in host memory, through the C ABI.

* An evolution kept in host memory (every step's input is the previous
  step's output, one pinned buffer updated in place) equals, bit for bit, the
  same steps run on a device-resident state: FP64 with one and two device
  slots; FP32-bulk with one slot (the Kahan compensation carries over) and
  with two or three slots and SF_HOST_RESET_KAHAN (against a device run that
  zeroes the compensation before every step).
* Independent steps from one input (two or three slots, copies overlapping
  the stages) each equal one device step from that input.
"""
import pytest
import torch

from paper_1806_04182_gb300 import build, capi, inputs
from paper_1806_04182_gb300.state import PatchState

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    return capi.lib()


CASES = [
    # system, n, precision, pitch, row offset
    (capi.SF_WAVE, (19, 7, 6), capi.SF_FP64, None, 0),
    (capi.SF_Z4, (12, 9, 7), capi.SF_FP64, None, 0),
    (capi.SF_Z4, (32, 96, 3), capi.SF_FP32_BULK_DW, 104, 1),
    (capi.SF_Z4, (37, 13, 5), capi.SF_FP32_BULK, 44, 0),
]


def make(system, n, precision, pitch, xo, seed=0):
    if system == capi.SF_Z4:
        U0, dx = inputs.z4_perturbed(n, seed=seed, amp=0.04)
    else:
        U0, dx = inputs.wave_plane(n, seed=seed)
    st = PatchState(system, n, dx, 0.25 * min(dx), precision=precision, x_pitch=pitch, x_offset=xo)
    st.upload(U0)
    return st


def slot_of(st):
    return capi.sf_state(u=st.ptr(st.A), s1=st.ptr(st.B), s2=st.ptr(st.C),
                         acc=st.ptr(st.D) if st.D is not None else None,
                         kahan=st.ptr(st.E) if st.E is not None else None)


def image(st, arr):
    """The state's host image: sf_state_span elements from ghosted (0,0,0)."""
    span = capi.sf_state_span(st.patch(arr, arr, arr))
    return arr.reshape(-1)[st.xo:st.xo + span]


def pinned_copy(t):
    h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
    h.copy_(t)
    return h


@pytest.mark.parametrize("system,n,precision,pitch,xo", CASES)
@pytest.mark.parametrize("nslots", [1, 2, 3])
def test_chained_host_evolution_equals_device_run(system, n, precision, pitch, xo, nslots):
    steps = 6
    ref = make(system, n, precision, pitch, xo)
    work = [make(system, n, precision, pitch, xo) for _ in range(nslots)]
    h = pinned_copy(image(ref, ref.A))
    reset = precision != capi.SF_FP64 and nslots > 1
    for _ in range(steps):
        if reset:
            ref.E.zero_()
        ref.step(1)
    cs = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    up.wait_stream(cs)
    down.wait_stream(cs)
    capi.sf_step_host(ref.prm, ref.patch(ref.A, ref.A, ref.B), [slot_of(w) for w in work],
                      [h.data_ptr()] * steps, [h.data_ptr()] * steps,
                      flags=capi.SF_HOST_RESET_KAHAN if reset else 0,
                      compute_stream=cs.cuda_stream, h2d_stream=up.cuda_stream,
                      d2h_stream=down.cuda_stream)
    down.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(h, image(ref, ref.A).cpu())


@pytest.mark.parametrize("system,n,precision,pitch,xo", CASES)
@pytest.mark.parametrize("nslots", [2, 3])
def test_independent_host_steps_equal_one_device_step(system, n, precision, pitch, xo, nslots):
    steps = 5
    ref = make(system, n, precision, pitch, xo, seed=3)
    h_in = pinned_copy(image(ref, ref.A))
    outs = [torch.empty_like(h_in).pin_memory() for _ in range(steps)]
    if ref.E is not None:
        ref.E.zero_()
    ref.step(1)
    want = image(ref, ref.A).cpu()
    work = [make(system, n, precision, pitch, xo) for _ in range(nslots)]
    cs = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    up.wait_stream(cs)
    down.wait_stream(cs)
    capi.sf_step_host(ref.prm, ref.patch(ref.A, ref.A, ref.B), [slot_of(w) for w in work],
                      [h_in.data_ptr()] * steps, [o.data_ptr() for o in outs],
                      flags=capi.SF_HOST_RESET_KAHAN if precision != capi.SF_FP64 else 0,
                      compute_stream=cs.cuda_stream, h2d_stream=up.cuda_stream,
                      d2h_stream=down.cuda_stream)
    down.synchronize()
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, want)


# ------------------------------------------------------------------ interior host images
def interior_image(st, arr):
    return st.interior(arr).contiguous().reshape(-1)


@pytest.mark.parametrize("system,n,precision,pitch,xo", CASES)
@pytest.mark.parametrize("nslots", [1, 3])
def test_interior_images_chained_evolution_equals_device_run(system, n, precision, pitch, xo, nslots):
    # host images without ghost shell or padding: the upload is spread into
    # the patch layout with its periodic ghost shell on the device, the new
    # interior gathered back; the evolution kept in host memory equals the
    # device run bit for bit
    steps = 4
    ref = make(system, n, precision, pitch, xo)
    work = [make(system, n, precision, pitch, xo) for _ in range(nslots)]
    assert capi.sf_interior_span(ref.patch(ref.A, ref.A, ref.A)) == ref.nf * n[0] * n[1] * n[2]
    h = pinned_copy(interior_image(ref, ref.A))
    reset = precision != capi.SF_FP64 and nslots > 1
    for _ in range(steps):
        if reset:
            ref.E.zero_()
        ref.step(1)
    cs = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    up.wait_stream(cs)
    down.wait_stream(cs)
    flags = capi.SF_HOST_INTERIOR | (capi.SF_HOST_RESET_KAHAN if reset else 0)
    capi.sf_step_host(ref.prm, ref.patch(ref.A, ref.A, ref.B), [slot_of(w) for w in work],
                      [h.data_ptr()] * steps, [h.data_ptr()] * steps, flags=flags,
                      compute_stream=cs.cuda_stream, h2d_stream=up.cuda_stream,
                      d2h_stream=down.cuda_stream)
    down.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(h, interior_image(ref, ref.A).cpu())


def test_interior_images_need_periodic_ghosts():
    st = make(capi.SF_Z4, (12, 9, 7), capi.SF_FP64, None, 0)
    prm = capi.params(ghosts=capi.SF_GHOSTS_NONE)
    h = pinned_copy(interior_image(st, st.A))
    with pytest.raises(capi.SfError, match="periodic"):
        capi.sf_step_host(prm, st.patch(st.A, st.A, st.B), [slot_of(st)], [h.data_ptr()],
                          [h.data_ptr()], flags=capi.SF_HOST_INTERIOR)
