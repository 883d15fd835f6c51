"""The C-ABI library builds, loads, exports every symbol of include/sf.h and
rejects bad arguments synchronously (no GPU work is enqueued by any call here)."""
import ctypes
import os
import re

import pytest

from paper_1806_04182_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return capi.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(sf_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(names) == sorted(capi.EXPORTS)


def test_struct_layouts_match_header():
    # sizes follow from the C declaration order with natural alignment
    assert ctypes.sizeof(capi.sf_params) == 4 + 4 + 8 * 4 + 4 * 4 + 8 * 4 + 4 + 4
    assert ctypes.sizeof(capi.sf_patch) == 12 + 4 + 24 + 8 + 4 + 4 + 24 + 5 * 8 + 8


def test_nfields(L):
    assert [capi.sf_nfields(s) for s in (capi.SF_WAVE, capi.SF_MHD, capi.SF_Z4)] == [5, 8, 25]
    assert capi.sf_nfields(7) == -1


def fake_patch(**kw):
    p = capi.sf_patch()
    p.n[:] = kw.get("n", (8, 8, 8))
    p.ghost = kw.get("ghost", 3)
    p.dx[:] = (0.1, 0.1, 0.1)
    p.dt = 0.01
    p.system = kw.get("system", capi.SF_WAVE)
    p.precision = kw.get("precision", capi.SF_FP64)
    base = 1 << 20
    p.u_stage = kw.get("u_stage", base)
    p.u_n = kw.get("u_n", base)
    p.acc = kw.get("acc", base * 2)
    p.u_next = kw.get("u_next", base * 3)
    p.kahan = kw.get("kahan", base * 4)
    return p


@pytest.mark.parametrize("kw, msg", [
    (dict(ghost=2), "ghost"),
    (dict(n=(0, 8, 8)), "n[0]"),
    (dict(system=9), "system"),
    (dict(precision=5), "precision"),
    (dict(u_next=1 << 20), "alias"),
    (dict(acc=0), "acc"),
    (dict(u_stage=(1 << 20) + 4), "misaligned"),
])
def test_bad_arguments_rejected(L, kw, msg):
    with pytest.raises(capi.SfError) as e:
        capi.sf_substep(capi.params(), fake_patch(**kw), 0)
    assert e.value.status == capi.SF_EINVAL
    assert msg in str(e.value)


def test_bad_stage_and_rk(L):
    with pytest.raises(capi.SfError, match="stage"):
        capi.sf_substep(capi.params(), fake_patch(), 4)
    with pytest.raises(capi.SfError, match="stage"):
        capi.sf_substep(capi.params(rk=capi.SF_SSPRK3), fake_patch(), 3)
    with pytest.raises(capi.SfError, match="rk"):
        capi.sf_substep(capi.params(rk=7), fake_patch(), 0)


def test_kahan_required_for_fp32_bulk_rk4(L):
    with pytest.raises(capi.SfError, match="kahan"):
        capi.sf_substep(capi.params(), fake_patch(precision=capi.SF_FP32_BULK, kahan=0), 0)


def test_in_place_only_in_last_stage(L):
    base = 1 << 20
    with pytest.raises(capi.SfError, match="alias"):
        capi.sf_substep(capi.params(), fake_patch(u_stage=base * 5, u_n=base, u_next=base), 1)


def test_fused_periodic_ghosts_need_n_at_least_ghost(L):
    with pytest.raises(capi.SfError, match="ghost"):
        capi.sf_substep(capi.params(), fake_patch(n=(2, 8, 8)), 0)


def test_cfl_rate_only_for_mhd(L):
    p = fake_patch()
    p.cfl_rate = 1 << 24
    with pytest.raises(capi.SfError, match="cfl_rate"):
        capi.sf_substep(capi.params(), p, 0)


def test_adjoint_only_for_wave(L):
    with pytest.raises(capi.SfError) as e:
        capi.sf_adjoint_substep(capi.params(), fake_patch(system=capi.SF_Z4), 0)
    assert e.value.status == capi.SF_ENOTSUP


def test_mixed_systems_rejected_by_substep(L):
    with pytest.raises(capi.SfError, match="sf_batch"):
        capi.sf_substep(capi.params(), [fake_patch(), fake_patch(system=capi.SF_Z4)], 0)


def test_selftest_wait_limit_checked(L):
    # rejected on the host before any device work
    for bad in (0, -5, 2_000_000_001):
        with pytest.raises(capi.SfError) as e:
            capi.sf_selftest_wait_timeout(bad)
        assert e.value.status == capi.SF_EINVAL
        assert "limit_cycles" in str(e.value)


def test_batch_tuned_rejects_null_batch(L):
    with pytest.raises(capi.SfError, match="batch is NULL"):
        capi.sf_batch_tuned(None)


def test_batch_set_halo_rejects_null_batch(L):
    # rejected on the host: no batch, so nothing reaches the device
    with pytest.raises(capi.SfError) as e:
        capi.sf_batch_set_halo(None, 0, [])
    assert e.value.status == capi.SF_EINVAL
    assert "batch is NULL" in str(e.value)


def test_state_span_counts_the_ghosted_image(L):
    p = fake_patch(n=(8, 8, 8), system=capi.SF_WAVE)
    p.sy, p.sz, p.sf = 14, 14 * 14, 14 ** 3
    assert capi.sf_state_span(p) == 5 * 14 ** 3  # dense layout: the whole array
    p = fake_patch(n=(32, 96, 4), system=capi.SF_Z4, precision=capi.SF_FP32_BULK_DW)
    p.sy, p.sz, p.sf = 104, 104 * 102, 104 * 102 * 10
    assert capi.sf_state_span(p) == 24 * p.sf + 9 * p.sz + 101 * p.sy + 38
    p.system = 9
    assert capi.sf_state_span(p) == -1


def test_step_host_rejects_bad_arguments(L):
    p = fake_patch(n=(8, 8, 8), system=capi.SF_WAVE)
    p.sy, p.sz, p.sf = 14, 14 * 14, 14 ** 3
    base = 1 << 20
    slot = capi.sf_state(u=base, s1=2 * base, s2=3 * base, acc=4 * base, kahan=None)
    prm = capi.params()
    with pytest.raises(capi.SfError, match="nslots"):
        capi.sf_step_host(prm, p, [slot] * 5, [base], [base])
    with pytest.raises(capi.SfError, match="flags"):
        capi.sf_step_host(prm, p, [slot], [base], [base], flags=4)
    with pytest.raises(capi.SfError, match="SF_HOST_RESET_KAHAN"):
        capi.sf_step_host(prm, p, [slot], [base], [base], flags=capi.SF_HOST_RESET_KAHAN)
    bad = capi.sf_state(u=base, s1=base, s2=3 * base, acc=4 * base, kahan=None)
    with pytest.raises(capi.SfError, match="u_next"):
        capi.sf_step_host(prm, p, [bad], [base], [base])
    with pytest.raises(capi.SfError, match="NULL"):
        capi.sf_step_host(prm, p, [slot], [0], [base])
