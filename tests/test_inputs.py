"""The seeded input generators are deterministic and follow SplitMix64."""
import numpy as np

from paper_1806_04182_gb300 import inputs


def test_splitmix64_reference_sequence():
    # SplitMix64 from state 0: the published first three outputs
    got = [int(v) for v in inputs.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_are_reproducible_and_offsettable():
    a = inputs.uniform(5, 100)
    b = inputs.uniform(5, 60, offset=40)
    np.testing.assert_array_equal(a[40:], b)
    assert np.all((a >= 0) & (a < 1))
    assert not np.array_equal(a, inputs.uniform(6, 100))


def test_normal_moments():
    z = inputs.normal(3, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_workload_shapes():
    U, dx = inputs.mhd_blast((8, 6, 4), seed=1)
    assert U.shape == (8, 4, 6, 8) and dx == (1 / 8, 1 / 6, 1 / 4)
    U, dx = inputs.z4_minkowski_noise((5, 4, 3))
    assert U.shape == (25, 3, 4, 5)
    assert inputs.wave_k(0) == inputs.wave_k(0)
    assert all(k in (1, 2, 3) for k in inputs.wave_k(7))
    t = inputs.amr_patch_table(512, seed=0)
    assert len(t) == 512 and all(16 <= s <= 64 for p in t for s in p["n"])
    assert {p["system"] for p in t} == {"wave", "z4"}
