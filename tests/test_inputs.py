"""The seeded input generators: splitmix64 against its published first
outputs, and the shapes/ranges of each workload's initial field."""
import numpy as np

import lbm_inputs as I


def test_splitmix64_reference_outputs():
    # splitmix64 seeded with 0 yields 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
    # 0x06C45D188009454F: the state advances by the golden gamma per draw.
    gamma = np.uint64(0x9E3779B97F4A7C15)
    keys = np.array([0, gamma, (2 * int(gamma)) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    out = I.splitmix64(keys)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_spinodal_field_range_and_determinism():
    a = I.spinodal_density(64, 48, rho0=0.25, amp=0.01, seed=14127228)
    b = I.spinodal_density(64, 48, rho0=0.25, amp=0.01, seed=14127228)
    assert a.shape == (48, 64) and np.array_equal(a, b)
    assert a.min() >= 0.25 * 0.99 and a.max() < 0.25 * 1.01
    assert abs(a.mean() / 0.25 - 1) < 1e-3


def test_droplet_and_slab_profiles():
    d = I.droplet_density(64, 64, 15, 0.36, 0.01)
    assert abs(d[32, 32] - 0.36) < 1e-9 and abs(d[0, 0] - 0.01) < 1e-9
    assert np.array_equal(d, d.T)
    s = I.slab_density(100, 4, 5.8, 1.47)
    assert abs(s[0, 50] - 5.8) < 1e-6 and abs(s[0, 0] - 1.47) < 1e-6


def test_sweep_instances_ranges():
    inst = I.sweep_instances(64, seed=7228)
    assert len(inst) == 64
    assert {i.L for i in inst} <= {128, 256, 512, 1024}
    assert all(0.6 <= i.T_over_Tc <= 0.85 and 0 <= i.kappa <= 0.6 for i in inst)
    assert all(abs(i.radius - 0.2 * i.L) < 1e-12 for i in inst)
