"""The seeded input generators (shared by the oracle and the GPU tests, no
method arithmetic): the mixer is SplitMix64's, pinned to the generator's
published first outputs for seed 0, and the counter-based streams are
consistent under offsets and chunking."""
import numpy as np

from paper_2305_05988_gb300 import inputs


def test_mixer_matches_splitmix64_reference_outputs():
    # SplitMix64 seeded with 0: state advances by the golden gamma, output = mix(state)
    expected = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    with np.errstate(over="ignore"):
        got = [int(inputs._mix64(np.uint64(inputs.GAMMA) * np.uint64(k))) for k in range(1, 5)]
    assert got == expected


def test_streams_are_counter_based():
    a = inputs.raw_u64(7, 3, 1000)
    assert np.array_equal(inputs.raw_u64(7, 3, 400, offset=600), a[600:])
    assert not np.array_equal(inputs.raw_u64(7, 4, 1000), a)
    assert not np.array_equal(inputs.raw_u64(8, 3, 1000), a)
    u = inputs.uniform(7, 3, 5000, chunk=777)
    assert np.array_equal(u, inputs.uniform(7, 3, 5000))
    assert u.min() >= 0.0 and u.max() < 1.0
    # 53-bit values: exactly representable multiples of 2^-53
    assert np.array_equal(np.ldexp(u, 53), np.floor(np.ldexp(u, 53)))


def test_uniform_moments():
    u = inputs.uniform(0, 1, 1 << 20)
    assert abs(u.mean() - 0.5) < 2e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    v = inputs.uniform_pm1(0, 1, 1 << 16)
    assert v.min() >= -1.0 and v.max() < 1.0
