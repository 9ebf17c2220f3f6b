"""Pins for the oracle's counter-based generators (published known answers)."""
import numpy as np

import oracle as O


def test_splitmix64_known_answers():
    # SplitMix64 stream from state 0 (Steele, Lea, Flood 2014; Vigna's reference
    # code): outputs are mix(0 + k*golden) for k = 1, 2, 3.
    g = 0x9E3779B97F4A7C15
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF
    assert O.splitmix64(g) == 0x6E789E6AA1B965F4
    assert O.splitmix64((2 * g) % 2**64) == 0x06C45D188009454F


def test_philox4x64_10_known_answer():
    # Random123 known-answer vector for philox4x64_10, counter 0, key 0.
    out = O.philox4x64_10([0, 0, 0, 0], [0, 0])
    assert [int(x) for x in out] == [0x16554D9ECA36314C, 0xDB20FE9D672D0FDC,
                                     0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]


def test_philox4x64_10_matches_numpy():
    # numpy.random.Philox is an independent Philox4x64-10; its first block is
    # produced after incrementing the counter.
    for key in (0, 7, 2**63 + 5):
        bg = np.random.Philox(key=np.array([key, 0], dtype=np.uint64),
                              counter=np.zeros(4, dtype=np.uint64))
        raw = bg.random_raw(12)
        mine = np.concatenate([O.philox4x64_10([c, 0, 0, 0], [key, 0]) for c in (1, 2, 3)])
        assert np.array_equal(raw, mine)


def test_uniform_pm1_exact_grid_and_range():
    u = O.uniform_pm1(99, 100_000)
    assert u.min() >= -1.0 and u.max() < 1.0
    k = (u + 1.0) * 2.0**52           # exact: 53-bit integers
    assert np.all(k == np.floor(k)) and np.all(k < 2.0**53)
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01
    # element i comes from word i%4 of block i//4
    w = O.philox4x64_10([1, 0, 0, 0], [99, 0])
    assert u[5] == (int(w[1]) >> 11) * 2.0**-52 - 1.0
