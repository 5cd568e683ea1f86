"""Pins for the oracle's random stream: Philox4x32-10 and the draws built on it."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers(orc):
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = orc.philox(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


def _curand_host():
    for name in ("libcurand.so", "libcurand.so.10",
                 "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator(orc):
    """cuRAND's CPU-side Philox4_32_10 generator is an independent implementation:
    with seed S its j-th block of four outputs is Philox(ctr=(0,0,j,0), key=S)."""
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161  # value from curand.h
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        rng = np.random.default_rng(5)
        for seed in [0, 1, 42, 0xFFFFFFFF, 1 << 32, 0xDEADBEEFCAFEF00D] + \
                [int(x) for x in rng.integers(0, 2**63, 4)]:
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(0)) == 0
            buf = np.zeros(4 * 64, dtype=np.uint32)
            assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_size_t(buf.size)) == 0
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for j in range(64):
                assert list(orc.philox([0, 0, j, 0], key)) == list(buf[4 * j:4 * j + 4]), (seed, j)
    finally:
        lib.curandDestroyGenerator(gen)


def test_root_uniform_chi_square(orc):
    """Roots (r*n)>>32 are uniform over V: chi-square over 40k samples, n = 37."""
    n, S = 37, 40000
    counts = np.bincount([orc.root(42, s, n) for s in range(S)], minlength=n)
    exp = S / n
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    # 36 degrees of freedom: P(chi2 > 80) < 1e-4
    assert chi2 < 80.0, chi2
    assert counts.min() > 0


def test_coins_uniform_and_distinct_lanes(orc):
    """IC coins of the four edges sharing a counter come from distinct lanes."""
    seed = 7
    vals = [orc.ic_coin(seed, 3, e) for e in range(4)]
    out = orc.philox([3, 0, 0, 2], [seed, 0])
    assert vals == [int(x) for x in out]
    # next block of four edges uses the next counter word
    assert orc.ic_coin(seed, 3, 4) == int(orc.philox([3, 1, 0, 2], [seed, 0])[0])
    # edge ids above 2^34 reach the third counter word
    e = (1 << 34) + 5
    assert orc.ic_coin(seed, 3, e) == int(orc.philox([3, 1, 1, 2], [seed, 0])[1])
    coins = np.array([orc.ic_coin(seed, s, e) for s in range(200) for e in range(50)],
                     dtype=np.float64) / 2**32
    assert abs(coins.mean() - 0.5) < 0.01


def test_partition_balance_and_determinism(orc):
    n, P = 200000, 148
    part = orc.partition(n, P, 42)
    assert part.min() >= 0 and part.max() < P
    assert np.array_equal(part, orc.partition(n, P, 42))
    assert not np.array_equal(part, orc.partition(n, P, 43))
    counts = np.bincount(part, minlength=P)
    exp = n / P
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 147 + 6 * np.sqrt(2 * 147), chi2
