"""Pins of the oracle's counter-based draws: Philox4x64-10 against NumPy's
independent implementation of the same published generator, and
Box-Muller against the normal distribution."""
import numpy as np
import pytest

from oracle import rng


@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)),
                                     ((1, 2, 3, 4), (5, 6)),
                                     ((2**64 - 2, 7, 2**63, 1), (2**64 - 1, 12345)),
                                     ((65535, 40, 0, 0), (2, 0x52))])
def test_philox_matches_numpy(ctr, key):
    # numpy.random.Philox is Philox4x64-10; it increments its 256-bit
    # counter before producing each block of four words.
    c = ctr[0] + (ctr[1] << 64) + (ctr[2] << 128) + (ctr[3] << 192)
    k = key[0] + (key[1] << 64)
    g = np.random.Philox(key=k, counter=(c - 1) % (1 << 256))
    want = [int(x) for x in g.random_raw(4)]
    assert list(rng.philox4x64(ctr, key)) == want


def test_mulhi_range():
    for m in (1, 2, 3, 128, 65536, 2**40 + 7):
        assert rng.mulhi64(0, m) == 0
        assert rng.mulhi64(2**64 - 1, m) == m - 1


def test_box_muller_normal():
    import scipy.stats as st
    z = rng.gaussian_block(2000, 16, seed=9).ravel()
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1) < 0.03
    assert st.kstest(z, "norm").pvalue > 1e-3


def test_block_columns_are_counter_addressed():
    full = rng.gaussian_block(40, 12, seed=4)
    part = rng.gaussian_block(40, 8, seed=4, col0=4)
    assert np.array_equal(full[:, 4:12], part)
    assert not np.array_equal(full, rng.gaussian_block(40, 12, seed=5))
