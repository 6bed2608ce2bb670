"""The synthetic inputs have the shapes and structure the workloads state:
seeded (same seed, same bits), mixture labels by component parity or one
class against the rest, image-like rows with about 80 % exact zeros and
values in [0, 1], and 16-bit-exact Gaussian blocks."""
import numpy as np

import synth


def test_mixture_shapes_labels_and_seed():
    X, y, Xt, yt, c, ct = synth.mixture(500, 8, 4, 0.7, 11, 50)
    assert X.shape == (500, 8) and Xt.shape == (50, 8)
    assert np.array_equal(y, np.where(c % 2 == 0, 1.0, -1.0))
    assert np.array_equal(yt, np.where(ct % 2 == 0, 1.0, -1.0))
    assert set(np.unique(c)) <= set(range(4))
    X2 = synth.mixture(500, 8, 4, 0.7, 11, 50)[0]
    assert np.array_equal(X, X2)
    assert not np.array_equal(X, synth.mixture(500, 8, 4, 0.7, 12, 50)[0])
    lab = synth.labels_one_vs_rest(c, 2)
    assert np.array_equal(lab == 1.0, c == 2)


def test_image_like_structure():
    X, y, Xt, yt = synth.image_like(200, 3, m_test=20)
    assert X.shape == (200, 784) and Xt.shape == (20, 784)
    assert X.min() >= 0.0 and X.max() <= 1.0
    zero = np.mean(X == 0.0)
    assert 0.75 <= zero <= 0.85
    assert set(np.unique(y)) <= {-1.0, 1.0} and set(np.unique(yt)) <= {-1.0, 1.0}
    assert np.array_equal(X, synth.image_like(200, 3, m_test=20)[0])


def test_gaussian_block_is_fp16_exact():
    R = synth.gaussian_block(300, 17, 5)
    assert R.dtype == np.float16 and R.shape == (300, 17)
    R32 = R.astype(np.float32)
    assert np.array_equal(R32.astype(np.float16), R)
    assert abs(float(R32.mean())) < 0.1 and 0.9 < float(R32.std()) < 1.1
