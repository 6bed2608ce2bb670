"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs.  It holds none of the method's arithmetic:
no kernel evaluation, no clustering, no compression, no solve.  Both the
CPU oracle and the CUDA path consume what it returns, so the same seed
gives both sides the same bits.

Workload shapes (the real UCI / MNIST8M sets of the paper's Section 5 are
not available, so these stand in for them):

* ``mixture``: isotropic Gaussian mixture, means uniform in [-2, 2]^d,
  common standard deviation ``sigma``, equal weights; label +1 for an even
  component index, -1 for an odd one.  With d=8 this is SUSY-shaped (the
  paper's SUSY has d=8, h=1, lambda=4 in its Table 2), with d=54 it is
  COVTYPE-shaped.
* ``image_like``: 28x28 vectors (d=784), about 80 % exact zeros, non-zeros
  in spatially correlated blobs with values in [0, 1]; 10 class prototypes
  plus noise, MNIST-shaped.
* ``gaussian_block``: an n x r block of N(0,1) values rounded to a 16-bit
  float, used as a fixed right-hand side for the sampling product.
"""
from __future__ import annotations

import numpy as np

__all__ = ["mixture", "image_like", "gaussian_block", "labels_pm1", "labels_one_vs_rest"]


def labels_pm1(component: np.ndarray) -> np.ndarray:
    """+1 for even component index, -1 for odd."""
    return np.where(component % 2 == 0, 1.0, -1.0)


def labels_one_vs_rest(component: np.ndarray, cls: int) -> np.ndarray:
    """+1 for component ``cls``, -1 otherwise (one-vs-all labels)."""
    return np.where(component == cls, 1.0, -1.0)


def mixture(n: int, d: int, n_comp: int, sigma: float, seed: int,
            m_test: int = 0):
    """Gaussian-mixture train/test draw.

    Returns ``(X, y, Xt, yt, comp, comp_t)``; X is n x d float64, y is +-1.
    Train and test points come from one stream so the test set is a fresh
    draw from the same mixture.
    """
    rng = np.random.default_rng(seed)
    means = rng.uniform(-2.0, 2.0, size=(n_comp, d))
    comp = rng.integers(0, n_comp, size=n)
    X = means[comp] + sigma * rng.standard_normal((n, d))
    comp_t = rng.integers(0, n_comp, size=m_test)
    Xt = means[comp_t] + sigma * rng.standard_normal((m_test, d))
    return X, labels_pm1(comp), Xt, labels_pm1(comp_t), comp, comp_t


def image_like(n: int, seed: int, m_test: int = 0, target_class: int = 5,
               n_class: int = 10, side: int = 28):
    """MNIST-shaped vectors: ~80 % exact zeros, blobs of values in [0, 1].

    Each class prototype is a sum of 2-4 Gaussian blobs on the side x side
    grid; a sample perturbs its prototype with a random shift of the blob
    centres and multiplicative noise, then zeroes pixels below a threshold
    chosen so that about 80 % of pixels are zero.  Labels are one-vs-all
    for ``target_class``.
    """
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:side, 0:side].astype(np.float64)
    protos = []
    for _ in range(n_class):
        k = rng.integers(2, 5)
        centres = rng.uniform(6, side - 6, size=(k, 2))
        widths = rng.uniform(2.0, 4.0, size=k)
        protos.append((centres, widths))

    def draw(m):
        cls = rng.integers(0, n_class, size=m)
        out = np.zeros((m, side * side))
        for i in range(m):
            centres, widths = protos[cls[i]]
            img = np.zeros((side, side))
            for (cy, cx), w in zip(centres + rng.normal(0, 1.0, centres.shape), widths):
                img += np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * w * w))
            img *= rng.uniform(0.6, 1.0, size=img.shape)
            img = img / img.max()
            thr = np.quantile(img, 0.8)
            img = np.where(img > thr, img, 0.0)
            out[i] = img.ravel()
        return out, cls

    X, c = draw(n)
    Xt, ct = draw(m_test)
    y = np.where(c == target_class, 1.0, -1.0)
    yt = np.where(ct == target_class, 1.0, -1.0)
    return X, y, Xt, yt


def gaussian_block(n: int, r: int, seed: int, dtype=np.float16) -> np.ndarray:
    """n x r standard normal block rounded to ``dtype`` (default float16)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, r)).astype(dtype)
