"""Feature standardization: zero-mean, unit-standard-deviation columns, as
the paper applies to every data set (Section 5.2, caption of Table 2 and
the paragraph after it).  Test points use the training mean and standard
deviation (the paper does not say; this is the usual reading).  A column
with zero spread is divided by 1.

TEST INFRASTRUCTURE ONLY.  FP64, population standard deviation (1/n).
"""
from __future__ import annotations

import numpy as np


def standardize(X, Xt=None):
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    mean = X.sum(axis=0) / n
    var = ((X - mean) ** 2).sum(axis=0) / n
    std = np.sqrt(var)
    std = np.where(std > 0, std, 1.0)
    Z = (X - mean) / std
    Zt = None if Xt is None else (np.asarray(Xt, dtype=np.float64) - mean) / std
    return Z, Zt, mean, std
