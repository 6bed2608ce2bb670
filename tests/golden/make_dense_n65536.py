"""Writes dense_n65536.txt: the exact dense KRR solve of the 65536-point
SUSY-shaped workload (Algorithm 1 steps 2-4; accuracy Eq. (2)), computed by
the FP64 oracle only (oracle.solve.krr_dense_large: the Gaussian kernel of
Eq. (1) in the difference form, K + lambda I factored by LAPACK's Cholesky
in place, the 32 GiB matrix held once).  The GPU test compares its HSS
solve's test accuracy with the dense accuracy stored here.

Workload: synth.mixture(65536, 8, 16 components, sigma 0.7, seed 2) with
4096 test points, standardized by oracle.prep (train statistics) and
rounded to FP32 (what the library is given), h = 1, lambda = 4, labels +-1
by component parity.

    python tests/golden/make_dense_n65536.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import kernel, prep, solve  # noqa: E402

N, D, COMPS, SIGMA, SEED, M_TEST, H, LAM = 65536, 8, 16, 0.7, 2, 4096, 1.0, 4.0


def main(out=os.path.join(HERE, "dense_n65536.txt")):
    X, y, Xt, yt, _, _ = synth.mixture(N, D, COMPS, SIGMA, SEED, M_TEST)
    Z, Zt, _, _ = prep.standardize(X, Xt)
    Z = Z.astype(np.float32).astype(np.float64)
    Zt = Zt.astype(np.float32).astype(np.float64)
    t0 = time.time()
    w = solve.krr_dense_large(Z, y, H, LAM)
    dec = solve.predict(Zt, Z, w, H)[:, 0]
    lab = solve.sign_pm1(dec)
    acc = solve.accuracy(lab, yt)
    # residual of the dense solve against the same operator, on 512 rows
    rows = np.random.default_rng(0).choice(N, 512, replace=False)
    rho = float(solve.residual(Z, H, LAM, w, y, rows=rows)[0])
    with open(out, "w") as f:
        f.write("# Exact dense FP64 KRR solve (Algorithm 1 steps 2-4, Eq. (2)) of the 65536-point\n")
        f.write("# SUSY-shaped workload; written by tests/golden/make_dense_n65536.py from the oracle\n")
        f.write("# only (LAPACK Cholesky of K + lambda I in place, %d host threads, %.0f s).\n"
                % (kernel.num_threads(), time.time() - t0))
        f.write("n: %d\nd: %d\nh: %g\nlambda: %g\nm_test: %d\n" % (N, D, H, LAM, M_TEST))
        f.write("accuracy: %.10f\n" % acc)
        f.write("dense_residual_512_rows: %.3e\n" % rho)
        f.write("labels: %s\n" % "".join("+" if v > 0 else "-" for v in lab))
    print(out, acc, rho)


if __name__ == "__main__":
    main()
