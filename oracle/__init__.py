"""CPU FP64 oracle for the randomized-HSS kernel ridge regression path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or
run anything in this package.  The CUDA path shares no code with it and
never calls it; it never reads an output of the CUDA path.

Plain, slow and written to be checked against the paper by eye:

* ``kernel``      Gaussian kernel, Eq. (1) / Algorithm 1 step 1, difference form.
* ``rng``         Philox4x64-10 (Salmon et al., SC'11) and Box-Muller; the
                  counter-based draws both sides make (random block R,
                  two-means seeding).
* ``prep``        column standardization (Section 5.2, Table 2 caption).
* ``cluster``     recursive two-means ordering and HSS tree (Sections 4.2-4.3).
* ``hss``         HSS representation (Section 3.1) built from explicit blocks
                  by column-pivoted QR interpolative decompositions.
* ``solve``       dense Cholesky solve of (K + lambda I) w = y (Algorithm 1
                  step 2), prediction and accuracy (Algorithm 1 steps 3-4,
                  Eq. (2)), relative residual.

* ``hmatrix``     H-matrix sampler (Section 3.2, H matrix representation):
                  strong admissibility, block partition, ACA, H product.

Parity unpinned: the ranks and memory of an HSS built with an
intermediate tolerance on the synthetic data (the paper prints such
figures only for its real data sets); the limits are pinned (h -> 0:
rank 0, memory of the diagonal blocks; h -> infinity: rank 1, memory by
formula).
"""
