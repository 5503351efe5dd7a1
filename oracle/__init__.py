"""FP64 CPU oracle for the coarse-grid correction of two-level DD-alpha-AMG.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the GPU library computes; it exists so the tests (and the
benchmark's CPU-baseline leg) can check the CUDA path against it.  Nothing in
the product path imports it, and it imports nothing from the product path.

Modules (each function cites the passage of arXiv:1512.04506 it follows):

* ``lattice`` -- geometry: blocks, aggregates, coarse neighbours (Sec. 2).
* ``dirac``   -- gamma matrices, clover field, Wilson-clover D (Alg. 7 terms).
* ``coarse``  -- Gram-Schmidt on aggregates, R, P = R^dagger, D_c = R D P,
                 restriction, coarse-operator application, prolongation
                 (Alg. 2, Alg. 5, Eq. R, Eq. cgo, Eq. dagger).
* ``krylov``  -- the restarted FGMRES coarse solve of Alg. 2.
* ``evenodd`` -- the even/odd (Schur complement) reduction of the coarse system
                 that Alg. 2's coarse solve is preconditioned with.
* ``smoother`` -- the domain-decomposition smoother of Alg. 3 (SAP over two
                 block colours, exact or minimal-residual block solves).
* ``mg``      -- the two-level method around the coarse-grid correction: the
                 V-cycle (Alg. 1), the adaptive setup (Alg. 4) and the outer
                 FGMRES solve of D u = f (Sec. 1).
* ``mg3``     -- a third level (Sec. 3 notes the method carries over): the
                 coarse lattice coarsened once more, R2, D_cc = R2 D_c P2, a
                 minimal-residual smoother on D_c, the two-grid cycle on level 1
                 and the three-level V-cycle.

All arithmetic is complex128.  Where the paper is silent (gamma basis, sign
and normalisation of D, the clover term, boundary conditions) the readings
are fixed in each function's docstring and pinned by tests/test_oracle_*.py
against closed forms and brute force, not against this code.
"""
