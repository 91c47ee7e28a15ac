"""FP64 CPU oracle for the structured-operator hot path (TEST INFRASTRUCTURE).

This package is the plain, slow, obviously-correct reference that the CUDA
library is checked against.  It is test infrastructure: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it.  The product path never calls it, and it never
imports the product package.

Every operator carries

* ``dense()``     -- its matrix written out from the definition (tiny sizes),
* ``row(i)``      -- one row of that matrix from the definition (sampled checks
                     at full size),
* ``apply(X, adjoint=False)`` -- the fast route the paper describes (FFT
                     convolution, Eq. (5); butterflies; mode products), in FP64,
                     with columns of ``X`` as vectors (shape ``[cols, K]``).

``fista`` follows the accelerated proximal-gradient iteration step by step;
``omp`` (module ``omp``) the greedy selection with a least-squares solve per
step; ``gradients`` the parameter gradients of Diag, Circulant and Toeplitz;
``ndt`` the block matrix and two-level Toeplitz of the ultrasound model;
``lfsr`` the shift-register sequence of the LFSR circulant.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (definitions against independent library
routines, closed forms, invariants and brute force).  Nothing is unpinned.
"""
from .operators import (  # noqa: F401
    Op, Fourier, Circulant, Toeplitz, Hadamard, Diag, Partial,
    Product, Sum, BlkDiag, Kron, embedding_spectrum,
)
from .fista import soft, lipschitz, lambda_from_b, fista, objective, fista_problem  # noqa: F401
from .ndt import Blocks, Toeplitz2  # noqa: F401
