"""FP64 CPU oracle for the 2D electrostatic trench PIC (test infrastructure).

This package is TEST INFRASTRUCTURE.  It is a plain, slow restatement of
the paper's per-timestep loop in double precision (numpy / scipy), written
from the paper (Lin & Nishimura, arXiv:1610.03918, Sec. II and III) and not
from the CUDA path: the two share no code.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline / reference arm
may import it.  The product library never calls into it.

Modules
  geometry  conductor cell mask, Dirichlet node mask and values (Sec. III)
  deposit   cloud-in-cell charge assignment (weighting not stated by the
            paper; bilinear is the reading taken)
  poisson   the normalised Poisson equation, Eq. (5), as a masked 5-point
            system; direct sparse solve, separable DFT solve (doubly
            periodic), Gauss-Seidel and Jacobi (the paper's own solvers)
  field     E = -grad(Phi) with central differences inside and two-point
            one-sided differences at boundaries (Sec. II)
  push      CIC gather, leapfrog of Eqs. (1)-(4), absorption with face
            classification and wall tallies (Sec. III-A, III-C)
  sim       the time loop and the diagnostics
  units     the normalisation of Sec. II and the Sec. III unit example

Parity status of each function is stated in its docstring ("pinned by"),
and the ones without an external pin say "parity unpinned".
"""
