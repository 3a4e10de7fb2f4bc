"""Plain, slow FP64 CPU oracle for the paper's method (arXiv 2306.17486).

TEST INFRASTRUCTURE ONLY.  This package is imported, called or executed only by
`tests/`, by `__graft_entry__.smoke()` (to check one small GPU result) and by
`bench.py`'s `cpu_baseline` / `--impl reference` legs.  The product path (the
CUDA library and its Python binding) never imports it, and it never imports the
product path.  Everything here is complex128 / float64 NumPy, written to be
checked against the paper by eye; each function cites the section or equation
it restates.

Modules
  helmholtz  - Eq. (1)-(3): operator, absorbing layer, frequency rule, mass terms
  multigrid  - Eq. (4), (6), (8), Algorithm 1: shifted-Laplacian V-cycle
  fgmres     - flexible GMRES (Saad 1993), right-preconditioned, restarted
  implicit   - Eq. (14), (15): implicit layer and Green's function, adjoints
  cnn        - encoder-solver U-Net (Sections 4.1-4.4, 5.3), forward + backward; also
               the explicit U-Net of Section 6 (the same network without the implicit step)
  training   - Eq. (16) loss, Eq. (17) data generation, Adam

Pins: every function above is checked against something other than itself (assembled
matrices, dense LU, closed forms, LFA, finite differences, the paper's printed
constants) by the `-m "not gpu"` tests.  Parity unpinned: the results of training and
the iteration counts of a trained network, implicit or explicit (the paper's datasets
and weights are not available).  `training.composed_preconditioner` is pinned by the
special cases its algebra fixes: a zero network output gives the plain V-cycle, the
exact error is returned unchanged, and z - e is the V-cycle of the remaining residual.
The boundary term that Neumann and Sommerfeld problems put on the coarse multigrid
levels follows a reading (each level carries the same condition on its own grid); each
level's operator is pinned against the ghost-value definition of the condition on that
grid and against its closed forms on the constant vector.
"""
