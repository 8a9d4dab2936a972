"""Plain, slow FP64 CPU oracle for the ghost-cell immersed-boundary pressure Poisson solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or calls this package; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code with the CUDA path: both receive the same inputs from the
seeded generators in ``synth`` and are compared on their outputs.

What it computes, and where the paper states it (arxiv 2605.04335):

* ``grid``     -- cell centres, widths and the 7-point finite-difference
                  coefficients on a stretched cell-centred Cartesian grid
                  (Sec. "Governing Equations and Numerical Methods": second-order
                  finite differences on a non-conformal Cartesian grid).
* ``classify`` -- "iblanking": inside/outside classification of cell centres
                  against a triangulated body (Sec. "GPU Porting", item 1),
                  ghost cells, boundary intercepts, image points and trilinear
                  interpolation weights of the ghost-cell method (item 2).
* ``system``   -- the discrete pressure Poisson system with ghost rows
                  enforcing dp/dn = 0 (fractional-step projection, same
                  section; ghost-cell method, Sec. "GPU Porting"), its
                  residual, the projected relative residual and the gauge.
* ``solve``    -- the exact discrete solution of that system by library
                  direct solvers (dense or sparse LU of the bordered system).

Every pin that ties these functions to something other than themselves
(closed forms, DCT solves, invariants, brute force) lives in
``tests/test_oracle_*.py``.  Parity status per function is listed in each
module's docstring.
"""
