"""FP64 CPU oracle for the nonconforming-grid transmission BEM (arXiv 2206.00708).

TEST INFRASTRUCTURE ONLY.  Only the tests, `__graft_entry__.smoke()` and the
`cpu_baseline` / reference legs of `bench.py` may import this package.  The CUDA
library never calls it, and this package never imports the CUDA library: the two
share no code.  Inputs come from `bem_inputs`, which holds no method arithmetic.

The oracle is plain, vectorised NumPy in float64/complex128, written to be read
against the paper:

* `quadrature`  -- degree-4 symmetric 6-point triangle rule (solved from its moment
                   equations), Gauss-Legendre on [0,1] (Sec. 5.1, "order four").
* `geometry`    -- triangle Jacobians, outward normals, P1 surface curls (Sec. 2.4).
* `helmholtz`   -- Green's function and the Galerkin V, K, T, D of Sec. 2.1, regular
                   pairs by tensor quadrature, coincident / edge / vertex pairs by
                   Sauter-Schwab transformations (Sec. 5.1).
* `mass`        -- P1 mass matrices M_int, M_ext (Sec. 3.1).
* `mortar`      -- mixed mass matrix P_int,ext between nonconforming grids (Sec. 3.1).
* `mtf`         -- plane-wave data f, g, the discrete multiple-traces system
                   (eq. mtf:discrete), mass-matrix preconditioning and unrestarted
                   GMRES (Sec. 3.3, Sec. 5.1).
* `mie`         -- Mie series for a penetrable sphere, the closed form the whole
                   solve is pinned to.

Parity status: every function is pinned by `tests/test_oracle_*.py` against
closed forms, invariants or brute force; the ellipsoid workloads are pinned only
through those invariants (no closed form exists).
"""
