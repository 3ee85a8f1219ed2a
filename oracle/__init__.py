"""Test oracle: a plain, slow, FP64 CPU restatement of the modal DG residual.

This package is TEST INFRASTRUCTURE.  Only the tests, the smoke check and
the benchmark's CPU-baseline leg may import it; the library never does, and
it imports nothing from the library.  It shares no code, table or constant
generator with the CUDA path: its quadrature rules, basis, mesh
connectivity, geometry, fluxes and adjoint are computed here independently,
written for a reader to check against the paper by eye rather than for
speed.

What it follows (arXiv:2209.01877, Sec. II):
  * conservative Euler equations, Eq. 1-4 (restated in 3D, Euler only);
  * the modal expansion Q = sum_j c_j b_j, Eq. 10;
  * the weak form with volume, interior-face and boundary-face integrals,
    Eq. 11, evaluated by Gaussian numerical integration (Sec. II-B);
  * a Roe inviscid flux (Sec. II-B); Rusanov is added as a second flux;
  * explicit Runge-Kutta time marching (Sec. III), here SSP-RK3;
  * the local time step and its global minimum (Sec. III-C).
Everything 3D- and tetrahedron-specific is a reading of the paper, listed in
each module's docstring.

Parity status per function (what pins it is in tests/test_oracle_*.py):
  quadrature rules     pinned: closed-form monomial moments
  basis                pinned: orthonormality under an independent rule,
                       hand-derived closed forms, finite-difference gradients
  mesh / geometry      pinned: face matching counts, closed-surface sums,
                       total volume
  fluxes               pinned: consistency, rotational invariance, Roe
                       property, dissipation matrix vs eigendecomposition
  residual             pinned: free-stream preservation, discrete
                       conservation, divergence theorem for constant states,
                       design order of accuracy on an exact solution
  SSP-RK3              pinned: amplification factor on y' = lambda y
  VJP / JVP            pinned: complex-step JVP vs central differences,
                       dot-product identity with the VJP
  boundary ghost states pinned: zero wall mass flux, free-stream preservation
                       with boundaries
  Navier-Stokes lines  pinned (oracle/ns.py): BR1 gradient exact for
  (BR1, viscous flux)  polynomial states, chain rule vs complex step,
                       conservation, free stream, shear-wave consistency
"""
