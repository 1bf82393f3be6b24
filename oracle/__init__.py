"""Plain FP64 CPU oracle of the spectral-difference residual (test infrastructure).

This package is the independent reference that the CUDA path is checked
against.  It is test infrastructure: only the tests, the smoke entry point and
the CPU-baseline leg of the benchmark may import it; the product library never
does and shares no code with it.  Every function follows the paper's
statement of the method (Wang, Liang & Miesch, JCP 2015, "A compressible
high-order unstructured spectral difference code for stratified convection
in rotating spherical shells") step by step, vectorised over elements with
numpy but with no blocking, fusion or reordering beyond that.

Modules
  sd_points  solution / flux points, Lagrange bases and 1D operators (Eqs. 13-16)
  geometry   20-node iso-parametric map, Jacobian, conservative curl-form metrics (Eqs. 10-12)
  mesh       face pairing, face-point correspondence, wall tagging
  physics    fluxes, sources, polytropic background (Eqs. 1-9, 20-27)
  residual   the semi-discrete SD residual (Eqs. 11-18, Rusanov, BR1-like averaging, Section 5 walls)
  state      seeded initial state (SplitMix64 entropy perturbation), time step
  rk         SSP-RK3 stage update
  diagnostics FP64 volume integrals (mass, energy, kinetic energy, angular momentum, Eq. 32)
"""
