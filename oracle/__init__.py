"""FP64 CPU oracle for the stochastic-GW (sROI) hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method in double precision (numpy), used to prove the CUDA
path right.  Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product path (the C-ABI library and its Python
binding) never does, and shares no code with it.

Modules:
  philox       Philox4x32-10 counter-based generator (the white-noise draws)
  hamiltonian  grid, kinetic energy, local potential, KB projectors, Poisson
  chebyshev    spectral bounds, gapped Heaviside filter (Eq. 3), Chebyshev propagator
  sgw          white noise, filtering, linear-response TDH, time ordering,
               zeta propagation, Sigma(t) (Eq. 4-5), exchange, Sigma(omega) (Eq. 7),
               QP equation (Eq. 6), statistics
  mlp          control variate: features of zeta-bar, the MLP (forward, backward,
               Adam) in FP64, and the unbiased paired estimator

Every function is pinned by tests against closed forms, LAPACK eigh / Casida
dense solves, published known-answer vectors or brute force.
"""
