"""FP64 CPU oracle for the phiks hot path (test infrastructure only).

This package is a plain, slow, independent restatement of what the method
computes, used by the tests, by `__graft_entry__.smoke()` and by the CPU
baseline leg of `bench.py`.  Nothing in the library package imports it, and it
imports nothing from the library: the two share only the seeded inputs in
`workloads`.

Modules
  phi_scalar    phi_l(z) of a scalar (definition Sec. 1; recurrence)
  kron          Kronecker sum (Sec. 1), mu-mode product and Tucker operator
                (Sec. 2, Lemma 1)
  expm          dense matrix exponential by Taylor scaling and squaring
  dense         O1: exact results from one augmented-matrix exponential
                (Theorem 2.1 of Al-Mohy & Higham 2011 as stated in Sec. 2)
  eig           O2: separable eigendecomposition of tridiagonal Toeplitz A_mu
                in extended precision
  taylor_action O3: Taylor action of the augmented matrix with K x applied by
                mu-mode products with the A_mu
  quadrature    Gauss-Lobatto-Legendre and Gauss-Legendre rules on [0, 1]
  params        choice of s and q (Sec. 3.3)
  phiks_ref     the phiks algorithm (Sec. 3.1, 3.2) restated step by step
  integrators   exponential Runge-Kutta schemes of Sec. 4 (exp. Euler, ETD2RK,
                expRK3, expRK4s5, expRK4s6) with every phi term its own Taylor
                action, and the ADR, Allen-Cahn and Brusselator nonlinear terms

Parity status: every function has pins (tests/test_oracle_pins.py,
tests/test_integrators.py, tests/test_complex_oracle.py); the parameter table
(Table 1) is reproduced softly, since it depends on readings of unstated
constants (see the `params` module header).
"""
