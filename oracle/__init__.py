"""CPU oracle for controlled reduction (zeta functions of smooth hypersurfaces).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, calls,
links or executes anything here; only the tests, the smoke check and the
benchmark's CPU-baseline leg do.  The oracle shares no code with the CUDA
path: the only module both sides use is the seeded input generator
(`zeta_inputs`), which holds none of the method's arithmetic.

The oracle is written for a reader checking it against the paper by eye:
exact integer arithmetic (Python big integers) mod p^M, the steps in the
paper's order and notation, no blocking or fusion.  A small C routine
(`horner.c`) runs Algorithm 2's inner loop for moduli below 2^63; it is the
same loop as `zeta.horner_python` and is tested against it.

Modules
  algebra     monomials, polynomials, Gaussian elimination mod p^k
  cohomology  smoothness and S-smoothness tests (Definition 3.1), monomial
              basis (Sec. 2.3), section of the map of J_S, R_{u,v} (Prop. 3.3,
              any index set S), final Griffiths-Dwork reduction (Sec. 3.3
              step (2))
  precision   r_m, N_m and the algorithm precision M (Sec. 2.5)
  policies    Tweak (Alg. 1), greedy direction (Alg. 3), the reduction game
              (Sec. 3.4) and the three policies of Sec. 4
  zeta        Frobenius expansion (Prop. 2.1), the reduction driver with
              Algorithm 2, normalisation, det(1 - T F) and the lift to Z[T]
  pins        independent checks: point counts over F_{p^r}, Gauss sums for
              diagonal hypersurfaces, Hasse-Witt matrices, Weil bounds
"""
