"""CPU oracle for the low-rank stabilizer-decomposition simulator.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64/integer
restatement of the method of Bravyi, Browne, Calpin, Campbell, Gosset and
Howard, "Simulation of quantum circuits by low-rank stabilizer
decompositions" (arXiv:1808.00128).  Only the test suite, the smoke check
and the benchmark's CPU-baseline leg may import it; the product path (the CUDA
library and its binding) never imports, links or runs anything here, and the
two share no code.  Its only shared dependency is the seeded workload module,
which holds no simulation arithmetic.

Modules
  rng       counter-based SplitMix64 draws (published definition)
  chform    CH-form stabilizer states and their gate rules (Sec. 4.1)
  dense     dense state-vector simulator (ground truth at small n)
  expsum    exponential sums Z(B) (Lemma 3, "Exponential Sum")
  decomp    sum-over-Cliffords decompositions and sparsification
            (Sec. 3.3.2, Lemma 6 "Sparsification")
  estimators  amplitudes, equatorial inner products, norm estimation
            (Sec. 4.3) and Metropolis chains (Sec. 4.2)
  exact     exact chi-sums in Z[zeta8] (integer coordinates, one final
            conversion): the pin against which FP64 and FP32 sums state their
            error per result
  marginals median of means and chain-rule marginal sampling (end of Sec. 4.3)
  mlp       the learned proposal's MADE network (not in the paper)

Parity pins live in tests/ (dense brute force, closed forms, invariants).
Functions without such a pin say "parity unpinned" in their docstring.
"""
