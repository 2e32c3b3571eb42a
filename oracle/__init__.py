"""CPU FP64 oracle for the NUFFT evaluation of phi = U * rho (arXiv:1410.3584).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct code that the GPU
path is checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import it; the product package never does,
and the two share no code (only the seeded input generators in workloads/).

Tiers (each function cites the passage it follows):
  O1  direct sums of the discrete quadrature definition      potential.eval_direct
  O2  plain FP64 NUFFT (type 2 -> scale -> type 1)            potential.eval_nufft
  O3  continuum closed forms for Gaussian densities           closed_forms
  plus Algorithm 1 (2D Poisson), the normalized gradient flow (Sec. 3) and
  time splitting (Sec. 4) built on these evaluators.

Parity pins (see tests/test_oracle_*.py): GL rules vs polynomial exactness,
O2 vs O1 on small grids, O1/O2 vs closed forms at the paper's printed error
levels (Tables tab:exmp1, tab:sqrt:nufft, tab_NUFFT_2D_Poisson), invariants of
the discrete operator, and ground-state energies vs Table tab:virial:3d:sps.
"""
