"""CPU FP64 oracle for bootstrapped block Lanczos (Zbikowski & Johnson, arXiv 2210.15763).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, step-by-step
restatement of the paper's method in numpy/scipy, used to check the CUDA
library.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg may import it.  The product path (paper_2210_15763_gb300) never imports,
calls or links anything here, and nothing here imports the product path.

Modules
  rng      - counter-based splitmix64 generator (random pivots, deflation)
  spmm     - W = H V  (Sec. II.B, Eq. 3)
  lanczos  - vector Lanczos (Algorithm 1 + full reorthogonalisation) and block
             Lanczos (Eqs. 4-12) with the paper's spectral normaliser and CholQR2
  pivot    - random and bootstrapped pivot blocks (Sec. II.B, Sec. III)
  mlp      - FP64 forward / backward / Adam of the learned-pivot MLP

Every function cites the passage it follows.  Parity status per function:
all are pinned by tests/test_oracle_*.py (closed forms, brute force,
invariants, library special cases) except the bootstrapped pivot's effect on
iteration counts, which the paper reports as a measured quantity:
"parity unpinned" for that effect only (the pivot itself is pinned).
"""
