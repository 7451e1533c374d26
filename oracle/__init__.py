"""CPU oracle for the sketched-and-truncated polynomial Krylov method (s-PKSM).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 NumPy/SciPy
restatement of the method of Palitta, Schweitzer and Simoncini, "Sketched and
truncated polynomial Krylov subspace methods: matrix Sylvester equations"
(arXiv 2311.16019): Algorithm 1 (s-PKSM), Algorithm 2 (t-PKSM), the full
block Arnoldi method of Section 2.1 and the sketch of Section 2.2.

Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference arm of
bench.py may import it.  It shares no code with the CUDA library (not a
kernel, header, helper, table or constant generator); the two meet only in
the seeded problem generators of paper_2311_16019_gb300.inputs, which hold
none of the method's arithmetic.

Modules
  sketch   - subsampled randomized Hadamard and DCT sketches from SplitMix64 draws
  spkms    - Algorithm 1 step by step (plus the Section 5 bordering update)
  tpkms    - Algorithm 2 (truncated Arnoldi, no sketch)
  arnoldi  - full block Arnoldi / Galerkin (Eq. (2.1), Eq. (3.7))
  measure  - gauge-free distances and true residuals of low-rank factors
  adjoint  - dense FP64 gradient of u^T X v for the adjoint checks

Parity status of each function is stated in its docstring; every function
here is pinned by tests/test_oracle_*.py unless it says "parity unpinned".
"""
