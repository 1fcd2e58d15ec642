"""Plain FP64 CPU oracle for the non-Hermitian FEAST eigensolver
(Kestyn, Polizzi, Tang, "FEAST eigensolver for non-Hermitian problems").

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import it.  It shares no code
with the CUDA path (paper_1506_04463_gb300/csrc) and imports nothing from it.

Every routine follows the paper step by step in numpy/scipy FP64:
  contour.py  - trapezoid nodes/weights (Sec. 2.3), rational filter (eq. rational)
  feast_nh.py - contour integration (eq. qr/ql), spurious test (Sec. 2.7),
                resize + B-bi-orthonormalisation (Sec. 2.5-2.6, eq. uu),
                Rayleigh-Ritz (Fig. alg:three step 4), residual (eq. res),
                convergence test (step 5) and the outer loop.
Pins (tests/test_oracle_*.py): closed forms of the filter, closed-form
spectra, brute-force QZ eigenvalues, invariants and the convergence-rate law.
"""
