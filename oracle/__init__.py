"""CPU oracle for the MPS Vlasov-Poisson hot path (test infrastructure only).

This package is a plain, slow FP64 restatement of Ye & Loureiro,
"A quantum-inspired method for solving the Vlasov-Poisson equations"
(arXiv:2205.11990).  It exists to check the CUDA library: only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
The product path never calls it and shares no code with it; the only module
both sides read is ``paper_2205_11990_gb300.inputs`` (seeded initial
conditions, no method arithmetic).

Modules
-------
mpo        MPOs exactly as printed in the SI ("Derivatives"), MPO sums,
           diagonal MPOs, and their placement on a site ordering.
mps        MPS algebra (SI "Matrix-vector multiplication", "Addition"),
           TT-SVD (Eq. for the MPS decomposition, Sec. "MPS Representation"),
           QR canonicalisation and truncated-SVD compression (SI
           "Canonicalization and Compression"), truncation error (Eq. for
           epsilon_j).
vp         one electron species Vlasov-Poisson operators and the RK4 step
           with compression level C1 (SI "Compressed time evolution").
dense_fd   the same finite-difference scheme on the full grid (no MPS).
dispersion linear dispersion relations (textbook plasma theory, not the
           paper) used to pin the physics of the dense solver.

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test against closed forms, brute force or
textbook values.
"""
