"""FP64 CPU oracle for the tensor-train point-mass filter (arXiv 2501.07942).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes this directory; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may.  The oracle shares no code with the CUDA
path: it is a plain, slow, dense full-grid point-mass filter written from the
paper's equations, in float64 numpy, plus a plain tensor-train toolkit used to
densify and check TT results.

Modules
-------
pmf     dense point-mass filter: grid, prior, predictive step (re-gridded
        transition and textbook direct sum), Bayes update, moments
        (Sec. 2: Eqs. pdf_pm, pdf_predII, TPMmat, tpmconvFFT,
        pmf_filtrace_a/b; Alg. 2 and Alg. 3 step structure).
kalman  Kalman filter for linear-Gaussian variants (used to pin the oracle).
tt      tensor-train format helpers (Sec. 3, Eq. ttd_exact): densify, inner
        products, TT rounding by the QR + truncated-SVD sweeps.

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against closed forms, invariants, special cases
or brute force; none is "parity unpinned".
"""
