"""FP64 CPU oracle for USBS (Unified Spectral Bundling with Sketching, arXiv 2312.11801).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of the method that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may import
it.  It shares no code with ``paper_2312_11801_gb300`` (the product): the one module
both read is ``paper_2312_11801_gb300.instances``, which only builds seeded inputs.

Modules
-------
``svec``   App. B: svec, the U matrix, the symmetric Kronecker product (two definitions).
``eig``    extreme eigenpairs: cyclic Jacobi (n <= 64), dense LAPACK (n <= 4096),
           block Lanczos with full reorthogonalisation and thick restart above that.
``ipm``    App. B.2 primal-dual interior point method for eq. compressed_subprob_2;
           App. B.1 as its special case with zero quadratic data; the closed form of
           the model value.
``nystrom`` the stable Nystrom reconstruction of the primal from its sketch (App. C,
           eq. nystrom_approx; Tropp et al. 2017, Algorithm 3) and MaxCut rounding (App. E).
``usbs``   problem scaling (App. E), the operators A, A*, the USBS iteration
           (Algorithm 1, Sec. 3) with the implicit primal and the Nystrom sketch
           (Sec. 4, App. C), the stopping gates (eq. relative_error_tol) and solve.

Parity status: every function is pinned by tests under ``tests/test_oracle_*.py``
except where a docstring says "parity unpinned".
"""
