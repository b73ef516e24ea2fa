"""CPU oracle for the hierarchical tile QR (HQR) of Dongarra, Faverge, Herault,
Langou and Robert, "Hierarchical QR factorization algorithms for multi-core
cluster systems" (arXiv 1110.1553).

This package is TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check
in ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it. The product path (the CUDA library and its
Python binding) never imports, links or executes anything in here, and nothing
in here imports the product package.

Everything is plain FP64 NumPy, written for a reader to check against the paper
by eye:

* ``elim_list``   -- the elimination-list generator (Sec. 4.1-4.2, Sec. 3.1-3.2,
                     Tables 1-4) and the validity rules of Sec. 2.
* ``kernels``     -- the six tile kernels GEQRT, TSQRT, TTQRT, UNMQR, TSMQR,
                     TTMQR (Sec. 2, Alg. 2), in the compact-WY Householder form.
* ``tile_qr``     -- the tile QR that replays an elimination list (Alg. 1 and
                     Alg. 2), and the application of Q / Q^T by replaying the
                     trees forward or in reverse (Sec. 5.1, correctness check).
* ``householder`` -- an unblocked column-by-column Householder QR (definition
                     oracle for R up to row signs).
* ``lstsq``       -- least squares through the tile QR, a compensated residual
                     (Ogita-Rump-Oishi Dot2) and refinement, and corrected
                     semi-normal equations (Bjorck 1987).
"""
