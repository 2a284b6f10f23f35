"""Plain FP64 CPU oracle for the space-time Schur-complement PCG method.

This package is TEST INFRASTRUCTURE.  It is a slow, deliberately unoptimised
restatement of the method of van Venetie & Westerdiep, "A parallel algorithm
for solving linear parabolic evolution equations" (arXiv 2009.08875), written
with numpy / scipy.sparse so that every step can be checked against the paper
by eye.  Only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the GPU library never does, and this package shares
no code, tables or constants with the CUDA sources.

Modules
-------
space   P1 finite elements on uniformly refined triangulations of the unit
        square and the L-shape (Sec. 5, model problem): mass / stiffness
        matrices assembled element by element, prolongation obtained by
        evaluating coarse basis functions at fine nodes, and the symmetric
        multigrid V-cycle that stands in for K_x and K_j (Sec. 3.1, Thm. 3.1,
        Sec. 5.1).
time    P1-in-time matrices M_t, A_t, L (Lemma 4.2), the DG test-space
        matrices T, N, O (Lemma 4.1) by Gauss quadrature, and the three-point
        wavelet transform W_t as the product of Eq. (3.1).
schur   S by Lemma 4.1 (route i) and by Lemma 4.2 (route ii), the
        preconditioner K_X (Thm. 3.1), the right-hand side (Lemma 4.1), PCG
        with the stopping rule (3.3), and Lanczos condition estimates.

Readings of points the paper leaves open are listed in the module docstrings
and collected in the repository's design notes.
"""
