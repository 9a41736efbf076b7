"""CPU FP64 oracle for the domain-decomposition elasticity solve.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
NumPy/SciPy restatement of what the method computes (Turner, Kocvara, Loghin,
"Parallel Solution of the Linear Elasticity problem with applications in
Topology Optimisation", arXiv:1501.06211).  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` / reference
leg may import it.  The GPU library never imports, links or calls it, and it
imports nothing from the GPU package: the two share no code.  The only common
module is ``workloads`` (seeded input generators, which hold none of the
method's arithmetic).

Modules
-------
fem      Lame constants, plane-stress D, element stiffness by Gauss quadrature,
         structured-grid numbering, global assembly K(rho) (Sec. 1, Sec. 2,
         eq. NumberTen), matrix-free element-by-element products, loads, BCs.
dd       Non-overlapping decomposition: Gamma / interior classification (Sec. 1),
         block partition (eq. NumberFour/NumberFive), Schur complement and the
         three-step solve (eq. 3MatSplit2), the face-local fractional interface
         preconditioner (eq. NumberEight, NumberNine, Sec. 3-4) and interface
         PCG, also in a relaxed mixed-precision form (a low-precision operator
         once the residual is small, with FP64 reliable updates).
direct   Global sparse direct solve with FP64 iterative refinement.
krylov   GMRES on the full block system with the block upper-triangular right
         preconditioner of Sec. 3.
topopt   Density filter, compliance, sensitivities and optimality-criteria
         update of the Picard loop of Sec. 5 (eq. NumberTen with SIMP p).

Every function whose result is not pinned by an independent check in
``tests/test_oracle_*.py`` says "parity unpinned" in its docstring.
"""
