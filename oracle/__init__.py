"""FP64 CPU oracle for the phase-field fracture hot path (Kolditz & Wick, arXiv 2404.03265).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2404_03265_gb300``) never imports it and has
no CPU fallback.  Nothing here shares code with the CUDA path: the quadtree, the
hanging-node constraints, the finite-element tables and every operator are
written out again from the paper, deliberately plainly (explicit sparse
assembly, full shape-function tables, no sum factorisation, no blocking).

Modules
-------
fe         1D Gauss rule and Q_k Lagrange basis on the unit square (Sec. 3: H^1
           conforming Q_k elements).
mesh       quadtree with 2:1 face balance, nodes, hanging-node constraints,
           Dirichlet nodes (Sec. 3, Sec. 4 local refinement).
operators  residual A(U) (Problem 2), Jacobian A'(U) (Sec. 3.1), constrained
           system, lumped mass, active set (Eq. AcInS, Algorithm 2), TCV (Sec. 4).
mg         level meshes, local-smoothing V-cycle with Chebyshev-Jacobi smoothing,
           eigenvalue estimate, transfers, coarse solve (Sec. 3.2).
solvers    left-preconditioned GMRES, Newton / primal-dual active set with line
           search (Algorithms 1 and 2).
adjoint    gradient of the total crack volume of a converged load step with
           respect to p, G_c and a per-cell Young's modulus (adjoint solve with
           the transposed constrained Jacobian of Sec. 3.1).

Parity status of each function is stated in its module header; the pins live
in ``tests/test_oracle_*.py``.
"""
