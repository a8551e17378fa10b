"""Plain FP64 CPU oracle of the domain-wall multigrid hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import this package; the product path
(the CUDA library and its Python binding) never does, and the two share no
code.  Everything here is written from the paper's definitions
(Brower, Clark, Howarth, Weinberg, "Multigrid for chiral lattice fermions:
domain wall", arXiv:2004.07732):

  dirac   -- Wilson kernel D_W (Sec. 2), Shamir D_DW(m) (Eq. DWoperator),
             D_PV = D_DW(1) (Sec. 2.2), adjoints, K_DW / D_ov (Eqs. DWFmatrix,
             Overlap), free-field momentum blocks (Sec. 2.2, App. A)
  mg      -- near-null relaxation, chiral doubling, block orthonormalisation,
             Galerkin P^dag D_W P, coarse D_DW / D_PV (Eq. coarsenDW),
             truncated restriction / prolongation (Eq. TruncProjectInterpolate),
             the K-cycle (Sec. 2.3 Summary, Table kcycle)
  solvers -- CGNR on the normal equations (Sec. 2.1), GCR
  force   -- gradient of |D_DW^-1 b|^2 with respect to U(1) link angles

Matrices are assembled explicitly as scipy.sparse CSR in the canonical
vector order psi[s][x_{nd-1}]...[x_0][spin][color] (x0 fastest).

Parity status: every function is pinned by a CPU test against a closed form,
a paper identity, brute force or finite differences, except the K-cycle's
iteration counts, which are "parity unpinned" (the paper's ensembles are not
available, so its counts cannot be reproduced).
"""
