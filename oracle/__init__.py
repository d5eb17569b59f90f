"""FP64 CPU oracle of the multigrid-preconditioned FGMRES solve (test infrastructure).

This package is test infrastructure, not product code.  Only the tests, the
smoke check in ``__graft_entry__`` and the CPU-baseline / reference legs of
``bench.py`` may import or run it; the CUDA library never does, and the
oracle shares no code with it (no kernels, headers, index helpers, tables or
pre/post-processing).  It is a plain, slow, step-by-step restatement of the
method of Section 4.3 in float64:

* ``mesh``      node, patch and Dirichlet bookkeeping on uniform meshes
* ``bsr``       block-sparse matrices of Section 4.3 and their product
* ``vanka``     patch matrices A_i = R_i A R_i^T, exact inverses, Eq. (vanka)
* ``transfer``  Q1 prolongation and its transpose (restriction)
* ``multigrid`` the V-cycle preconditioner of item (II)
* ``fgmres``    the outer flexible GMRES of item (I)
* ``solver``    the whole solve
* ``coupling``  problems (2) and (3) of Section 4.2 around the momentum solve

Where the paper is silent (transfers, coarse solver, stopping norm, GMRES
variant) each module states the reading it implements.
"""

from .solver import OracleSolver, solve  # noqa: F401
