"""Seeded synthetic inputs for the condensed-momentum solve.

This package builds the inputs that both the CUDA library and the CPU oracle
consume: the level matrices of the condensed momentum Jacobian (problem (1)
of Section 4.2, with the solid deformation eliminated through the discrete
relation d_t u = v of Eq. (defgrad) and the ALE derivatives dropped as in
Eq. (REDUCEDMATRIX)), rediscretised on every multigrid level, plus the
right-hand side and the Dirichlet mask; and the same for the ALE-extension
problem (problem (3) of Section 4.2, n_c = d).  It holds none of the
solver's arithmetic (no matrix-vector product, smoother, transfer or Krylov
step).
"""

from .q1fsi import (  # noqa: F401
    Coefficients,
    ConvectionField,
    LevelMatrix,
    Problem,
    SyntheticSystem,
    assemble_ale_level,
    assemble_level,
    build_ale_system,
    build_system,
    config_problem,
    level_cells,
    reference_element,
)
