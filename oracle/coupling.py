"""Problems (2) and (3) of Section 4.2 around the momentum solve (oracle side).

Test infrastructure, like the rest of ``oracle/``.

With the ALE derivatives dropped (Eq. (REDUCEDMATRIX)) the Newton system of a
time step splits into three sub-steps solved in order:

* problem (1), the condensed momentum system for the pressure and velocity
  updates (dp, dv): the path the CUDA library solves;
* problem (2), the discrete zero-order relation between deformation and
  velocity on the interface and in the solid,
  u_n = u_{n-1} + k (1 - theta) v_{n-1} + k theta v_n.  Both sides of its
  Newton step carry the same mass matrix, so it is one vector addition:
  du = r + k theta dv on the nodes of solid cells (interface included),
  velocity components only, with r the relation's residual in nodal form;
* problem (3), the extension of the deformation into the fluid,
  E_ff du_f = b_5 - E_fi du_i: the deformation now known on the fixed nodes
  (from problem (2) on solid and interface nodes, zero on the outer boundary)
  enters the free rows through the coupling of the extension operator before
  the fixed rows and columns are reduced to the identity.

Readings: theta and k are the time-stepping parameter and step size (only
their product enters); r is given in nodal form; the deformation is
prescribed (du = 0) on the outer boundary, so r is zero there.
"""

from __future__ import annotations

import numpy as np


def deformation_update(r, dv, k_theta, solid_nodes, dim):
    """Problem (2): du = r + k theta dv on the nodes flagged in solid_nodes
    (bool per node), zero on every other node.  r and du hold dim components
    per node, dv the dim + 1 components of problem (1) (velocity, then
    pressure)."""
    solid_nodes = np.asarray(solid_nodes, dtype=bool).reshape(-1)
    nodes = solid_nodes.size
    du = np.zeros(nodes * dim)
    U = du.reshape(nodes, dim)
    V = np.asarray(dv).reshape(nodes, dim + 1)[:, :dim]
    R = np.asarray(r).reshape(nodes, dim)
    U[solid_nodes] = R[solid_nodes] + k_theta * V[solid_nodes]
    return du


def extension_rhs(E_full, b5, fixed_nodes, g, dim):
    """Right-hand side of problem (3) with the fixed rows reduced to the
    identity: g on the unknowns of fixed nodes, b5 - E_full g_hat on the free
    ones (g_hat = g on the fixed unknowns, zero elsewhere; E_full the extension
    operator as assembled, a BlockMatrix)."""
    fixed = np.repeat(np.asarray(fixed_nodes, dtype=bool).reshape(-1), dim)
    g_hat = np.where(fixed, g, 0.0)
    rhs = np.asarray(b5, dtype=np.float64) - E_full.matvec(g_hat)
    rhs[fixed] = g[fixed]
    return rhs


def linear_newton_step(solve1, b1, r, k_theta, solid_nodes, solve3, E_full, b5, fixed_nodes, dim):
    """The three sub-steps in order: dw = (dp, dv) from problem (1) (solve1 maps
    a right-hand side to the solution), du on solid and interface nodes from
    problem (2), then du on the fluid nodes from problem (3) (solve3 solves the
    reduced extension system).  Returns (dw, du)."""
    dw = solve1(b1)
    du_s = deformation_update(r, dw, k_theta, solid_nodes, dim)
    du = solve3(extension_rhs(E_full, b5, fixed_nodes, du_s, dim))
    return dw, du
