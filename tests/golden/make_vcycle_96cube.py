"""Writes vcycle_96cube_oracle.txt: the FP64 oracle's V(2,2) cycle on the 3d 96^3
workload (Section 4.3 (II): one multigrid V-cycle with the additive Vanka smoother
of Eq. (vanka), omega 0.8, overlap-averaged, zero start on every level), applied
to the workload's seeded right-hand side, at sampled mesh nodes.

The GPU tests compare the library's V-cycle at full size with these values node
by node (a V-cycle is global, and its 110,592 patch inversions do not fit in a
test's time budget).  Only gen/ and oracle/ are used.  Run from the repository
root:  python tests/golden/make_vcycle_96cube.py   (about 30 GB of host memory).
"""

from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from gen import build_system, config_problem  # noqa: E402
from oracle.multigrid import Hierarchy  # noqa: E402
from oracle.precision import with_fp32_arithmetic  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "vcycle_96cube_oracle.txt")
SAMPLES = 1024


def sample_nodes(cells, k, seed):
    """k seeded uniform nodes plus the corners, the centre and one node on each
    side of the solid interface plane z = 1/3 of this workload."""
    nn = [c + 1 for c in cells]
    nodes = int(np.prod(nn))
    rng = np.random.default_rng(seed)
    pick = set(int(v) for v in rng.integers(0, nodes, k))
    for z in (0, nn[2] - 1, nn[2] // 3 - 1, nn[2] // 3, nn[2] // 3 + 1, nn[2] // 2):
        for y in (0, nn[1] // 2, nn[1] - 1):
            for x in (0, 1, nn[0] // 2, nn[0] - 2, nn[0] - 1):
                pick.add(x + nn[0] * (y + nn[1] * z))
    return np.array(sorted(pick), dtype=np.int64)


def main():
    t0 = time.time()
    s = build_system(config_problem("cfg4"))
    h = Hierarchy(s.levels, s.dirichlet)
    r = s.rhs.astype(np.float32).astype(np.float64)   # what the library's binary32 V-cycle is given
    z = h.vcycle(r)
    # the same cycle run the reduced-precision way (binary32 matrices, vectors and arithmetic,
    # inverses rounded to each storage format): the scale of the rounding errors, per component
    nc = s.problem.ncomp
    r32 = r.astype(np.float32)
    dz = {fmt: np.abs(with_fp32_arithmetic(h, fmt).vcycle(r32) - z).reshape(-1, nc).max(axis=0)
          for fmt in ("fp32", "bf16")}
    Z = z.reshape(-1, nc)
    nodes = sample_nodes(s.fine.cells, SAMPLES, 96)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle V(2,2) cycle z = M r on the 3d 96^3 workload (Section 4.3 (II), Eq. (vanka),\n")
        f.write("# omega 0.8, overlap-averaged patch corrections, 6 levels, exact coarse solve), r = the\n")
        f.write("# workload's right-hand side (rhs seed 1, convection seed 0) rounded to binary32.  Written by\n")
        f.write("# tests/golden/make_vcycle_96cube.py from gen/ and oracle/ only.\n")
        f.write(f"# max_abs_z {np.abs(z).max():.17e}\n")
        f.write(f"# norm2_z {np.linalg.norm(z):.17e}\n")
        # per component: how far the binary32 model of the cycle lies from z (r rounded to binary32)
        f.write("# max_abs_dz_fp32_model " + " ".join(f"{v:.17e}" for v in dz["fp32"]) + "\n")
        f.write("# max_abs_dz_bf16_model " + " ".join(f"{v:.17e}" for v in dz["bf16"]) + "\n")
        f.write("# node z_0 z_1 z_2 z_3\n")
        for v in nodes:
            f.write(f"{v} " + " ".join(f"{Z[v, c]:.17e}" for c in range(nc)) + "\n")
    print(f"wrote {OUT}: {nodes.size} nodes in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
