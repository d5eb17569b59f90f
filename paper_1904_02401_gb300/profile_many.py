"""Drives the multi-vector V-cycle for an ncu capture: builds the 3d n^3
condensed-momentum hierarchy (FP32 patch inverses only, solid z < 0.25) with
the given number of levels and runs two 8-column V-cycles with plain launches.

    python paper_1904_02401_gb300/profile_many.py 48 4
"""
import sys
import numpy as np
import torch
sys.path.insert(0, ".")
from gen import Problem, build_system
from paper_1904_02401_gb300 import nmg
from paper_1904_02401_gb300.session import Session, solve_opts
n = int(sys.argv[1]); levels = int(sys.argv[2])
s = build_system(Problem(dim=3, n=(n, n, n), levels=levels, solid=(2, -1, 0.25)))
S = Session(3, s.problem.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels], s.dirichlet, precisions=(1 << 1))
K = 8
R = torch.from_numpy(np.tile(s.rhs.astype(np.float32), (K, 1))).cuda()
Z = torch.zeros_like(R)
om = solve_opts(precision=1, use_graph=0)
for _ in range(2):
    nmg.check(nmg.nmg_vcycle_many(S.handle, om, K, R, Z))
torch.cuda.synchronize()
print("ok", float(Z.abs().sum()))
S.close()
