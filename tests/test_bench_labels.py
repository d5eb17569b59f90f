"""bench.py names the finest-level apply kernel the library launches for a
workload: the streaming ring for FP32 and BF16 inverses, the warp-per-patch
kernel for FP64, for 2d extension patches and for 3d extension levels of more
than 4096 patches (the rule in launch_vanka_apply)."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("workload,ring", [("cfg2", True), ("cfg3", True), ("cfg4", True),
                                           ("ale2", False), ("ale3", True), ("ale4", False)])
def test_apply_kernel_name(workload, ring):
    import bench
    from gen import config_problem
    p = config_problem(bench.ALE_BASE.get(workload, workload))
    ncomp = p.dim if workload in bench.ALE_BASE else p.dim + 1
    for prec in (1, 2):
        assert bench.apply_kernel_name(p, ncomp, prec) == ("k_vanka_apply_ring" if ring else "k_vanka_apply")
    assert bench.apply_kernel_name(p, ncomp, 0) == "k_vanka_apply"
