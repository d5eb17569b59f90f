"""The level matrix's stencil layout (stencil_off in nmg_internal.cuh), checked
on the host: for 2d and 3d geometries and block sizes 4, 9 and 16, every
(position, entry, node) maps to its own offset inside the nst * nb * ld
elements the library allocates, 3d blocks of one node and position are
contiguous, and 2d entries of consecutive nodes are.  The check program is
compiled with nvcc and runs on the CPU only (the helpers are host-callable)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_02401_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "nmg_internal.cuh"
using namespace nmg;

template <int DIM, int NB>
static int check(int64_t nodes) {
    const int nst = DIM == 3 ? 27 : 9;
    const int64_t ld = (nodes + 31) / 32 * 32;
    const int64_t total = (int64_t)nst * NB * ld;
    std::vector<unsigned char> seen((size_t)total, 0);
    for (int s = 0; s < nst; ++s)
        for (int e = 0; e < NB; ++e)
            for (int64_t i = 0; i < ld; ++i) {
                const int64_t o = stencil_off<DIM, NB>(ld, s, e, i);
                if (o != stencil_off(DIM, NB, ld, s, e, i)) { printf("runtime/template differ\n"); return 1; }
                if (o < 0 || o >= total) { printf("out of range\n"); return 1; }
                if (seen[(size_t)o]++) { printf("offset used twice\n"); return 1; }
                if (e + 1 < NB && stencil_off<DIM, NB>(ld, s, e + 1, i) - o != stencil_estride<DIM>(ld)) {
                    printf("entry stride\n"); return 1;
                }
                if (DIM == 3 && e == 0 && (o * 4) % 16 != 0 && NB % 4 == 0) { printf("block alignment\n"); return 1; }
                if (DIM == 2 && i + 1 < ld && stencil_off<DIM, NB>(ld, s, e, i + 1) != o + 1) {
                    printf("2d node stride\n"); return 1;
                }
            }
    return 0;
}

int main() {
    int bad = 0;
    bad |= check<2, 4>(35);  bad |= check<2, 9>(35);  bad |= check<2, 9>(289);
    bad |= check<3, 9>(125); bad |= check<3, 16>(125); bad |= check<3, 16>(729);
    printf(bad ? "FAIL\n" : "OK\n");
    return bad;
}
"""


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_stencil_layout_offsets(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "layout_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "layout_check"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout + out.stderr
