"""The plane layout's geometry in the CUDA sources against the grid of the
paper, on the CPU.

A host-only program compiled with nvcc prints, from csrc/common.cuh, every
plane's half-lattice offset, the partner plane holding its neighbours along
each axis, the cell shift of the neighbour at +-dx_a/2 and the sign class of
the y/z differences.  They must follow from the grid definitions (Sect. 2:
A (j), (j+(1/2,1/2,0)); B (j+(1/2,0,1/2)), (j+(0,1/2,1/2)); C (j+(0,0,1/2)),
(j+(1/2,1/2,1/2)); D (j+(1/2,0,0)), (j+(0,1/2,0)); Sect. 3: u, v = A, D
without z): a neighbour of a value at half-lattice 2j+o lies at 2j+o+-e_a,
on the plane with that offset, in cell floor((o_a +- 1)/2) + j_a; the sign
class is (o_x + o_y) mod 2 (Eqs. ss1-ss4: A, C (and u) one pattern, B, D
(and v) the other).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1309_3452_gb300", "csrc")

# the paper's grid, in units of dx/2, in the canonical plane order
GRID = {3: [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1), (0, 0, 1), (1, 1, 1), (1, 0, 0), (0, 1, 0)],
        2: [(0, 0, 0), (1, 1, 0), (1, 0, 0), (0, 1, 0)]}
UPPER = {3: 4, 2: 2}  # A, B (u) first

PROGRAM = r"""
#include <cstdio>
#include "common.cuh"
using namespace dirac;
template <int D> void dump() {
  for (int p = 0; p < nplanes<D>(); ++p)
    for (int a = 0; a < 3; ++a)
      std::printf("%d %d %d %d %d %d %d %d %d\n", D, p, a, plane_off<D>(p, a), a < D ? partner<D>(p, a) : -9,
                  a < D ? nb_shift<D>(p, a, +1) : -9, a < D ? nb_shift<D>(p, a, -1) : -9, sign_class<D>(p),
                  (int)is_upper<D>(p));
}
int main() { dump<3>(); dump<2>(); return 0; }
"""


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("geom")
    src = d / "geom.cu"
    src.write_text(PROGRAM)
    exe = d / "geom"
    subprocess.run(["nvcc", "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    rows = {}
    for line in out.splitlines():
        dims, p, a, off, part, up, dn, sc, upper = map(int, line.split())
        rows[(dims, p, a)] = (off, part, up, dn, sc, upper)
    return rows


@pytest.mark.parametrize("dims", [2, 3])
def test_plane_geometry_follows_the_grid(table, dims):
    grid = GRID[dims]
    for p, o in enumerate(grid):
        for a in range(3):
            off, part, up, dn, sc, upper = table[(dims, p, a)]
            assert off == o[a], (dims, p, a)
            assert sc == (o[0] + o[1]) % 2
            assert upper == (p < UPPER[dims])
            assert upper == ((o[0] + o[1] + o[2]) % 2 == 0)  # upper values: x+y+z even on the half lattice
            if a >= dims:
                continue
            want = list(o)
            want[a] ^= 1
            assert part == grid.index(tuple(want)), (dims, p, a)
            assert up == (o[a] + 1) // 2 and dn == (o[a] - 1) // 2, (dims, p, a)
