"""Bounds and coverage of the matrix-free kernels' index arithmetic, checked on
the host (no GPU): tests/bounds/stencil_index_check.cpp replays the loop
skeleton of the operator pass and the fused CG pass (tile columns marching
along z, staged halo tile, row sums, boundary rows) with the kernels' own index
functions from csrc/fe_stencil_geom.cuh and fails on any global index outside
[0, m), any shared-memory index outside the staged tiles, or any row not
written exactly once.  Shapes cover the tile edges (nx - 1 = 31, 32, 33;
ny - 1 = 15, 16, 17), meshes one element thick, and the sizes the tests and
the benchmark run; grids cover the launch sizes (SMs x resident blocks) and
extremes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "bounds", "stencil_index_check.cpp")
CSRC = os.path.join(ROOT, "paper_1505_08023_gb300", "csrc")
BIN = os.path.join(ROOT, "tests", "bounds", "_build", "stencil_index_check")

SHAPES = [(1, 1, 1), (2, 2, 2), (1, 3, 5), (3, 1, 2), (5, 4, 1), (32, 16, 2), (33, 17, 9),
          (34, 18, 3), (31, 15, 2), (65, 33, 4), (30, 30, 30), (64, 64, 64), (97, 61, 45),
          (129, 129, 129), (256, 256, 256)]
GRIDS = [1, 7, 152, 304, 456, 608, 4096]


@pytest.fixture(scope="module")
def checker():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    os.makedirs(os.path.dirname(BIN), exist_ok=True)
    tmp = BIN + f".tmp{os.getpid()}"
    subprocess.run([cxx, "-O2", "-std=c++17", "-Wall", "-Werror", "-I", CSRC, "-o", tmp, SRC], check=True)
    os.replace(tmp, BIN)
    return BIN


@pytest.mark.parametrize("dims", SHAPES)
def test_matrix_free_indices_in_bounds_and_rows_covered_once(checker, dims):
    grids = GRIDS if dims[0] * dims[1] * dims[2] <= 2_000_000 else [304, 456]
    r = subprocess.run([checker, *map(str, dims), *map(str, grids)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert r.stdout.count("ok ") == len(grids)


def test_largest_matrix_free_mesh(checker):
    """N = 512, the largest mesh the matrix-free tests solve (past the CSR
    form's int32 limit), in the CG kernel's launch size."""
    r = subprocess.run([checker, "512", "512", "512", "304"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
