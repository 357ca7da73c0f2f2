"""The sum-factorised evaluation plan on the host (no GPU): for several grid
shapes the plan built by the library evaluates the interpolant's sum exactly
as the direct sum over the nodes (an FP64 emulation of the kernel's products,
epilogue and CUDA-core columns, tests/host/sf_plan_check.cu), every table read
stays in range and every accumulator read was written.  Shapes whose plan
does not fit report so and fall back to the per-node kernel."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    from paper_1507_04769_gb300 import build
    lib = build.build()
    nvcc = build.nvcc()
    out = str(tmp_path_factory.mktemp("sfplan") / "sf_plan_check")
    src = os.path.join(ROOT, "tests", "host", "sf_plan_check.cu")
    libdir = os.path.dirname(lib)
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1", src, "-o", out, f"-L{libdir}", "-lsg",
                        "-Xlinker", f"-rpath={libdir}"], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr[-2000:])
    return out


@pytest.mark.parametrize("d,L,k", [(6, 4, 3), (6, 2, 3), (3, 5, 2), (6, 3, 8), (2, 1, 1), (4, 3, 5), (8, 2, 2),
                                   (5, 3, 7), (6, 4, 1), (2, 6, 3), (6, 0, 3), (7, 3, 4), (4, 4, 3), (6, 1, 3)])
def test_plan_reproduces_the_direct_sum(checker, d, L, k):
    r = subprocess.run([checker, str(d), str(L), str(k)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("d,L,k", [(6, 5, 3), (1, 5, 2), (6, 4, 9)])
def test_shapes_without_a_plan_fall_back(checker, d, L, k):
    r = subprocess.run([checker, str(d), str(L), str(k)], capture_output=True, text=True)
    assert r.returncode == 2, r.stdout + r.stderr
