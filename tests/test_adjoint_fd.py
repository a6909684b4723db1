"""The hand-written reverse pass of one pixel's sweep update (the photometric
factor of Eq. 3, the identity messages of Eq. 5, the normal-integration messages
of Eq. 6, the structured belief solve and the mean update) against central
finite differences of the same forward, on the CPU: `adjoint_fd/pixel_vjp_fd.cu`
compiles the library's per-pixel functions for the host and checks the gradient
of <ybar, update(x)> with respect to all 395 inputs, with and without the Huber
branch, for an applied and a skipped update and for a border pixel."""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def fd_binary(tmp_path_factory):
    exe = nvcc()
    if exe is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("adjoint_fd") / "pixel_vjp_fd")
    cmd = [exe, "-x", "cu", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2606_03989_gb300", "csrc"),
           "-I", os.path.join(ROOT, "include"), "-o", out, os.path.join(HERE, "adjoint_fd", "pixel_vjp_fd.cu")]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-4000:]
    return out


@pytest.mark.parametrize("huber", [0, 1])
@pytest.mark.parametrize("case", [0, 1, 2], ids=["applied", "skipped", "border"])
def test_pixel_vjp_matches_finite_differences(fd_binary, huber, case):
    res = subprocess.run([fd_binary, str(huber), str(case)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    m = re.search(r"inputs (\d+) nonzero (\d+) mismatches (\d+) worst (\S+)", res.stdout)
    assert m, res.stdout
    n_in, nonzero, bad = int(m.group(1)), int(m.group(2)), int(m.group(3))
    assert n_in == 395
    assert bad == 0, res.stdout
    # gradients reach the inputs (a border pixel has two neighbours fewer)
    assert nonzero >= (200 if case == 2 else 380), res.stdout
