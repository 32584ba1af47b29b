"""A plain C program (tests/c_abi_client.c) uses the library through the C
ABI alone: the header compiles as C11, the program links against the
in-tree library, and on a GPU its answer matches the oracle's direct solve
(relative error <= 1e-6, FP64 residual <= 1e-8 recomputed by the oracle)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import fsi_inputs as F

from oracle.sparse import BlockOperator, rel_residual

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_client.c")


def _cuda_lib_dirs():
    """Directories holding libcudart next to the nvcc that built the library."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    dirs = [os.path.join(root, "lib64")]
    dirs += [os.path.join(root, "targets", t, "lib") for t in ("x86_64-linux", "sbsa-linux", "aarch64-linux")]
    return [d for d in dirs if os.path.isdir(d)]


def _compile(out_dir):
    from paper_2206_06996_gb300 import build
    lib = build.build()
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(lib)
    rpath = ":".join([libdir] + _cuda_lib_dirs())
    exe = os.path.join(out_dir, "c_abi_client")
    cmd = [gcc, "-std=c11", "-O1", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), SRC,
           "-L", libdir, "-l:" + os.path.basename(lib)]
    for d in _cuda_lib_dirs():
        cmd += ["-L", d]
    cmd += ["-Wl,-rpath," + rpath, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_header_compiles_as_c_and_the_client_links(tmp_path):
    """No GPU needed: compile with -Wall -Wextra -Werror and link."""
    exe = _compile(str(tmp_path))
    assert os.access(exe, os.X_OK)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c_client_solves_like_the_oracle(tmp_path, mini_system, mini_direct, precision):
    exe = _compile(str(tmp_path))
    sysf, xf = str(tmp_path / "system.bin"), str(tmp_path / "x.bin")
    F.save_system(mini_system, sysf)
    r = subprocess.run([exe, sysf, xf, precision], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    words = r.stdout.split()
    assert words[0] == "status" and words[1] == "0"
    assert float(words[words.index("rel_res") + 1]) <= 1e-8
    x = np.fromfile(xf, dtype=np.float64)
    assert x.size == mini_system.n
    op = BlockOperator.from_system(mini_system)
    assert rel_residual(op, x, mini_system.b) <= 1e-8
    assert np.linalg.norm(x - mini_direct) <= 1e-6 * np.linalg.norm(mini_direct)
