"""The C ABI used from a plain C program (tests/c_abi/rhs_demo.c): the header compiles as C11
with gcc and the program links against libacs.so and the CUDA runtime (CPU); on a GPU the
program runs without Python or PyTorch in its address space and its outputs match the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2306_13002_gb300 import build as acs_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _compile(tmp_path) -> str:
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    lib = acs_build.build()
    exe = str(tmp_path / "rhs_demo")
    cmd = ["gcc", "-std=c11", "-O1", "-Wall", "-Werror", os.path.join(ROOT, "tests", "c_abi", "rhs_demo.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           "-L", os.path.dirname(lib), "-lacs", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           "-Wl,-rpath," + os.path.dirname(lib), "-Wl,-rpath," + os.path.join(CUDA, "lib64"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_compiles_and_links(tmp_path):
    _compile(tmp_path)


@pytest.mark.gpu
def test_c_program_matches_oracle(tmp_path):
    import oracle
    from paper_2306_13002_gb300 import inputs
    from _parity import assert_parity
    exe = _compile(tmp_path)
    nx, ny, nz = 37, 21, 19
    U = inputs.rhs_field(nx, ny, nz, halo=2, seed=6800)
    np.ascontiguousarray(U, dtype="<f8").tofile(tmp_path / "u.bin")
    r = subprocess.run([exe, str(nx), str(ny), str(nz), str(tmp_path / "u.bin"), str(tmp_path / "sat.bin"),
                        str(tmp_path / "plain.bin")], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ok" in r.stdout
    ref = oracle.rhs(U)
    for name in ("sat", "plain"):
        out = np.fromfile(tmp_path / f"{name}.bin", dtype="<f8").reshape(5, nz, ny, nx)
        assert_parity(out, ref, what=f"C program, {name}")
