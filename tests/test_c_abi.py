"""The C ABI from a plain C99 program, with no Python or PyTorch in the process (tests/c/abi_parity.c):
the header compiles as strict C99, the library links and answers from C, and on a GPU its joint
histograms and MI agree with the CPU oracle's."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "abi_parity.c")


@pytest.fixture(scope="module")
def abi_parity(tmp_path_factory):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    import oracle
    from paper_1909_10690_gb300 import _lib

    libdir = os.path.dirname(_lib.build())
    oradir = os.path.dirname(oracle.build())
    exe = str(tmp_path_factory.mktemp("c_abi") / "abi_parity")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O2", "-I", os.path.join(ROOT, "include"),
           SRC, "-o", exe, "-L", libdir, "-lmi_gb300", "-L", oradir, "-lmi_oracle", "-lm",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{oradir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_host_calls(abi_parity):
    r = subprocess.run([abi_parity, "host"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr


@pytest.mark.gpu
def test_c_program_histograms_and_mi_against_the_oracle(abi_parity, cuda_lib):
    r = subprocess.run([abi_parity, "gpu"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
