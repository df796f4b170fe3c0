"""The C ABI from a plain C program (tests/c/abi_example.c): it compiles
against include/pm.h alone and, on a GPU, runs the Sec. 2.5 example through
libpm.so."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "c", "abi_example.c")
LIBDIR = os.path.join(ROOT, "paper_1611_06115_gb300")


def _compile(tmp_path, link: bool) -> str:
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    exe = str(tmp_path / ("abi_example" if link else "abi_example.o"))
    cmd = [gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), SRC]
    if link:
        cmd += ["-L", LIBDIR, "-lpm", f"-Wl,-rpath,{LIBDIR}", "-o", exe]
    else:
        cmd += ["-c", "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_c_example_compiles_against_the_header(tmp_path):
    _compile(tmp_path, link=False)


@pytest.mark.gpu
def test_c_example_runs_on_the_gpu(tmp_path):
    if not os.path.exists(os.path.join(LIBDIR, "libpm.so")):
        pytest.fail("libpm.so is not built")
    exe = _compile(tmp_path, link=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "abi_example ok" in r.stdout
