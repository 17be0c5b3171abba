"""The C ABI used from plain C: `tests/c_abi_example.c` compiles against
include/mphf.h, links against the in-tree libmphf.so and the CUDA runtime,
and (on a GPU) builds, queries, verifies, serialises and reloads functions
with rotation-fitting and ShockHash leaves."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PKG = os.path.join(ROOT, "paper_2212_09562_b300")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _compile(tmp_path) -> str:
    from paper_2212_09562_b300 import build
    build.build()
    exe = str(tmp_path / "c_abi_example")
    cc = shutil.which("gcc") or "cc"
    subprocess.check_call([
        cc, "-O2", "-std=c11", "-Wall", "-Wextra", os.path.join(HERE, "c_abi_example.c"),
        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
        "-L", PKG, "-lmphf", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
        f"-Wl,-rpath,{PKG}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}", "-o", exe])
    return exe


def test_c_example_compiles_and_links(tmp_path):
    exe = _compile(tmp_path)
    assert os.access(exe, os.X_OK)


@pytest.mark.gpu
def test_c_example_runs(tmp_path):
    exe = _compile(tmp_path)
    r = subprocess.run([exe, "300000"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.strip().splitlines()
    assert lines[-1] == "ok" and sum("bijection=yes" in l for l in lines) == 3, r.stdout
    assert sum("loaded=same" in l for l in lines) == 3, r.stdout


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c", "c11"), ("c++", "c++11"), ("c++", "c++17")])
def test_header_compiles_alone(tmp_path, lang, std):
    """include/mphf.h needs nothing but the C standard headers, in C and C++."""
    cc = shutil.which("gcc") or "cc"
    src = tmp_path / "only_header.c"
    src.write_text('#include "mphf.h"\nint main(void) { mphf_build_params p; (void)p; return 0; }\n')
    subprocess.check_call([cc, "-x", lang, f"-std={std}", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-fsyntax-only", "-I", os.path.join(ROOT, "include"), str(src)])
