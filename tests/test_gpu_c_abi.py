"""The C ABI used from plain C: tests/c/jz_abi_example.c is compiled with the host C compiler
against include/jz.h, linked to the in-tree libjz.so and run (free-stream preservation and
conservation on a curvilinear periodic box, both precision forms)."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program(tmp_path):
    from paper_2003_08746_gb300 import build
    lib = build.build()
    exe = tmp_path / "jz_abi_example"
    libdir = os.path.dirname(lib)
    cudalib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    subprocess.run(["gcc", "-O2", "-std=c99", "-Wall", "-Werror", os.path.join(ROOT, "tests", "c", "jz_abi_example.c"),
                    "-I", os.path.join(ROOT, "include"), "-L", libdir, "-ljz", f"-Wl,-rpath,{libdir}",
                    f"-Wl,-rpath,{cudalib}", "-lm", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout, r.stderr)
    assert r.returncode == 0
    assert "C ABI example OK" in r.stdout
