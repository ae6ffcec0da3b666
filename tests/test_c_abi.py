"""The C ABI used from C alone: tests/c_abi_example.c includes only amr.h and
links only libamr.so.  It compiles and links here; on a GPU it renders a
uniform complete tree and checks the closed form (column 1, 8 leaves)."""
import os
import subprocess

import pytest

from paper_1210_8014_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_example():
    lib = _build.build_amr()
    exe = lib.parent / "c_abi_example"
    cmd = ["gcc", "-std=c11", "-O1", "-Wall", "-Wextra", "-Werror", os.path.join(ROOT, "tests", "c_abi_example.c"),
           "-I", os.path.join(ROOT, "include"), "-L", str(lib.parent), "-lamr", f"-Wl,-rpath,{lib.parent}", "-lm",
           "-o", str(exe)]
    out = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    assert out.returncode == 0, out.stdout
    return exe


def test_c_example_compiles_and_links():
    assert build_example().exists()


@pytest.mark.gpu
def test_c_example_renders_the_closed_form():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    exe = build_example()
    out = subprocess.run([str(exe)], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=300)
    assert out.returncode == 0 and "c abi ok" in out.stdout, out.stdout
