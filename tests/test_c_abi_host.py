"""The C ABI from plain C: tests/c_abi_host.c is compiled as strict C99
against include/align.h, linked with the library and run (host-only calls,
no GPU)."""
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2310_17864_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_program_uses_the_abi():
    lib = build.build()
    libdir = os.path.dirname(lib)
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "c_abi_host")
        subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                               "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi_host.c"),
                               "-L" + libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "0 failed" in out.stdout
