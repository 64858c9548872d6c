"""The C ABI end to end from a plain C program (no Python on the path): host
buffers in, one alignment, host buffers out, bit for bit against the oracle."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2310_17864_gb300 import build, synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_program_aligns_like_the_oracle():
    lib = build.build()
    libdir = os.path.dirname(lib)
    u = synth.make_utterance(2024, 700, 32, 160, repeat_frac=0.1)
    lp = np.ascontiguousarray(u.lp.numpy(), dtype=np.float32)
    tg = np.asarray(u.targets, dtype=np.int32)
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "c_abi_gpu")
        subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-O1",
                               "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi_gpu.c"),
                               "-L" + libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir, "-o", exe])
        lp.tofile(os.path.join(d, "lp.bin"))
        tg.tofile(os.path.join(d, "tg.bin"))
        with open(os.path.join(d, "dims.txt"), "w") as f:
            f.write(f"{lp.shape[0]} {lp.shape[1]} {tg.size}\n")
        run = subprocess.run([exe, d], capture_output=True, text=True, timeout=120)
        assert run.returncode == 0, run.stdout + run.stderr
        path = np.fromfile(os.path.join(d, "path.bin"), dtype=np.int32)
        scores = np.fromfile(os.path.join(d, "scores.bin"), dtype=np.float32)
        total = np.fromfile(os.path.join(d, "total.bin"), dtype=np.float32)[0]
    o = oracle.viterbi_f32(lp, tg, 0)
    assert o["status"] == 0
    assert np.array_equal(path, o["path"])
    assert scores.tobytes() == o["scores"].tobytes()
    assert np.float32(total).tobytes() == np.float32(o["total"]).tobytes()
