"""Host logic of the mixed variants' tensor-core sweeps: the work lists of
csrc/sweep_schedule.h (which CTA sums which K-blocks of which tile, into
which partial slot, and which slots each tile's leaf adds) checked for every
tile count 1..200 and several larger ones by tests/sweep_schedule_check.cpp,
compiled here with the host compiler (no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1607_06303_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "vector_types.h")):
            return os.path.join(d, "include")
    return None


@pytest.mark.skipif(shutil.which("g++") is None or _cuda_include() is None, reason="needs g++ and the CUDA headers")
def test_sweep_work_lists(tmp_path):
    exe = str(tmp_path / "sweep_schedule_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-I", CSRC, "-I", _cuda_include(),
                    os.path.join(ROOT, "tests", "sweep_schedule_check.cpp"), "-o", exe], check=True)
    # tile counts 1..200, the 16384 headline (256 tiles) and larger ones up
    # to n = 33280
    out = subprocess.run([exe, "200", "256", "257", "383", "512", "520"], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-3000:]
    assert out.stdout.startswith("ok ")
