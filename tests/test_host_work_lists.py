"""Host logic of the GPU variants, compiled here with the host compiler and
checked without a GPU:
  - the tensor-core sweeps' work lists (csrc/sweep_schedule.h: which CTA sums
    which K-blocks of which tile into which partial slot, and which slots each
    tile's leaf adds), for every tile count 1..200 and several larger ones,
    by tests/sweep_schedule_check.cpp;
  - the needed residual's gathered layout and job lists
    (csrc/gathered_layout.h: index order, block coverage, K trimming that
    drops no term, workspace bounds), for seeded sign patterns of many sizes,
    by tests/gathered_layout_check.cpp;
  - the Parlett-Sylvester reorder's rounds of Givens swaps
    (csrc/reorder_schedule.h: a stable partition by sign in the minimum
    number of swaps, disjoint pairs of the round's parity), by
    tests/reorder_schedule_check.cpp;
  - the batched path's per-level task tables (csrc/batched_plan.h: every
    tile's block sums once, slots disjoint) and its workspace bound, which
    must hold for every subset of a batch's matrices, by
    tests/batched_plan_check.cpp."""
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


def _compile_and_run(tmp_path, source, args=()):
    exe = str(tmp_path / os.path.splitext(source)[0])
    inc = ["-I", CSRC] + (["-I", _cuda_include()] if _cuda_include() else [])
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall"] + inc + [os.path.join(ROOT, "tests", source), "-o", exe],
                   check=True)
    out = subprocess.run([exe] + list(args), capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-3000:]
    assert out.stdout.startswith("ok ")


@pytest.mark.skipif(shutil.which("g++") is None or _cuda_include() is None, reason="needs g++ and the CUDA headers")
def test_sweep_work_lists(tmp_path):
    # tile counts 1..200, the n = 16384 headline (256 tiles) and larger ones
    # up to n = 33280
    _compile_and_run(tmp_path, "sweep_schedule_check.cpp", ["200", "256", "257", "383", "512", "520"])


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_gathered_layout_and_residual_jobs(tmp_path):
    _compile_and_run(tmp_path, "gathered_layout_check.cpp")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_reorder_rounds(tmp_path):
    _compile_and_run(tmp_path, "reorder_schedule_check.cpp")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_batched_plan_and_workspace_bound(tmp_path):
    _compile_and_run(tmp_path, "batched_plan_check.cpp")
