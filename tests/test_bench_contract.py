"""bench.py's output line, checked without a GPU: the keys and types of the
JSON line that the benchmark contract fixes (value, e2e, roofline, clocks,
launch count, ...), for the tensor-core step, the batched workload and the
reference arm.

The GPU steps run against stand-ins for the CUDA calls and for the library
binding that do no computation at all, so only the line's shape is under
test: the single-problem step runs without its CPU-baseline leg, and the
batched workload's leg times the oracle and compares outputs the stand-ins
never wrote (the parity figure it reports here means nothing).  The
reference arm runs the oracle, as it does on the GPU machine, on a small
window."""
import json
import os
import sys
import time
import types

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _Event:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3


@pytest.fixture
def no_gpu_step(monkeypatch):
    import torch

    import paper_1607_06303_gb300 as st
    from paper_1607_06303_gb300 import signtri as sm

    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    real_to_device = st.to_device
    monkeypatch.setattr(st, "to_device", lambda T: real_to_device(T, device="cpu"))
    calls = {"solves": 0}

    def solve(*args):
        calls["solves"] += 1
        return 0

    def solve_batch(ns, *args):
        calls["solves"] += 1
        return 0, [0] * len(ns)

    classes = {sm.KC_BLOCK_SUMS_TC: ("block_sums_tc", 120, 6.0), sm.KC_RESIDUAL: ("residual", 9, 4.0),
               sm.KC_OFFDIAG_LEAF_MIXED: ("offdiag_leaf_mixed", 30, 1.5)}

    def info():
        i = st.Info()
        i.variant = int(st.Variant.PH_MIXED_FP16)
        i.cutoff = 64
        i.refine_steps = 1
        return i

    for name, fn in {
        "load": lambda: None, "sign_tri": solve, "sign_tri_host": solve, "signtri_set_cutoff": lambda b: 0,
        "signtri_probe_fp64_peak": lambda h=None: 1200.0, "signtri_profile_reset": lambda: 0,
        "signtri_profile_enable": lambda on: 0,
        "signtri_profile_read": lambda c: classes[c][1:] if c in classes else (0, 0.0),
        "signtri_profile_read_bytes": lambda c: 5e9 if c == sm.KC_BLOCK_SUMS_TC else 0.0,
        "signtri_profile_read_flops": lambda c: 3e12,
        "signtri_kernel_class_name": lambda c: classes[c][0] if c in classes else "class%d" % c,
        "signtri_get_info": info,
        "signtri_autotune": lambda n_max, h=None: 0,
        "signtri_get_cutoff_table": lambda length=32: [0] * length,
        "signtri_get_variant_table": lambda length=32: [0] * length,
        "signtri_batched_cache_stats": lambda: (2, 1),
        "sign_tri_batched": solve_batch,
    }.items():
        monkeypatch.setattr(st, name, fn)
    return calls


def _last_json(capsys):
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_step_line(no_gpu_step, capsys, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--n", "192", "--steps", "3", "--warmup", "3", "--no-cpu-baseline"])
    assert bench.main() == 0
    line = _last_json(capsys)
    for key, typ in [("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                     ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                     ("dtype", str), ("data", str), ("config", dict), ("gpu_launches", int), ("roofline", dict),
                     ("clocks", dict), ("e2e", dict)]:
        assert isinstance(line[key], typ), key
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] == 3
    assert line["vs_baseline"] is None and line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["gpu_launches"] == 159
    assert "workload" in line["config"] and "l2" in line["config"]
    roof = line["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in roof, key
    assert roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    # the method's work of the 3 timed steps (per step the oracle's useful
    # flops of the initial sweep, 4 C(n,3) for the one correction) over 120
    # launches of 6 ms in all
    import math
    import numpy as np
    from paper_1607_06303_gb300 import workload
    from paper_1607_06303_gb300.inputs import make_T
    useful = workload.useful_flops(np.sign(np.diag(make_T(192, 0.5, seed=0))))
    assert roof["achieved"] == pytest.approx(3 * (useful + 4 * math.comb(192, 3)) / 6e-3 / 1e12)
    # beside it: 5e9 operand bytes over 120 launches of 6 ms in all against the copy bandwidth
    assert roof["hbm_view"]["achieved_gbs"] == pytest.approx(5e9 / 6e-3 / 1e9)
    assert roof["executed_tflops"] == pytest.approx(3e12 / 6e-3 / 1e12)
    assert line["dtype"] == "fp16+f32+f64"
    assert line["roofline_second"]["bound"] == "tensor"
    e2e = line["e2e"]
    assert e2e["unit"] == line["unit"] and e2e["value"] > 0
    # T's upper triangle by 128-column panels (192 columns: 128 x 128 and 64 x 192), all of U back
    assert e2e["h2d_bytes_per_step"] == 8 * (128 * 128 + 64 * 192)
    assert e2e["d2h_bytes_per_step"] == 8 * 192 * 192
    for key in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert key in line["clocks"], key
    assert [c["variant"] for c in line["compare"]] == ["PH_MIXED_TF32", "PH_FP64_EFFICIENT", "PH_FP64"]
    for key in ("wall", "copies", "kernels", "rest"):
        assert key in e2e["one_call_ms"], key
    # warm-up, timed steps, e2e (one warm call + three repetitions + one
    # profiled call for the breakdown), comparisons
    assert no_gpu_step["solves"] == 3 + 3 + 1 + 3 * 3 + 1 + 3 * (1 + 2)


def test_reference_line(capsys, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--n", "256", "--steps", "1",
                                      "--warmup", "0", "--cpu-sample", "96"])
    assert bench.main() == 0
    line = _last_json(capsys)
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config"):
        assert key in line, key
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and "96" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_defaults_meet_the_timing_rules():
    a = bench.parse_args([])
    assert a.warmup >= 3 and a.steps >= 1 and a.gpus == 1 and a.n == 16384


def test_batched_line(no_gpu_step, capsys, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "batched", "--batch", "6", "--steps", "3",
                                      "--warmup", "3"])
    assert bench.main() == 0
    line = _last_json(capsys)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "gpu_launches", "clocks", "cpu_baseline"):
        assert key in line, key
    assert line["steps"] == 3 and line["warmup"] == 3 and no_gpu_step["solves"] == 6
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and line["sample_size"] == 6
    # the oracle-free check is reported on every run (here on outputs the
    # stand-ins never wrote: only its presence and shape are tested)
    assert set(line["probe_residuals"]) >= {"involution_max", "commutation_max"}
    assert line["graph_cache"] == {"hits": 2, "builds": 1}
