"""The flop models bench.py divides by (float64 roofline), checked against a
brute-force count of the block-sum terms (Section 5.3): every (row, k,
column) triple with k in the K-blocks strictly between the row's and the
column's block, 6 flops in the matrix-multiply form, 2 (equal signs, Y only)
or 4 (opposite signs, X only) in the arithmetic-efficient form."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def brute(n, b, signs):
    nb = (n + b - 1) // b
    mm = eff = 0
    for i in range(n):
        for j in range(n):
            I, J = i // b, j // b
            if J < I + 2:
                continue
            k_between = (J - I - 1) * b          # interior K-blocks are full
            mm += 6 * k_between
            eff += (2 if signs[i] == signs[j] else 4) * k_between
    return mm, eff


@pytest.mark.parametrize("n,b", [(1, 16), (40, 16), (64, 16), (97, 16), (130, 32), (200, 64)])
def test_block_sum_flop_models(n, b):
    rng = np.random.default_rng(n * 131 + b)
    signs = np.where(rng.random(n) < 0.4, -1.0, 1.0)
    mm, eff = brute(n, b, signs)
    assert bench.block_sum_flops(n, b) == mm
    assert bench.block_sum_flops_efficient(n, b, signs) == eff


def test_efficient_is_between_third_and_two_thirds_of_mm():
    # all one sign: 2 of the MM form's 6 flops per term; alternating signs: 4 of 6 at most
    n, b = 256, 16
    same = np.ones(n)
    assert 3 * bench.block_sum_flops_efficient(n, b, same) == bench.block_sum_flops(n, b)
    alt = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    e = bench.block_sum_flops_efficient(n, b, alt)
    assert bench.block_sum_flops(n, b) / 3 < e < 2 * bench.block_sum_flops(n, b) / 3 + 1


def _replica_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: a step of 10 + r ms over 1e12 (1 + r) useful flops
        t = bench.reduce_over_ranks(dist, 10.0 + rank, "max", "cpu")
        w = bench.reduce_over_ranks(dist, 1e12 * (1 + rank), "sum", "cpu")
        with open(os.path.join(out_dir, "r%d.txt" % rank), "w") as f:
            f.write("%r %r\n" % (t, w))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks(tmp_path):
    """The N > 1 bench path: the time is the slowest replica's, the work the
    sum of all replicas' (each rank solves its own seeded input)."""
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, w = map(float, (tmp_path / ("r%d.txt" % r)).read_text().split())
        assert t == 11.0 and w == 3e12
    assert bench.reduce_over_ranks(None, 7.5, "max", "cpu") == 7.5


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun only rank 0 times the oracle; the other ranks exit
    without work."""
    assert bench.run_reference(bench.parse_args(["--impl", "reference"]), 1) is None


def _cited_bench_commands():
    """The bench.py argument lists cited by the summaries under profiles/
    (continuation lines joined; commands with placeholders -- [optional]
    parts or shell variables -- skipped)."""
    import glob
    import shlex
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = []
    for path in sorted(glob.glob(os.path.join(root, "profiles", "*.txt"))):
        text = open(path).read().replace("\\\n", " ")
        for line in text.splitlines():
            if "python bench.py" not in line or "[" in line or "$" in line:
                continue
            rest = line.split("python bench.py", 1)[1]
            toks = []
            for t in shlex.split(rest.replace(">", " > ").replace("&&", " && ").replace("|", " | ")):
                if t in (">", "&&", "|", ")") or t.endswith(")"):
                    break
                toks.append(t)
            out.append((os.path.basename(path), toks))
    return out


def test_profile_commands_parse():
    """Every bench command a profile summary cites still parses (no flag it
    uses was renamed or dropped)."""
    cmds = _cited_bench_commands()
    assert len(cmds) >= 10
    for name, toks in cmds:
        try:
            bench.parse_args(toks)
        except SystemExit:
            pytest.fail("%s cites an invalid bench command: %s" % (name, " ".join(toks)))
