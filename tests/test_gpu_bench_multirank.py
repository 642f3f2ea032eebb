"""The bench's multi-rank path end to end: two torchrun ranks (weak scaling),
here sharing the one GPU with host-side gloo collectives (their kernels never
wait on one another), print exactly one line, from rank 0, whose value counts
both ranks' pairs over the slowest rank's time."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_two_ranks_one_line_with_both_ranks_work():
    env = dict(os.environ, GEM_BENCH_BACKEND="gloo")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", "29517", "bench.py", "--gpus", "2", "--steps", "2",
           "--warmup", "3", "--workload", "small", "--no-extras", "--no-cpu-baseline"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["scaling"] == "weak"
    B, n_sets = d["config"]["queries"], d["config"]["n_sets"]
    assert abs(d["value"] - 2 * B * n_sets / (d["ms_per_step"] * 1e-3)) <= 1e-6 * d["value"]
