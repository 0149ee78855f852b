"""The N > 1 path of bench.py on the CPU: two ranks over gloo.

Under torchrun every rank solves its own map (independent replicas, no collective on
the data path); the only exchange is the host-side reduction of the step times, whose
maximum over the ranks is the job's time, and the whole-job value counts every rank's
pixels.  These tests run that reduction with two gloo ranks on 127.0.0.1, and check
that the reference arm's other ranks exit without work or output.
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, sys
sys.path.insert(0, {root!r})
import bench
rank, world, local, dist = bench.init_ranks("gloo")
# rank r reports step times (ms, plain ms, e2e ms) that differ per rank and per slot
mine = [[10.0, 40.0, 12.0], [11.5, 38.0, 12.5]][rank]
ms, ms_plain, ms_e2e = bench.max_over_ranks(mine, dist)
dist.barrier()
print(json.dumps({{"rank": rank, "world": world, "local": local, "max": [ms, ms_plain, ms_e2e],
                  "value": bench.job_throughput(2048 * 2048, world, ms)}}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ)
    env.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "CUDA_VISIBLE_DEVICES": ""})
    return env


def _run_ranks(cmds, world, timeout=120):
    port = _free_port()
    procs = [subprocess.Popen(cmds(r), env=_env(r, world, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, cwd=ROOT) for r in range(world)]
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=timeout)
            outs.append((p.returncode, out, err))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
                p.wait()
    return outs


def test_step_time_is_the_max_over_two_gloo_ranks():
    script = RANK_SCRIPT.format(root=ROOT)
    outs = _run_ranks(lambda r: [sys.executable, "-c", script], 2)
    lines = []
    for rc, out, err in outs:
        assert rc == 0, err
        lines.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(l["rank"] for l in lines) == [0, 1]
    for l in lines:
        assert l["world"] == 2 and l["local"] == l["rank"]
        # every rank receives the slowest rank's time, slot by slot
        assert l["max"] == [11.5, 40.0, 12.5]
        # both maps counted over the slowest rank's step: 2 x 4194304 px / 11.5 ms
        assert abs(l["value"] - 2 * 2048 * 2048 / 11.5e3) < 1e-9


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    rank, world, local, dist = bench.init_ranks("gloo")
    assert (rank, world, local, dist) == (0, 1, 0, None)
    assert bench.max_over_ranks([3.0, 1.0]) == [3.0, 1.0]
    assert bench.job_throughput(1000, 1, 2.0) == 1000 / 2e3


def test_reference_arm_other_ranks_exit_without_output():
    # rank 1 of a two-rank reference run returns before any work; rank 0 alone would
    # time the oracle, so only rank 1 is started here
    port = _free_port()
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "3"], env=_env(1, 2, port), cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
