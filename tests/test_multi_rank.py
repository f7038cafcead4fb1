"""The N > 1 path on the CPU: world-size-2 gloo ranks (127.0.0.1).

The hot path shards by batch with no exchange, so the only cross-rank steps are the benchmark's:
a barrier around the timed region, the maximum of the per-rank times, and the whole-job value (units
of all ranks over the slowest rank's time).  The reference arm under torchrun prints one line from
rank 0; the other ranks exit 0 without work."""

from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        # rank-dependent timings: rank 0 is slower on the first value, rank 1 on the second
        got = bench.max_over_ranks([10.0 - rank, 3.0 + 2.0 * rank])
        dist.barrier()
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump(got, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        with open(tmp_path / ("rank%d.json" % r)) as f:
            assert json.load(f) == [10.0, 5.0]


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]


def test_whole_job_value_is_weak_scaling():
    import bench
    # each rank runs a replica of the step: N ranks do N times the units in the slowest rank's time
    assert bench.whole_job_value(1e9, 1, 10.0) == pytest.approx(1e11)
    assert bench.whole_job_value(1e9, 4, 10.0) == pytest.approx(4e11)
    assert bench.whole_job_value(1e9, 4, 20.0) == pytest.approx(2e11)


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "parallel_b1_n64_v64_d91"]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["unit"] == "samples/s"
    assert line["config"]["workload"] == "parallel_b1_n64_v64_d91" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0


def test_reference_arm_never_loads_the_library():
    """The reference arm is the FP64 oracle alone: its config and sample counts come from ``oracle``,
    so the process neither imports the package nor maps libradon.so."""
    code = (
        "import sys\n"
        "sys.path.insert(0, %r)\n"
        "import bench\n"
        "sys.argv = ['bench.py', '--impl', 'reference', '--steps', '1', '--warmup', '0',\n"
        "            '--workload', 'parallel_b1_n64_v64_d91']\n"
        "bench.main()\n"
        "maps = open('/proc/self/maps').read()\n"
        "assert 'libradon' not in maps, 'libradon.so mapped'\n"
        "assert 'paper_2009_14788_gb300' not in sys.modules, 'package imported'\n"
        "assert 'liboracle' in maps\n"
        "print('REF_OK')\n"
    ) % ROOT
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=dict(os.environ, OMP_NUM_THREADS="2"),
                         capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    assert "REF_OK" in res.stdout
    line = json.loads([l for l in res.stdout.splitlines() if l.startswith("{")][0])
    assert line["config"]["samples_per_image"] > 0 and line["config"]["det_count"] == 91
