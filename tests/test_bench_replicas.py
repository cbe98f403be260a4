"""The multi-process (replica) path of bench.py on CPU: world size 2 over
gloo on 127.0.0.1.  Each rank reports its own step time; the job's time is
the slowest rank's, and the throughput counts the bytes of every rank."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local = [1.5, 4.25][rank]                      # each rank's own step time
    ms = bench.max_over_ranks(local, ws, "cpu")
    gbs = bench.replica_throughput(1e9, ws, ms * 1e-3)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{ms} {gbs}\n")


def test_max_over_ranks_and_whole_job_throughput(tmp_path):
    import torch.multiprocessing as mp
    port = free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    vals = [tuple(map(float, open(tmp_path / f"r{r}.txt").read().split())) for r in range(2)]
    for ms, gbs in vals:
        assert ms == 4.25                           # the slowest rank
        assert gbs == pytest.approx(2 * 1e9 / 4.25e-3 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.replica_throughput(2e9, 1, 0.5) == pytest.approx(4.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "3", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_recorded_traffic_follows_code_not_comments():
    """bench.py reports a recorded DRAM-traffic figure only while the
    library's code is the one it was measured on: comments and layout do
    not count as a change, code does."""
    sys.path.insert(0, ROOT)
    import bench
    a = "int f() { return 1; }  // one\n/* a block\n   comment */\n\n"
    b = "// header\nint f() { return 1; }\n"
    c = "int f() { return 2; }\n"
    assert bench.code_text(a) == bench.code_text(b) == "int f() { return 1; }"
    assert bench.code_text(c) != bench.code_text(a)
