"""N > 1 runs are independent replicas (the method's data-parallel path has no
exchange on one GPU per problem): the bench's rank setup, barriers and the
max-over-ranks timing, run as two gloo processes on the CPU."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import sys
sys.path.insert(0, {root!r})
import bench
import torch.distributed as dist
world, rank, local = bench.dist_setup()
bench.barrier(world)
t = bench.max_over_ranks(10.0 + 5.0 * rank, world)
bench.barrier(world)
print("RESULT", world, rank, local, t, flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_share_the_slowest_time():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    seen = sorted(line.split()[1:] for o in outs for line in o.splitlines()
                  if line.startswith("RESULT"))
    assert seen == [["2", "0", "0", "15.0"], ["2", "1", "1", "15.0"]]


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    env = {k: os.environ.get(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    try:
        for k in env:
            os.environ.pop(k, None)
        assert bench.dist_setup() == (1, 0, 0)
        assert bench.max_over_ranks(3.5, 1) == 3.5
        bench.barrier(1)
    finally:
        for k, v in env.items():
            if v is not None:
                os.environ[k] = v
