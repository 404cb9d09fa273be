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


FAILING_WORKER = r"""
import os, sys, time
sys.path.insert(0, {root!r})
import bench
world, rank, local = bench.dist_setup()
bench.barrier(world)  # both ranks get here
if rank == 1:
    if {mode!r} == "raise":
        raise RuntimeError("replica 1 fails between steps")
    time.sleep(60)  # "stall": never reaches the next barrier in time
t0 = time.time()
try:
    bench.barrier(world)
    print("RESULT no-error", flush=True)
except Exception as e:
    print("RESULT peer-failure %.1f %s" % (time.time() - t0, type(e).__name__), flush=True)
"""


def test_a_failed_replica_ends_the_others_barrier_with_an_error():
    """A replica that raises between steps, or stalls past the process-group
    timeout, does not leave the others waiting forever: rank 0's next
    barrier fails with an error well within the test's limit (failure made
    on the host, as two gloo processes on the CPU)."""
    for mode in ("raise", "stall"):
        port = _free_port()
        procs = []
        for r in range(2):
            env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                       MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="",
                       AUNMF_PG_TIMEOUT_S="5")
            procs.append(subprocess.Popen(
                [sys.executable, "-c", FAILING_WORKER.format(root=ROOT, mode=mode)], env=env,
                stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
        out0, err0 = procs[0].communicate(timeout=120)
        procs[1].kill()
        procs[1].communicate(timeout=30)
        line = [x for x in out0.splitlines() if x.startswith("RESULT")]
        assert line and line[0].startswith("RESULT peer-failure"), (mode, out0, err0[-2000:])
        assert float(line[0].split()[2]) < 60.0
