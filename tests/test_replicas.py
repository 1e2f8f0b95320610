"""The multi-GPU form is independent replicas: one process per GPU, no data
exchanged, the whole job's time the slowest rank's. The host side of that
(process group, barrier, max over ranks, whole-job throughput) runs here as
two gloo ranks on the CPU."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(None)
    bench.barrier(w)
    # each rank's "time" differs; everyone must see the slowest
    ms = bench.max_over_ranks(w, 100.0 + 10.0 * r)
    out.put((r, w, dist.get_backend(), ms, bench.replica_throughput(1000, 4, w, ms)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_whole_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for r, w, backend, ms, value in got:
        assert w == 2 and backend == "gloo"
        assert ms == 110.0
        # 2 replicas x 1000 cells x 4 steps in 0.110 s
        assert abs(value - 2 * 1000 * 4 / 0.110) < 1e-6


def test_one_rank_is_the_single_gpu_run():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1, 42.0) == 42.0
    assert bench.replica_throughput(4194304, 20, 1, 1000.0) == 4194304 * 20
