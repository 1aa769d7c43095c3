"""Worker functions of the multi-process CPU tests (importable by spawned children)."""
import os
import sys
import time


def job_time_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r = bench._dist()
    assert (ws, r) == (world, rank)
    dist.barrier()
    t0 = time.perf_counter()
    time.sleep(0.05 * (rank + 1))  # ranks finish at different times
    ms = 1e3 * (time.perf_counter() - t0)
    job = bench._job_ms(ms, ws, "cpu")
    dist.barrier()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write("%r %r %d\n" % (ms, job, bench._replica_seed(1, rank)))
    dist.destroy_process_group()
