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


def slab_worker(rank, world, port, out_dir, frames):
    """One rank of the probe-slab split with the oracle as its engine; its
    probes' results per frame and the final atlases go to an .npz file."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    for d in (root, here):
        if d not in sys.path:
            sys.path.insert(0, d)
    import numpy as np
    import torch.distributed as dist

    from _slab_oracle import OracleSlabRank, rank_record
    from paper_2301_05125_gb300 import scenegen as S
    from paper_2301_05125_gb300.slab import DistExchange, SlabPart, slab_ranges, slab_update

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = S.small_city(4, n_boxes=800, dims=(9, 5, 7), rays_avg=40)
    ranges = slab_ranges(w.volume["dims"], world)
    part = SlabPart(OracleSlabRank(w), rank, ranges[rank])
    ex = DistExchange(w.volume["dims"], ranges)
    out = {}
    for f in range(frames):
        slab_update([part], ex, f)
        for k, v in rank_record(part.backend, part.rng).items():
            out["f%d_%s" % (f, k)] = v
    ov = part.backend.ov
    for k, v in (("irr", ov.irr()), ("irr_n", ov.irr_n()), ("dep", ov.dep()), ("dep_n", ov.dep_n())):
        out["final_" + k] = v
    np.savez(os.path.join(out_dir, "slab_rank%d.npz" % rank), **out)
    dist.barrier()
    dist.destroy_process_group()
