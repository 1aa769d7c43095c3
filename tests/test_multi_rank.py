"""The N > 1 path of bench.py on CPU (gloo, world size 2).

The update does not shard: N GPUs run N independent replicas (own seed each,
no data-path collective), and the only exchange is the maximum of the step
times over ranks, which these tests check with two gloo ranks.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

from _mp_workers import job_time_worker

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_job_time_is_the_max_over_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=job_time_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    rows = [open(tmp_path / ("rank%d.txt" % r)).read().split() for r in range(2)]
    ms = [float(r[0]) for r in rows]
    job = [float(r[1]) for r in rows]
    seeds = [int(r[2]) for r in rows]
    assert job[0] == job[1] == max(ms)
    assert seeds[0] != seeds[1]  # replicas run different volumes


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), dict(workload="box_room", seed=1, steps=1, warmup=3))()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_cpu_baseline_reports_all_cores_and_one_thread():
    # the oracle timed as it stands, on the small room workload: all host
    # cores on whole updates, then one thread on a probe sample
    pytest.importorskip("numpy")
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    from paper_2301_05125_gb300 import scenegen as S

    w = S.box_room(1)
    args = type("A", (), dict(sampler=False, alpha=1.0, cpu_budget=2.0))()
    rays = w.n_probes * w.volume["rays_avg"]
    line = bench._cpu_baseline_line(w, rays, args)
    assert line["kind"] == "oracle" and line["unit"] == "rays/s" and line["value"] > 0
    assert line["cores"] == (os.cpu_count() or 1)
    one = line["single_thread"]
    assert one["cores"] == 1 and one["value"] > 0 and "one thread" in one["sample"]
