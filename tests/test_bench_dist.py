"""The bench's multi-rank logic on CPU: two gloo ranks over 127.0.0.1.  Each
rank reports its own time; every rank must see the slowest one, the
whole-job value is the units of all ranks over that time, and only rank 0
runs the reference arm."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import argparse
    import bench
    w, r, local = bench._dist()
    t_max = bench.max_over_ranks(10.0 + 5.0 * r, w, "cpu")
    value = bench.whole_job_value(1000.0, 4, w, t_max)
    ref = bench._reference_arm(argparse.Namespace(steps=1, warmup=0)) if r != 0 else "skipped"
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, t_max, value, ref))


def test_two_gloo_ranks_aggregate_like_the_bench():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    assert all(o[3] == 15.0 for o in out)                       # the slowest rank's time on every rank
    assert all(abs(o[4] - 1000.0 * 4 * 2 / 0.015) < 1e-6 * o[4] for o in out)
    assert out[1][5] is None                                    # rank 1 runs no reference work


def test_traffic_lookup_scales_and_checks_the_source_hash(tmp_path, monkeypatch):
    """The DRAM traffic and counters of a capture are scaled to a launch by its
    pixel-samples and reported while the tile kernels' sources hash to the
    captured ones; withheld (null) once they differ."""
    import importlib.util
    import json
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    B = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(B)
    fake = tmp_path / "repo"
    (fake / "profiles").mkdir(parents=True)
    (fake / "paper_2603_27151_gb300" / "csrc").mkdir(parents=True)
    for n in B.TILE_KERNEL_SOURCES:
        src = open(os.path.join(root, "paper_2603_27151_gb300", "csrc", n), "rb").read()
        (fake / "paper_2603_27151_gb300" / "csrc" / n).write_bytes(src)
    monkeypatch.setattr(B, "ROOT", str(fake))
    d = {"source_sha1": B._source_sha1(), "pixel_samples": 1000, "bytes": {"raster_bwd": 5000},
         "counters": {"raster_bwd": {"issue_active": 0.5}}, "profile": "profiles/x.md"}
    (fake / "profiles" / "dram_traffic.json").write_text(json.dumps(d))
    assert B._traffic("raster_bwd", 2000) == 10000
    assert B._traffic("no_such_kernel", 1) is None
    assert B._counters("raster_bwd") == {"issue_active": 0.5, "source": "profiles/x.md"}
    # a tile kernel changed after the capture: no traffic, no counters
    p = fake / "paper_2603_27151_gb300" / "csrc" / "ds_raster.cu"
    p.write_bytes(p.read_bytes() + b"// changed\n")
    assert B._traffic("raster_bwd", 1000) is None and B._counters("raster_bwd") is None
