"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2):
the job's time is each timed value's maximum over the ranks, every rank
runs its own independent sequence (replicas, no data exchange), and the
reference arm runs on rank 0 alone."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        vals = bench.max_over_ranks([1.5 + rank, 10.0 - rank, 3.0])
        out.put((rank, vals, bench.rank_seed(7, rank), bench.dist_env()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_max_over_ranks_and_rank_seeds_with_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, vals, seed, env in res:
        assert vals == [2.5, 10.0, 3.0]          # max over ranks, identical on every rank
        assert seed == 7 + rank
        assert env == (world, rank, rank)
    assert res[0][2] != res[1][2]


def test_single_rank_values_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.0, 2.0]) == [1.0, 2.0]


def test_rank_sequences_are_independent_replicas():
    import scenes
    sys.path.insert(0, ROOT)
    import bench
    a = scenes.street(bench.rank_seed(0, 0), n_frames=2, scale=0.25)
    b = scenes.street(bench.rank_seed(0, 1), n_frames=2, scale=0.25)
    assert repr(a.scene.boxes) != repr(b.scene.boxes)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    import argparse
    ns = argparse.Namespace(gpus=2, steps=1, warmup=0, impl="reference", seed=0, no_cpu_baseline=True,
                            config="street", half=False, batch_size=64)
    assert bench.run_reference(ns) == 0      # rank 1: no work, exit 0


def test_reference_arm_json_line_on_the_tiny_frame():
    # the reference arm (the FP64 oracle on the host cores) prints one JSON
    # line with the keys the bench contract asks for; the tiny frame keeps it
    # to a few seconds of CPU work
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "tiny",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "frames/s" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("tiny-160x128")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["ms_per_step"] > 0
