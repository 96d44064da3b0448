"""The multi-rank path of one frame (paper_1809_06132_gb300.shard) run by two
processes that share one GPU and exchange the plane-range records over
gloo (which stages the buffers through host memory; no kernel of one
process waits on the other's).  Each rank sweeps its plane ranges, the
records are all-gathered, both ranks merge them and fuse into their hash
part of the map: both depth maps must equal one process's psweep_depth
bit for bit, and the two parts together must be one process's map."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_FRAMES = 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    import scenes
    return scenes.street(0, n_frames=N_FRAMES, scale=0.25)


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import scenes
    import paper_1809_06132_gb300 as P
    from paper_1809_06132_gb300.shard import ShardedFrame
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        wl = _workload()
        src = scenes.FrameSource(wl)
        sw = P.Sweep(wl.rig, wl.levels, filters=scenes.Filters())
        T = P.Tsdf(wl.tsdf, wl.rig.ref)
        frame = ShardedFrame(sw, T)
        depths = []
        for f in range(N_FRAMES):
            imgs, _ = src.frame(f)
            dev = [torch.from_numpy(i.numpy()).cuda() for i in imgs]
            d = frame.step(dev, boxes=wl.boxes[f], world_to_ref=wl.world_to_ref[f], local_center=wl.local_center(f))
            depths.append(d.cpu().numpy())
        k, D, W = T.extract()
        out.put((rank, frame.ranges[rank], depths, k.cpu().numpy(), D.cpu().numpy(), W.cpu().numpy(),
                 T.sync_status(), sw.sync_status()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_on_one_gpu_match_one_process():
    import scenes
    import paper_1809_06132_gb300 as P
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=240) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # one process, the whole frame
    wl = _workload()
    src = scenes.FrameSource(wl)
    sw = P.Sweep(wl.rig, wl.levels, filters=scenes.Filters())
    T = P.Tsdf(wl.tsdf, wl.rig.ref)
    ref = []
    for f in range(N_FRAMES):
        imgs, _ = src.frame(f)
        d = sw.depth([torch.from_numpy(i.numpy()).cuda() for i in imgs], boxes=wl.boxes[f])
        T.integrate(d, wl.world_to_ref[f], wl.local_center(f))
        ref.append(d.cpu().numpy())
    k, D, W = (x.cpu().numpy() for x in T.extract())
    whole = {tuple(key): i for i, key in enumerate(k.tolist())}
    (r0, rng0, dep0, k0, D0, W0, ts0, ss0), (r1, rng1, dep1, k1, D1, W1, ts1, ss1) = res
    assert rng0[1] == rng1[0] and rng0[0] == [0] * len(rng0[0])      # consecutive plane ranges
    assert (ts0, ss0, ts1, ss1) == (P.PS_OK,) * 4
    for f in range(N_FRAMES):
        assert np.array_equal(dep0[f], ref[f]) and np.array_equal(dep1[f], ref[f]), f
    keys0 = [tuple(x) for x in k0.tolist()]
    keys1 = [tuple(x) for x in k1.tolist()]
    assert not set(keys0) & set(keys1)                              # disjoint hash parts
    assert set(keys0) | set(keys1) == set(whole)                    # together: the whole map
    for keys, Dp, Wp in ((keys0, D0, W0), (keys1, D1, W1)):
        for i, key in enumerate(keys):
            j = whole[key]
            assert np.array_equal(Dp[i], D[j]) and np.array_equal(Wp[i], W[j])
    assert len(keys0) > 50 and len(keys1) > 50
