"""End to end: one frame from host memory through psweep_frame_host equals
the device-resident path, and a multi-frame street run keeps both the depth
and the map consistent with the oracle where they are checked."""
import numpy as np
import pytest
import torch

import oracle
import scenes
from tests.parity import TSDF_ABS, tsdf_compare

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1809_06132_gb300 as P  # noqa: E402


def test_frame_host_matches_device_path():
    wl = scenes.street(1, n_frames=2, scale=0.25)
    src = scenes.FrameSource(wl)
    sw = P.Sweep(wl.rig, wl.levels)
    T1 = P.Tsdf(wl.tsdf, wl.rig.ref)
    T2 = P.Tsdf(wl.tsdf, wl.rig.ref)
    for f in range(2):
        imgs, _ = src.frame(f)
        imgs = [i.numpy() for i in imgs]
        host = [torch.from_numpy(i).pin_memory() for i in imgs]
        out = torch.empty((wl.rig.ref.height, wl.rig.ref.width), dtype=torch.float32).pin_memory()
        sw.frame_host(host, boxes=wl.boxes[f], tsdf=T1, world_to_ref=wl.world_to_ref[f],
                      local_center=wl.local_center(f), depth_out=out)
        dev = sw.depth([torch.from_numpy(i).cuda() for i in imgs], boxes=wl.boxes[f])
        T2.integrate(dev, wl.world_to_ref[f], wl.local_center(f))
        torch.cuda.synchronize()
        assert torch.equal(out, dev.cpu())
    k1, D1, W1 = T1.extract()
    k2, D2, W2 = T2.extract()
    o1 = {tuple(k): i for i, k in enumerate(k1.cpu().numpy().tolist())}
    o2 = {tuple(k): i for i, k in enumerate(k2.cpu().numpy().tolist())}
    assert set(o1) == set(o2)
    i1 = [o1[k] for k in sorted(o1)]
    i2 = [o2[k] for k in sorted(o2)]
    assert torch.equal(D1[i1], D2[i2]) and torch.equal(W1[i1], W2[i2])


def test_oracle_depth_fused_like_oracle():
    # both sides fuse the oracle's own depth maps of a swept frame (the same
    # float32 input), through the dense grid of the tiny workload
    wl = scenes.tiny(2, n_frames=2)
    src = scenes.FrameSource(wl)
    T = P.Tsdf(wl.tsdf, wl.rig.ref)
    O = oracle.Tsdf(wl.tsdf)
    for f in range(2):
        imgs, _ = src.frame(f)
        d = oracle.depth_frame(wl, [i.numpy() for i in imgs])["depth"].astype(np.float32)
        T.integrate(torch.from_numpy(d).cuda(), wl.world_to_ref[f])
        O.integrate(d, wl.rig.ref, wl.world_to_ref[f])
    k, D, W = T.extract()
    ok, oD, oW, oamb = O.dump()
    s = tsdf_compare(ok, oD, oW, oamb, k.cpu().numpy(), D.cpu().numpy(), W.cpu().numpy())
    assert s["n_updated"] > 1000
    assert s["D_abs_max"] <= TSDF_ABS and s["W_mismatch"] == 0, s


def _sorted_map(T):
    k, D, W = T.extract()
    k, D, W = k.cpu().numpy(), D.cpu().numpy(), W.cpu().numpy()
    o = np.lexsort((k[:, 2], k[:, 1], k[:, 0]))
    return k[o], D[o], W[o]


def test_tsdf_fusion_is_deterministic():
    # every voxel is updated by one thread: two maps fed the same frames are bit-identical
    wl = scenes.street(2, n_frames=4, scale=0.25)
    src = scenes.FrameSource(wl, device="cuda")
    A, B = P.Tsdf(wl.tsdf, wl.rig.ref), P.Tsdf(wl.tsdf, wl.rig.ref)
    for f in range(4):
        _, rng = src.frame(f, with_range=True)
        d = torch.from_numpy(rng.numpy().astype(np.float32)).cuda()
        for T in (A, B):
            T.integrate(d, wl.world_to_ref[f], wl.local_center(f))
    a, b = _sorted_map(A), _sorted_map(B)
    assert len(a[0]) > 100
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_hundred_frame_street_trajectory():
    # the whole path over the 100-frame trajectory: estimated depth against the
    # renderer's true range, fusion status and the local-map-bounded block count
    wl = scenes.street(0, n_frames=100, scale=0.25)
    src = scenes.FrameSource(wl, device="cuda")
    sw = P.Sweep(wl.rig, wl.levels, filters=scenes.Filters())
    T = P.Tsdf(wl.tsdf, wl.rig.ref)
    rels, counts = [], []
    for f in range(100):
        imgs, rng = src.frame(f, with_range=True)
        dev = [torch.from_numpy(i.numpy()).cuda() for i in imgs]
        depth = sw.depth(dev, boxes=wl.boxes[f])
        T.integrate(depth, wl.world_to_ref[f], wl.local_center(f))
        if f % 10 == 9:
            d = depth.cpu().numpy()
            gt = rng.numpy()
            v = (d > 0) & (gt > 0)
            assert v.mean() > 0.1, f
            rels.append(float(np.median(np.abs(d[v] - gt[v]) / gt[v])))
            assert T.status() == P.PS_OK, f
            counts.append(T.count())
    print("median relative depth error per 10 frames", [round(r, 4) for r in rels], "blocks", counts)
    assert max(rels) < 0.05
    assert counts == sorted(counts) and 0 < counts[-1] < wl.tsdf.pool_blocks
