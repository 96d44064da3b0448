"""The multi-GPU split of one frame, on one GPU: the sweep's plane ranges
swept one after another (psweep_depth_planes) and merged
(psweep_merge_records) give psweep_depth's outputs bit for bit, and a map
fused as hash parts (tsdf_set_partition) is the whole map block for block
and voxel for voxel.  (One process per GPU and the all-gather between them
are covered on CPU ranks in tests/test_shard.py.)"""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1809_06132_gb300 as P  # noqa: E402
from paper_1809_06132_gb300.shard import split_planes  # noqa: E402


def _dev(imgs):
    return [torch.from_numpy(np.ascontiguousarray(i)).cuda() for i in imgs]


@pytest.fixture(scope="module", params=["street-small", "tiny"])
def frame(request):
    if request.param == "tiny":
        wl = scenes.tiny(0)
    else:
        wl = scenes.street(0, n_frames=1, scale=0.25)
    imgs, _ = scenes.FrameSource(wl).frame(0)
    return wl, _dev([i.numpy() for i in imgs])


def _parts(K, los_per_level):
    return [[los[p] for los in los_per_level] for p in range(len(los_per_level[0]))]


@pytest.mark.parametrize("split", ["one", "halves", "thirds", "uneven", "empty-part", "singles"])
def test_plane_ranges_merge_to_the_whole_sweep(frame, split):
    wl, imgs = frame
    sw = P.Sweep(wl.rig, wl.levels, filters=scenes.Filters() if len(wl.levels) > 1 else None)
    boxes = wl.boxes[0]
    ref_outs = sw.alloc_level_outputs()
    ref = sw.depth(imgs, boxes=boxes, level_outs=ref_outs).clone()
    K = sw.n_planes()
    if split == "one":
        los = [[0] for k in K]
    elif split == "halves":
        los = [[0, k // 2] for k in K]
    elif split == "thirds":
        los = [[r[0][l] for r in split_planes(K, 3)] for l in range(len(K))]
    elif split == "uneven":
        los = [[0, 1, min(k - 1, 37), k - 1] for k in K]
    elif split == "empty-part":
        los = [[0, k // 3, k // 3, k] for k in K]           # parts 1 and 3 hold no plane
    else:
        los = [list(range(0, min(k, 16))) for k in K]        # 16 parts of one plane, then the rest
        los = [l_ + [l_[-1]] * (16 - len(l_)) for l_ in los]
    parts = _parts(K, los)
    recs = []
    for p, lo in enumerate(parts):
        hi = parts[p + 1] if p + 1 < len(parts) else K
        recs.append(sw.depth_planes(imgs, lo, hi))
    outs = sw.alloc_level_outputs()
    got = sw.merge_records(parts, recs, boxes=boxes, level_outs=outs)
    torch.cuda.synchronize()
    assert sw.sync_status() == P.PS_OK
    assert torch.equal(got, ref), split
    for a, b in zip(outs, ref_outs):
        for k in ("depth", "c1", "c2", "kstar"):
            assert torch.equal(a[k], b[k]), (split, k)
    assert (ref > 0).float().mean().item() > 0.1


def test_bad_plane_ranges_are_rejected(frame):
    wl, imgs = frame
    sw = P.Sweep(wl.rig, wl.levels)
    K = sw.n_planes()
    with pytest.raises(P.PsError) as e:
        sw.depth_planes(imgs, [k // 2 for k in K], [k // 4 for k in K])
    assert e.value.status == P.PS_ERR_ARG
    recs = [sw.depth_planes(imgs, [0] * len(K), K)]
    with pytest.raises(P.PsError):
        sw.merge_records([[1] * len(K)], recs)               # the first part must start at plane 0


def test_hash_parts_fuse_to_the_whole_map():
    wl = scenes.street(0, n_frames=4, scale=0.25)
    src = scenes.FrameSource(wl)
    depths = []
    for f in range(4):
        _, rng = src.frame(f, with_range=True)
        depths.append(torch.from_numpy(rng.numpy().astype(np.float32)).cuda())
    G = 3
    maps = [P.Tsdf(wl.tsdf, wl.rig.ref) for _ in range(G + 1)]
    for g in range(G):
        maps[g].set_partition(G, g)
    for f in range(4):
        for T in maps:
            T.integrate(depths[f], wl.world_to_ref[f], wl.local_center(f))
    whole = maps[G].extract()
    wk = whole[0].cpu().numpy()
    ref = {tuple(k): i for i, k in enumerate(wk.tolist())}
    seen = set()
    for g in range(G):
        assert maps[g].sync_status() == P.PS_OK
        k, D, W = (x.cpu().numpy() for x in maps[g].extract())
        assert len(k) > 50
        for i, key in enumerate(map(tuple, k.tolist())):
            assert key not in seen
            seen.add(key)
            j = ref[key]
            assert np.array_equal(D[i], whole[1][j].cpu().numpy()) and np.array_equal(W[i], whole[2][j].cpu().numpy())
    assert seen == set(ref)
    with pytest.raises(P.PsError):
        maps[0].set_partition(2, 2)
    dense = P.Tsdf(scenes.tiny(0).tsdf, scenes.tiny(0).rig.ref)
    with pytest.raises(P.PsError):
        dense.set_partition(2, 0)
