"""Edge cases of the sweep through the C ABI: the largest rig (4 matching
cameras, 9x9 windows: the most shared memory per CTA) against the oracle,
the full 64-sweep batch mix against single calls, featureless images, a
single plane, and images barely larger than the window."""
import dataclasses
import os

import numpy as np
import pytest
import torch

import oracle
import scenes
from scenes.configs import DOWNSAMPLE, FRONTO, Level, PlaneSet, Rig
from tests.parity import assert_sweep_parity

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1809_06132_gb300 as P  # noqa: E402


def _dev(imgs):
    return [torch.from_numpy(np.ascontiguousarray(i)).cuda() for i in imgs]


def test_four_cameras_nine_by_nine_against_the_oracle():
    wls = scenes.batch_mix(11, n=40, sizes=((640, 512),), planes=(64,), max_cams=4)
    wl = next(w for w in wls if len(w.rig.cams) == 4)
    wl.levels = [dataclasses.replace(wl.levels[0], window=9)]
    imgs, _ = scenes.FrameSource(wl, device="cuda").frame(0)
    imgs = [i.numpy() for i in imgs]
    sw = P.Sweep(wl.rig, wl.levels)
    outs = sw.alloc_level_outputs()
    sw.depth(_dev(imgs), level_outs=outs)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in outs[0].items()}
    rng = np.random.default_rng(3)
    flat = rng.choice(632 * 504, 20000, replace=False)
    pix = np.stack([4 + flat % 632, 4 + flat // 632], axis=1).astype(np.int32)
    oracle.set_threads(os.cpu_count() or 1)
    o = oracle.sweep_level(wl.rig, wl.levels[0], imgs, pix=pix)
    s = assert_sweep_parity(o, {k: v[pix[:, 1], pix[:, 0]] for k, v in g.items()}, min_gated=5000,
                            src=(wl.rig, wl.levels[0], imgs, pix))
    print("4 cameras, 9x9", s)


def test_full_batch_mix_equals_single_calls():
    wls = scenes.batch_mix(0, n=64)
    sweeps, images, boxes = [], [], []
    for wl in wls:
        imgs, _ = scenes.FrameSource(wl, device="cuda").frame(0)
        images.append(_dev([i.numpy() for i in imgs]))
        sweeps.append(P.Sweep(wl.rig, wl.levels))
        boxes.append(wl.boxes[0])
    single = [sw.depth(im, boxes=bx).clone() for sw, im, bx in zip(sweeps, images, boxes)]
    outs = P.Batch(sweeps, use_graph=False).run(images, boxes=boxes)
    torch.cuda.synchronize()
    for i, (o, s) in enumerate(zip(outs, single)):
        assert torch.equal(o, s), f"sweep {i} ({wls[i].name})"


def test_featureless_images_give_no_depth():
    wl = scenes.tiny(0)
    flat = [np.full((wl.rig.ref.height, wl.rig.ref.width), 128, np.uint8) for _ in range(2)]
    sw = P.Sweep(wl.rig, wl.levels)
    outs = sw.alloc_level_outputs()
    d = sw.depth(_dev(flat), level_outs=outs)
    torch.cuda.synchronize()
    assert (d == 0).all() and (outs[0]["kstar"] == -1).all()
    assert torch.isinf(outs[0]["c1"]).all()


def test_single_plane_and_tiny_images():
    wl = scenes.tiny(1)
    imgs, _ = scenes.FrameSource(wl).frame(0)
    imgs = [i.numpy() for i in imgs]
    # one plane: every valid pixel picks it, no parabola (a set end)
    lv = Level(kind=DOWNSAMPLE, factor=1, window=5, sets=[PlaneSet(FRONTO, 1, 3.0, 3.0)])
    sw = P.Sweep(wl.rig, [lv])
    outs = sw.alloc_level_outputs()
    sw.depth(_dev(imgs), level_outs=outs)
    o = oracle.sweep_level(wl.rig, lv, imgs)
    k = outs[0]["kstar"].cpu().numpy()
    assert ((k == 0) == (o["kstar"] == 0)).mean() > 0.999 and (k == 0).mean() > 0.3
    assert (k <= 0).all()
    # images barely larger than the window (7 x 6, 5 x 5 window): a 3 x 2 interior
    cam = dataclasses.replace(wl.rig.ref, width=7, height=6, cx=3.0, cy=2.5)
    rig = Rig(ref=cam, cams=[cam], ref_to_cam=wl.rig.ref_to_cam)
    small = [np.ascontiguousarray(i[60:66, 76:83]) for i in imgs]
    lv2 = Level(kind=DOWNSAMPLE, factor=1, window=5, sets=[PlaneSet(FRONTO, 8, 0.5, 20.0)])
    sw2 = P.Sweep(rig, [lv2])
    outs2 = sw2.alloc_level_outputs()
    d = sw2.depth(_dev(small), level_outs=outs2).cpu().numpy()
    o2 = oracle.sweep_level(rig, lv2, small)
    k2 = outs2[0]["kstar"].cpu().numpy()
    border = np.ones((6, 7), bool)
    border[2:4, 2:5] = False
    assert (d[border] == 0).all() and (k2[border] == -1).all()
    assert np.array_equal(k2 >= 0, o2["kstar"] >= 0)
