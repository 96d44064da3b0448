"""Precision at scale: the ring workload (reference + 3 matching cameras,
1280x1024, 256 full-resolution planes, 9x9 window) swept with float32 and
with FP16 storage of the matching images (arithmetic stays float32),
both against the FP64 oracle on 40,000 sampled pixels.  The float32 path
meets the parity criteria; the FP16 form's error against the oracle is
reported per result (plane agreement, relative depth percentiles,
validity) and bounded."""
import os

import numpy as np
import pytest
import torch

import oracle
import scenes
from tests.parity import assert_sweep_parity, sweep_stats

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1809_06132_gb300 as P  # noqa: E402

N_SAMPLES = 40000


def _levels(sw, imgs):
    dev = [torch.from_numpy(i).cuda() for i in imgs]
    outs = sw.alloc_level_outputs()
    sw.depth(dev, level_outs=outs)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in outs[0].items()}


def test_ring_fp32_and_fp16_storage():
    wl = scenes.ring(0, n_frames=1000)
    imgs, _ = scenes.FrameSource(wl, device="cuda").frame(3)
    imgs = [i.numpy() for i in imgs]
    g32 = _levels(P.Sweep(wl.rig, wl.levels), imgs)
    g16 = _levels(P.Sweep(wl.rig, wl.levels, image_half=True), imgs)
    lv = wl.levels[0]
    H, W = g32["kstar"].shape
    rho = lv.window // 2
    rng = np.random.default_rng(9)
    flat = rng.choice((H - 2 * rho) * (W - 2 * rho), N_SAMPLES, replace=False)
    pix = np.stack([rho + flat % (W - 2 * rho), rho + flat // (W - 2 * rho)], axis=1).astype(np.int32)
    oracle.set_threads(os.cpu_count() or 1)
    o = oracle.sweep_level(wl.rig, lv, imgs, pix=pix)
    at = lambda g: {k: v[pix[:, 1], pix[:, 0]] for k, v in g.items()}  # noqa: E731
    s32 = assert_sweep_parity(o, at(g32), min_gated=5000, src=(wl.rig, lv, imgs, pix))
    s16 = sweep_stats(o, at(g16))
    # FP16 storage against the float32 form over the whole frame
    v = (g32["kstar"] >= 0) & (g16["kstar"] >= 0)
    same = (g32["kstar"] == g16["kstar"])[v].mean()
    rel = np.abs(g16["depth"][v] - g32["depth"][v]) / g32["depth"][v]
    pct = {q: float(np.percentile(rel, q)) for q in (50, 90, 99, 99.9)}
    print("ring fp32 vs oracle", s32)
    print("ring fp16 vs oracle", s16)
    print("ring fp16 vs fp32 (whole frame)", dict(plane_agree=float(same), rel_depth_pct=pct))
    # FP16 storage rounds every matching intensity by up to 2^-12 (a few
    # percent of one grey level): the winning plane moves on a small share of
    # the gated pixels, and where it stays the depth moves by the sub-plane
    # fit's response to the cost change
    assert s16["index_agree"] >= 0.99, s16
    assert s16["valid_mismatch"] <= 0.002, s16
    assert s16["depth_rel_p90"] <= 1e-3, s16
    assert same >= 0.99 and pct[50] < 1e-4
