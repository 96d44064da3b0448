"""Precision at scale: the ring workload (reference + 3 matching cameras,
1280x1024, 256 full-resolution planes, 9x9 window) swept with float32 and
with FP16 storage of the matching images (arithmetic stays float32),
against the FP64 oracle on sampled pixels.  The float32 path meets the
parity criteria; the FP16 form's agreement and depth-error percentiles are
reported and bounded."""
import numpy as np
import pytest
import torch

import oracle
import scenes
from tests.parity import sweep_stats

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1809_06132_gb300 as P  # noqa: E402


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
    pix = np.stack([rng.integers(rho, W - rho, 250), rng.integers(rho, H - rho, 250)], axis=1)
    o = oracle.sweep_level(wl.rig, lv, imgs, pix=pix)
    s32 = sweep_stats(o, {k: v[pix[:, 1], pix[:, 0]] for k, v in g32.items()})
    s16 = sweep_stats(o, {k: v[pix[:, 1], pix[:, 0]] for k, v in g16.items()})
    # FP16 storage against the float32 form over the whole frame
    v = (g32["kstar"] >= 0) & (g16["kstar"] >= 0)
    same = (g32["kstar"] == g16["kstar"])[v].mean()
    rel = np.abs(g16["depth"][v] - g32["depth"][v]) / g32["depth"][v]
    pct = {q: float(np.percentile(rel, q)) for q in (50, 90, 99)}
    print("ring fp32 vs oracle", s32)
    print("ring fp16 vs oracle", s16)
    print("ring fp16 vs fp32", dict(plane_agree=float(same), rel_depth_pct=pct))
    assert s32["n_gated"] >= 60
    assert s32["valid_mismatch"] <= 0.01 and s32["index_agree"] >= 0.99 and s32["depth_ok"] >= 0.99
    assert s16["index_agree"] >= 0.95
    assert same >= 0.95 and pct[50] < 1e-3
