"""The bounds-checked build (libpsweep_check.so, -DPS_CHECK) runs the sweep
with filters and boxes, a batch, the frame pipeline, hashed fusion with a
swap-out and a reload, dense fusion, and the differentiable forms with their
gradients, and records no out-of-range access.  It runs in a subprocess so
that the checked library is the one that process loads."""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np, torch, scenes
import paper_1809_06132_gb300 as P
assert "checked" in P.version(), P.version()
bits = 0
# sweep with filters and boxes, both levels
wl = scenes.street(0, n_frames=3, scale=0.25)
src = scenes.FrameSource(wl, device="cuda")
sw = P.Sweep(wl.rig, wl.levels, filters=scenes.Filters())
T = P.Tsdf(wl.tsdf, wl.rig.ref)
for f in range(3):
    imgs, _ = src.frame(f)
    dev = [torch.from_numpy(i.numpy()).cuda() for i in imgs]
    d = sw.depth(dev, boxes=wl.boxes[f])
    T.integrate(d, wl.world_to_ref[f], wl.local_center(f))
k, D, W = T.swap_out(tuple(np.array(wl.local_center(2)) + np.array([4.0, 0.0, 0.0])))
T.load_blocks(k, D, W)
T.extract()
bits |= P.check_read()
# a batch of uneven sweeps, 16-row tiles and one-plane passes too
wls = scenes.batch_mix(3, n=4, sizes=((256, 200), (320, 256)), planes=(32, 64))
sws, ims = [], []
for w in wls:
    i, _ = scenes.FrameSource(w, device="cuda").frame(0)
    ims.append([torch.from_numpy(x.numpy()).cuda() for x in i])
    sws.append(P.Sweep(w.rig, w.levels))
for opts in (dict(), dict(tile_h=16, kp=1, plane_chunk=8)):
    P.Batch(sws, **opts).run(ims, boxes=[w.boxes[0] for w in wls])
bits |= P.check_read()
# frame pipeline
pipe = P.Pipeline(P.Sweep(wl.rig, wl.levels), P.Tsdf(wl.tsdf, wl.rig.ref))
for f in range(3):
    imgs, _ = src.frame(f)
    pipe.push([i.numpy() for i in imgs], boxes=wl.boxes[f], world_to_ref=wl.world_to_ref[f],
              local_center=wl.local_center(f), depth_out=np.empty((wl.rig.ref.height, wl.rig.ref.width), np.float32))
pipe.flush()
bits |= P.check_read()
# dense fusion (static entry point) and its gradient; the differentiable sweep
tw = scenes.tiny(0, n_frames=1)
_, rng = scenes.FrameSource(tw).frame(0, with_range=True)
depth = torch.from_numpy(rng.numpy().astype(np.float32)).cuda()
vox = torch.zeros((512, 512, 2), dtype=torch.float32, device="cuda")
out = P.dense_fuse(vox.requires_grad_(True), depth, tw.tsdf, tw.rig.ref, tw.world_to_ref[0])
out[..., 0].sum().backward()
dw = scenes.diff(0)
i, _ = scenes.FrameSource(dw).frame(0)
dims = [torch.from_numpy(x.numpy().astype(np.float32) / 255.0).cuda().requires_grad_(True) for x in i]
ss = P.SoftSweep(dw.rig, dw.levels[0])
r, c = P.soft_depth(ss, dims, torch.zeros((2, 6), dtype=torch.float64, requires_grad=True))
(r.sum() + c.sum()).backward()
bits |= P.check_read()
print("CHECK_BITS", bits)
'''


def test_checked_build_records_no_out_of_range_access():
    env = dict(os.environ, PSWEEP_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("CHECK_BITS")]
    assert line == ["CHECK_BITS 0"], r.stdout[-2000:]
