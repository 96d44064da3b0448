"""The frame pipeline (ps_pipe_* through the C ABI: copy-in, sweep and
fuse + copy-out streams with two frames in flight) gives every frame the
depth map psweep_frame_host gives it, and the same fused volume."""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1809_06132_gb300 as P  # noqa: E402


def _sorted(k, D, W):
    k, D, W = k.cpu().numpy(), D.cpu().numpy(), W.cpu().numpy()
    o = np.lexsort((k[:, 2], k[:, 1], k[:, 0]))
    return k[o], D[o], W[o]


@pytest.mark.parametrize("with_tsdf", [True, False])
def test_pipeline_matches_serial_frames(with_tsdf):
    wl = scenes.street(3, n_frames=7, scale=0.25)
    src = scenes.FrameSource(wl, device="cuda")
    frames = [[i.numpy() for i in src.frame(f)[0]] for f in range(7)]
    H, W = wl.rig.ref.height, wl.rig.ref.width
    sw1, sw2 = P.Sweep(wl.rig, wl.levels), P.Sweep(wl.rig, wl.levels)
    T1 = P.Tsdf(wl.tsdf, wl.rig.ref) if with_tsdf else None
    T2 = P.Tsdf(wl.tsdf, wl.rig.ref) if with_tsdf else None
    serial = []
    for f in range(7):
        out = np.empty((H, W), np.float32)
        sw1.frame_host(frames[f], boxes=wl.boxes[f], tsdf=T1, world_to_ref=wl.world_to_ref[f],
                       local_center=wl.local_center(f), depth_out=out)
        serial.append(out)
    pipe = P.Pipeline(sw2, T2)
    outs = [np.full((H, W), -1.0, np.float32) for _ in range(7)]
    for f in range(7):
        pipe.push(frames[f], boxes=wl.boxes[f], world_to_ref=wl.world_to_ref[f], local_center=wl.local_center(f),
                  depth_out=outs[f] if f != 3 else None)   # frame 3 without a host copy
        if f >= 2 and f - 2 != 3:
            assert np.array_equal(outs[f - 2], serial[f - 2]), f - 2   # delivered by the push two frames later
    pipe.flush()
    for f in range(7):
        if f == 3:
            assert (outs[f] == -1.0).all()
        else:
            assert np.array_equal(outs[f], serial[f]), f
    if with_tsdf:
        assert T1.status() == P.PS_OK and T2.status() == P.PS_OK
        a, b = _sorted(*T1.extract()), _sorted(*T2.extract())
        assert len(a[0]) > 100
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    pipe.close()
