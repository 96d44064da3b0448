"""The allocation-free fusion entry point gives the same map as the ordinary one.

Some callers cannot allocate GPU memory while they run: real-time loops
whose memory is planned once up front, and hosts whose device memory belongs
to another allocator.  For them tsdf_integrate_dense_static fuses a depth map into a
dense grid that the caller owns, using a fixed static device array as its
only working memory.  This test calls it through the C ABI twice in a row
and checks each result against tsdf_create + tsdf_integrate on the same
dense grid, within the tolerance the other fusion tests use.
"""
import numpy as np
import pytest
import torch

import scenes
from tests.parity import TSDF_ABS

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1809_06132_gb300 as P  # noqa: E402
from paper_1809_06132_gb300 import psweep as B  # noqa: E402


def test_static_entry_point_matches_allocating_path():
    wl = scenes.tiny(0, n_frames=2)
    p = wl.tsdf
    src = scenes.FrameSource(wl)
    T = P.Tsdf(p, wl.rig.ref)                      # ordinary path: handle-owned dense grid
    n_blocks = (p.dense_dim[0] // 8) * (p.dense_dim[1] // 8) * (p.dense_dim[2] // 8)
    voxels = torch.zeros((n_blocks, 512, 2), dtype=torch.float32, device="cuda")   # caller-owned grid
    for f in range(2):                             # two calls in a row
        _, rng = src.frame(f, with_range=True)
        depth = torch.from_numpy(rng.numpy().astype(np.float32)).cuda()
        T.integrate(depth, wl.world_to_ref[f])
        P.tsdf_integrate_dense_static(voxels, p.dense_dim, p.origin, p.voxel_size, p.mu, p.w_max, depth,
                                      wl.rig.ref, wl.world_to_ref[f])
        torch.cuda.synchronize()
        keys, D, W = T.extract()
        assert keys.shape[0] == n_blocks
        assert (W > 0).sum().item() > 1000
        assert torch.max(torch.abs(voxels[..., 0] - D)).item() <= TSDF_ABS
        assert torch.equal(voxels[..., 1], W)
        assert W.max().item() == f + 1


def test_static_entry_point_rejects_grids_over_the_limit():
    wl = scenes.tiny(0)
    p = wl.tsdf
    depth = torch.zeros((wl.rig.ref.height, wl.rig.ref.width), dtype=torch.float32, device="cuda")
    voxels = torch.zeros((1, 512, 2), dtype=torch.float32, device="cuda")
    # through the C ABI directly: the binding's own size checks would stop
    # these calls before the library's limit check
    lib = P.load()
    d = lambda *v: (B.C.c_int32 * 3)(*v)  # noqa: E731
    o = (B.C.c_double * 3)(*p.origin)
    cz, pz = B.camera(wl.rig.ref), B.pose(wl.world_to_ref[0])
    for dims in ((512, 512, 512), (1 << 30, 1 << 30, 8), (2147483640, 2147483640, 2147483640)):
        st = lib.tsdf_integrate_dense_static(voxels.data_ptr(), d(*dims), o, p.voxel_size, p.mu, p.w_max,
                                             depth.data_ptr(), B.C.byref(cz), B.C.byref(pz), None)
        assert st == P.PS_ERR_ARG, dims
        assert str(P.STATIC_MAX_BLOCKS) in lib.ps_last_error().decode()
