"""The C ABI library builds for sm_103a, loads without a GPU, exports every
entry point include/psweep.h declares, and rejects bad arguments before any
CUDA call."""
import ctypes as C
import os
import re

import pytest

import paper_1809_06132_gb300 as P
from paper_1809_06132_gb300 import psweep as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "psweep.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", txt, flags=re.M)))


def test_library_exports_every_declared_symbol():
    L = P.load()
    names = _declared()
    assert set(names) == set(P.EXPORTS)
    for n in names:
        assert hasattr(L, n), n
    assert "sm_103a" in P.version()


def test_struct_sizes_match_header_layout():
    # the ctypes mirrors must match the C layout (natural alignment)
    assert C.sizeof(B.ps_camera) == 10 * 8 + 2 * 4
    assert C.sizeof(B.ps_pose) == 12 * 8
    assert C.sizeof(B.ps_plane_set) == 8 + 2 * 8 + 3 * 8
    assert C.sizeof(B.ps_level) == 6 * 4 + 4 * C.sizeof(B.ps_plane_set)
    assert C.sizeof(B.ps_box) == 16


def test_argument_errors_without_gpu():
    L = P.load()
    h = C.c_void_p()
    assert L.psweep_create(None, C.byref(h)) == P.PS_ERR_ARG
    assert b"NULL" in L.ps_last_error()
    d = B.ps_sweep_desc()
    d.ref = B.ps_camera(xi=1.0, fx=80, fy=80, cx=80, cy=64, r2_max=1e30, width=160, height=128)
    d.n_cams = 0
    assert L.psweep_create(C.byref(d), C.byref(h)) == P.PS_ERR_ARG
    assert h.value is None
    cams = (B.ps_camera * 1)(d.ref)
    poses = (B.ps_pose * 1)()
    lv = (B.ps_level * 1)()
    lv[0].kind = 0
    lv[0].factor = 1
    lv[0].window = 6          # unsupported window
    lv[0].n_sets = 1
    lv[0].sets[0] = B.ps_plane_set(family=0, count=8, a=0.5, b=20.0)
    d.n_cams, d.cams, d.ref_to_cam, d.n_levels, d.levels = 1, cams, poses, 1, lv
    assert L.psweep_create(C.byref(d), C.byref(h)) == P.PS_ERR_ARG
    assert b"window" in L.ps_last_error()
    lv[0].window = 5
    lv[0].factor = 3          # does not divide 160x128
    assert L.psweep_create(C.byref(d), C.byref(h)) == P.PS_ERR_ARG
    lv[0].factor = 1
    lv[0].sets[0] = B.ps_plane_set(family=0, count=8, a=5.0, b=1.0)   # near > far
    assert L.psweep_create(C.byref(d), C.byref(h)) == P.PS_ERR_ARG
    td = B.ps_tsdf_desc()
    td.cam = d.ref
    td.voxel_size, td.mu, td.w_max, td.block_dim = 0.1, 0.5, 100.0, 4
    assert L.tsdf_create(C.byref(td), C.byref(h)) == P.PS_ERR_ARG
    td.block_dim = 8
    td.hash_slots = 1000      # not a power of two
    td.pool_blocks = 16
    assert L.tsdf_create(C.byref(td), C.byref(h)) == P.PS_ERR_ARG
    assert L.psweep_depth(None, None, None, 0, None, None, None) == P.PS_ERR_ARG
    assert L.tsdf_integrate(None, None, None, None, None) == P.PS_ERR_ARG
    n = C.c_int64()
    assert L.tsdf_listed(None, C.byref(n), None) == P.PS_ERR_ARG
    assert b"tsdf_listed" in L.ps_last_error()


def test_batch_argument_errors_without_gpu():
    L = P.load()
    h = C.c_void_p()
    assert C.sizeof(B.ps_batch_opts) == 8 * 4
    assert L.psbatch_create(None, 0, None, C.byref(h)) == P.PS_ERR_ARG
    # options are checked before any handle is used (the handles below are never dereferenced)
    fake = (C.c_void_p * 2)(0x1000, 0x2000)
    for bad in (dict(tile_h=20), dict(kp=3), dict(plane_chunk=-1), dict(order=5), dict(grid=-2),
                dict(wait_limit_ms=100000)):
        o = P.batch_opts(**bad)
        assert L.psbatch_create(fake, 2, C.byref(o), C.byref(h)) == P.PS_ERR_ARG, bad
        assert h.value is None
    same = (C.c_void_p * 2)(0x1000, 0x1000)
    assert L.psbatch_create(same, 2, None, C.byref(h)) == P.PS_ERR_ARG
    assert b"twice" in L.ps_last_error()
    assert L.psbatch_run(None, None, None, None, None, None) == P.PS_ERR_ARG
    assert L.psbatch_timing(None, None, None) == P.PS_ERR_ARG
    assert L.psbatch_status(None) == P.PS_ERR_ARG
    assert L.psbatch_queue_stats(None, None) == P.PS_ERR_ARG
    best = C.c_int32()
    ms = (C.c_double * 1)()
    assert L.psbatch_autotune(None, 0, None, None, None, None, None, 0, 1, C.byref(best), ms, None) == P.PS_ERR_ARG


def test_pipeline_argument_errors_without_gpu():
    L = P.load()
    h = C.c_void_p()
    assert L.ps_pipe_create(None, None, C.byref(h)) == P.PS_ERR_ARG
    assert h.value is None
    assert L.ps_pipe_push(None, None, None, 0, None, None, None) == P.PS_ERR_ARG
    assert L.ps_pipe_flush(None) == P.PS_ERR_ARG


def test_differentiable_argument_errors_without_gpu():
    L = P.load()
    h = C.c_void_p()
    assert L.psdiff_create(None, C.byref(h)) == P.PS_ERR_ARG
    d = B.ps_diff_desc()
    d.ref = B.ps_camera(xi=1.0, fx=48, fy=48, cx=48, cy=40, r2_max=1e30, width=96, height=80)
    cams = (B.ps_camera * 1)(d.ref)
    d.n_cams, d.cams = 1, cams
    d.level.kind, d.level.factor, d.level.window, d.level.n_sets = 0, 2, 5, 1      # factor 2: refused
    d.level.sets[0] = B.ps_plane_set(family=0, count=8, a=1.0, b=10.0)
    d.temperature = 0.05
    assert L.psdiff_create(C.byref(d), C.byref(h)) == P.PS_ERR_ARG
    d.level.factor = 1
    d.temperature = 0.0                                                           # T must be > 0
    assert L.psdiff_create(C.byref(d), C.byref(h)) == P.PS_ERR_ARG
    assert b"temperature" in L.ps_last_error()
    assert h.value is None
    assert L.psdiff_forward(None, None, None, None, None, None, None) == P.PS_ERR_ARG
    assert L.psdiff_backward(None, None, None, None, None, None, None, None, None) == P.PS_ERR_ARG
    assert L.tsdf_dense_fuse_backward(None, None, None, 0.1, 0.3, 100.0, None, None, None, None, None, None, None,
                                      None) == P.PS_ERR_ARG


def test_kernel_outputs_must_be_device_memory():
    # extract and swap_out write through kernels: host tensors are refused before any call
    from paper_1809_06132_gb300.psweep import _cuda_device
    with pytest.raises(ValueError):
        _cuda_device("cpu", "extract")
    assert _cuda_device("cuda", "extract").type == "cuda"


def test_points_argument_errors_without_gpu():
    L = P.load()
    n = C.c_int64()
    assert L.tsdf_extract_points(None, 3.0, None, None, 0, C.byref(n), None) == P.PS_ERR_ARG


def test_static_fusion_wrapper_checks_tensor_sizes():
    # the C entry point sees only pointers; the binding must refuse tensors
    # whose size does not match the grid or the camera before calling it
    import torch
    import scenes
    wl = scenes.tiny(0)
    p = wl.tsdf
    n_blocks = (p.dense_dim[0] // 8) * (p.dense_dim[1] // 8) * (p.dense_dim[2] // 8)
    good_vox = torch.zeros((n_blocks, 512, 2))
    good_depth = torch.zeros((wl.rig.ref.height, wl.rig.ref.width))
    cases = [(torch.zeros((n_blocks - 1, 512, 2)), good_depth, p.dense_dim),
             (good_vox, torch.zeros((wl.rig.ref.height - 1, wl.rig.ref.width)), p.dense_dim),
             (good_vox, good_depth, (p.dense_dim[0], p.dense_dim[1], 12))]
    for vox, dep, dims in cases:
        with pytest.raises(ValueError):
            P.tsdf_integrate_dense_static(vox, dims, p.origin, p.voxel_size, p.mu, p.w_max, dep, wl.rig.ref,
                                          wl.world_to_ref[0])


def test_sync_status_rejects_what_is_no_handle():
    L = P.load()
    assert L.ps_sync_status(None, None) == P.PS_ERR_ARG
    junk = (C.c_uint32 * 16)()            # host memory whose first word is no handle type
    assert L.ps_sync_status(C.cast(junk, C.c_void_p), None) == P.PS_ERR_ARG
    assert b"not a handle" in L.ps_last_error()
