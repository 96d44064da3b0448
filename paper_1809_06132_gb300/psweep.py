"""Python binding of libpsweep.so (ctypes): argument marshalling only.

Every step of the fisheye plane sweep and the TSDF fusion runs in the CUDA
kernels behind the C ABI declared in include/psweep.h.  This module converts
camera / pose / level descriptions (any objects with the attribute names
used below) into the C structs, passes torch tensors as raw device pointers
and torch streams as cudaStream_t, and raises on every non-zero status.
There is no fallback: if the library cannot be loaded, importing it fails.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import _build

PS_OK, PS_ERR_ARG, PS_ERR_OOM, PS_ERR_CAPACITY, PS_ERR_CUDA, PS_ERR_TIMEOUT, PS_ERR_STATE = range(7)
STATUS_NAMES = {1: "PS_ERR_ARG", 2: "PS_ERR_OOM", 3: "PS_ERR_CAPACITY", 4: "PS_ERR_CUDA", 5: "PS_ERR_TIMEOUT",
                6: "PS_ERR_STATE"}
MAX_SETS, MAX_CAMS, MAX_LEVELS = 4, 4, 2

# every symbol include/psweep.h declares
EXPORTS = ["psweep_create", "psweep_depth", "psweep_destroy", "tsdf_create", "tsdf_integrate", "tsdf_count", "tsdf_listed",
           "tsdf_extract", "tsdf_status", "tsdf_destroy", "psweep_frame_host", "psweep_profile",
           "psweep_profile_read", "tsdf_profile", "tsdf_profile_read", "tsdf_integrate_dense_static",
           "tsdf_swap_out", "tsdf_load", "tsdf_extract_points", "psbatch_create", "psbatch_run", "psbatch_timing", "psbatch_status",
           "psbatch_queue_stats", "psbatch_destroy", "psbatch_autotune", "ps_pipe_create", "ps_pipe_push",
           "ps_pipe_flush", "ps_pipe_destroy", "psdiff_create", "psdiff_forward", "psdiff_backward",
           "psdiff_destroy", "tsdf_dense_fuse_backward",
           "ps_check_read", "ps_last_error", "ps_version", "ps_sync_status", "psweep_depth_planes",
           "psweep_merge_records", "tsdf_set_partition", "psweep_level_outputs"]
MAX_PARTS = 16
N_RECORD = 7  # floats per pixel in a plane-range record


class PsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ps_camera(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("xi", "fx", "fy", "cx", "cy", "k1", "k2", "p1", "p2", "r2_max")] + \
               [("width", C.c_int32), ("height", C.c_int32)]


class ps_pose(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3)]


class ps_plane_set(C.Structure):
    _fields_ = [("family", C.c_int32), ("count", C.c_int32), ("a", C.c_double), ("b", C.c_double),
                ("n", C.c_double * 3)]


class ps_level(C.Structure):
    _fields_ = [("kind", C.c_int32), ("factor", C.c_int32), ("crop_w", C.c_int32), ("crop_h", C.c_int32),
                ("window", C.c_int32), ("n_sets", C.c_int32), ("sets", ps_plane_set * MAX_SETS)]


class ps_filter(C.Structure):
    _fields_ = [("enable", C.c_int32), ("window", C.c_int32), ("alpha_upper", C.c_double),
                ("alpha_lower", C.c_double), ("split_row", C.c_double), ("ratio_min", C.c_double),
                ("gamma", C.c_double), ("delta", C.c_double)]


class ps_sweep_desc(C.Structure):
    _fields_ = [("ref", ps_camera), ("n_cams", C.c_int32), ("cams", C.POINTER(ps_camera)),
                ("ref_to_cam", C.POINTER(ps_pose)), ("n_levels", C.c_int32), ("levels", C.POINTER(ps_level)),
                ("filter", ps_filter), ("image_half", C.c_int32)]


class ps_box(C.Structure):
    _fields_ = [("x0", C.c_int32), ("y0", C.c_int32), ("x1", C.c_int32), ("y1", C.c_int32)]


class ps_level_out(C.Structure):
    _fields_ = [("depth", C.c_void_p), ("best_cost", C.c_void_p), ("second_cost", C.c_void_p),
                ("plane_idx", C.c_void_p)]


class ps_batch_opts(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("tile_h", "kp", "plane_chunk", "order", "use_graph", "grid",
                                         "wait_limit_ms", "drill_unmet_wait")]


class ps_diff_desc(C.Structure):
    _fields_ = [("ref", ps_camera), ("n_cams", C.c_int32), ("cams", C.POINTER(ps_camera)), ("level", ps_level),
                ("temperature", C.c_double)]


class ps_tsdf_desc(C.Structure):
    _fields_ = [("cam", ps_camera), ("voxel_size", C.c_double), ("mu", C.c_double), ("w_max", C.c_double),
                ("block_dim", C.c_int32), ("dense_dim", C.c_int32 * 3), ("origin", C.c_double * 3),
                ("local_half", C.c_double * 3), ("hash_slots", C.c_int64), ("pool_blocks", C.c_int64)]


_lib = None


def _checked() -> bool:
    """PSWEEP_CHECKED=1 selects the bounds-checked build of the library."""
    return os.environ.get("PSWEEP_CHECKED", "") == "1"


def lib_path() -> str:
    return _build.LIB_CHECK if _checked() else _build.LIB


def load(build_if_missing: bool = True):
    """Load libpsweep.so (building it in-tree first if it is missing);
    libpsweep_check.so when PSWEEP_CHECKED=1."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"{os.path.basename(path)} not built at {path}")
        _build.build(check=_checked())
    L = C.CDLL(path)
    P = C.c_void_p
    L.psweep_create.argtypes = [C.POINTER(ps_sweep_desc), C.POINTER(C.c_void_p)]
    L.psweep_depth.argtypes = [P, P, P, C.c_int32, P, P, P]
    L.psweep_destroy.argtypes = [P]
    L.psweep_destroy.restype = None
    L.tsdf_create.argtypes = [C.POINTER(ps_tsdf_desc), C.POINTER(C.c_void_p)]
    L.tsdf_integrate.argtypes = [P, P, C.POINTER(ps_pose), P, P]
    L.tsdf_count.argtypes = [P, C.POINTER(C.c_int64), P]
    L.tsdf_listed.argtypes = [P, C.POINTER(C.c_int64), P]
    L.tsdf_extract.argtypes = [P, C.c_float, P, P, P, C.c_int64, C.POINTER(C.c_int64), P]
    L.tsdf_status.argtypes = [P, P]
    L.tsdf_destroy.argtypes = [P]
    L.tsdf_destroy.restype = None
    L.psweep_frame_host.argtypes = [P, P, P, P, C.c_int32, C.POINTER(ps_pose), P, P, P]
    L.psweep_profile.argtypes = [P, C.c_int32]
    L.psweep_profile_read.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_int32)]
    L.tsdf_profile.argtypes = [P, C.c_int32]
    L.tsdf_profile_read.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_int32)]
    L.tsdf_swap_out.argtypes = [P, P, P, P, P, C.c_int64, C.POINTER(C.c_int64), P]
    L.tsdf_load.argtypes = [P, P, P, P, C.c_int64, P]
    L.tsdf_extract_points.argtypes = [P, C.c_float, P, P, C.c_int64, C.POINTER(C.c_int64), P]
    L.tsdf_integrate_dense_static.argtypes = [P, P, P, C.c_double, C.c_double, C.c_double, P,
                                              C.POINTER(ps_camera), C.POINTER(ps_pose), P]
    L.psbatch_create.argtypes = [P, C.c_int32, C.POINTER(ps_batch_opts), C.POINTER(C.c_void_p)]
    L.psbatch_run.argtypes = [P, P, P, P, P, P]
    L.psbatch_timing.argtypes = [P, P, P]
    L.psbatch_status.argtypes = [P]
    L.psbatch_queue_stats.argtypes = [P, P]
    L.psbatch_destroy.argtypes = [P]
    L.psbatch_destroy.restype = None
    L.psbatch_autotune.argtypes = [P, C.c_int32, P, P, P, P, C.POINTER(ps_batch_opts), C.c_int32, C.c_int32,
                                   C.POINTER(C.c_int32), P, P]
    L.ps_pipe_create.argtypes = [P, P, C.POINTER(C.c_void_p)]
    L.ps_pipe_push.argtypes = [P, P, P, C.c_int32, C.POINTER(ps_pose), P, P]
    L.ps_pipe_flush.argtypes = [P]
    L.ps_pipe_destroy.argtypes = [P]
    L.ps_pipe_destroy.restype = None
    L.psdiff_create.argtypes = [C.POINTER(ps_diff_desc), C.POINTER(C.c_void_p)]
    L.psdiff_forward.argtypes = [P, P, P, P, P, P, P]
    L.psdiff_backward.argtypes = [P, P, P, P, P, P, P, P, P]
    L.psdiff_destroy.argtypes = [P]
    L.psdiff_destroy.restype = None
    L.tsdf_dense_fuse_backward.argtypes = [P, P, P, C.c_double, C.c_double, C.c_double, P, C.POINTER(ps_camera),
                                           C.POINTER(ps_pose), P, P, P, P, P]
    L.ps_check_read.argtypes = [C.POINTER(C.c_uint32)]
    L.ps_sync_status.argtypes = [P, P]
    L.psweep_depth_planes.argtypes = [P, P, P, P, P, P]
    L.psweep_merge_records.argtypes = [P, C.c_int32, P, P, P, C.c_int32, P, P, P]
    L.tsdf_set_partition.argtypes = [P, C.c_int32, C.c_int32]
    L.psweep_level_outputs.argtypes = [P, P, P]
    L.ps_last_error.restype = C.c_char_p
    L.ps_version.restype = C.c_char_p
    _lib = L
    return L


def _check(st: int):
    if st != PS_OK:
        raise PsError(st, load().ps_last_error().decode())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def camera(c) -> ps_camera:
    return ps_camera(xi=c.xi, fx=c.fx, fy=c.fy, cx=c.cx, cy=c.cy, k1=c.k1, k2=c.k2, p1=c.p1, p2=c.p2,
                     r2_max=min(float(c.r2_max), 1e300), width=c.width, height=c.height)


def pose(p) -> ps_pose:
    o = ps_pose()
    R = np.asarray(p.R, dtype=np.float64).reshape(-1)
    t = np.asarray(p.t, dtype=np.float64).reshape(-1)
    for i in range(9):
        o.R[i] = R[i]
    for i in range(3):
        o.t[i] = t[i]
    return o


def level(lv) -> ps_level:
    assert len(lv.sets) <= MAX_SETS
    o = ps_level(kind=lv.kind, factor=lv.factor, crop_w=lv.crop_w, crop_h=lv.crop_h, window=lv.window,
                 n_sets=len(lv.sets))
    for i, s in enumerate(lv.sets):
        o.sets[i].family = s.family
        o.sets[i].count = s.count
        o.sets[i].a = s.a
        o.sets[i].b = s.b
        for k in range(3):
            o.sets[i].n[k] = s.n[k]
    return o


def boxes_array(boxes):
    b = np.zeros((0, 4), dtype=np.int32) if boxes is None else np.ascontiguousarray(boxes, dtype=np.int32)
    n = len(b)
    arr = (ps_box * max(1, n))()
    for i in range(n):
        arr[i] = ps_box(*[int(v) for v in b[i]])
    return arr, n


def _cuda_device(device, name: str):
    """Output buffers that kernels write must be device memory."""
    d = torch.device(device)
    if d.type != "cuda":
        raise ValueError(f"{name}: outputs are written by kernels and must be on a CUDA device, not {d}")
    return d


def _dev(t: torch.Tensor, dtype, name: str) -> int:
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t.data_ptr()


def level_shape(ref, lv):
    if lv.kind == 0:
        return ref.height // lv.factor, ref.width // lv.factor
    return lv.crop_h, lv.crop_w


class Sweep:
    """Multi-scale fisheye plane sweep of one rig (psweep_create / psweep_depth)."""

    def __init__(self, rig, levels, filters=None, image_half: bool = False):
        L = load()
        self.rig = rig
        self.levels = list(levels)
        self._cams = (ps_camera * len(rig.cams))(*[camera(c) for c in rig.cams])
        self._poses = (ps_pose * len(rig.cams))(*[pose(p) for p in rig.ref_to_cam])
        self._levels = (ps_level * len(self.levels))(*[level(lv) for lv in self.levels])
        d = ps_sweep_desc(ref=camera(rig.ref), n_cams=len(rig.cams), cams=self._cams, ref_to_cam=self._poses,
                          n_levels=len(self.levels), levels=self._levels, image_half=1 if image_half else 0)
        if filters is not None and filters.enable:
            d.filter = ps_filter(enable=1, window=filters.window, alpha_upper=filters.alpha_upper,
                                 alpha_lower=filters.alpha_lower, split_row=filters.split_row,
                                 ratio_min=filters.ratio_min, gamma=filters.gamma, delta=filters.delta)
        h = C.c_void_p()
        _check(L.psweep_create(C.byref(d), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().psweep_destroy(self.h)
            self.h = None

    __del__ = close

    def profile(self, capacity: int):
        """Record stage events for the next `capacity` depth calls (0 = off)."""
        _check(load().psweep_profile(self.h, int(capacity)))

    def profile_read(self):
        """(summed ms per stage [prep, sweep kernel, merge], calls recorded)."""
        ms = (C.c_double * 3)()
        n = C.c_int32()
        _check(load().psweep_profile_read(self.h, ms, C.byref(n)))
        return list(ms), n.value

    def sync_status(self, stream=None) -> int:
        """ps_sync_status: synchronise the stream, return and clear the
        handle's latched device status (a PS_* code)."""
        return load().ps_sync_status(self.h, _stream_ptr(stream))

    def level_shapes(self):
        return [level_shape(self.rig.ref, lv) for lv in self.levels]

    def alloc_level_outputs(self, device="cuda"):
        outs = []
        for (h, w) in self.level_shapes():
            outs.append(dict(depth=torch.empty((h, w), dtype=torch.float32, device=device),
                             c1=torch.empty((h, w), dtype=torch.float32, device=device),
                             c2=torch.empty((h, w), dtype=torch.float32, device=device),
                             kstar=torch.empty((h, w), dtype=torch.int32, device=device)))
        return outs

    def depth(self, images: Sequence[torch.Tensor], boxes=None, out: Optional[torch.Tensor] = None,
              level_outs=None, stream=None) -> torch.Tensor:
        """images: [ref, cam_1, ...] contiguous uint8 CUDA tensors (H, W)."""
        n = 1 + len(self.rig.cams)
        if len(images) != n:
            raise ValueError(f"expected {n} images")
        ptrs = (C.c_void_p * n)(*[_dev(im, torch.uint8, f"images[{i}]") for i, im in enumerate(images)])
        if out is None:
            out = torch.empty((self.rig.ref.height, self.rig.ref.width), dtype=torch.float32,
                              device=images[0].device)
        bx, nb = boxes_array(boxes)
        lo = None
        if level_outs is not None:
            lo = (ps_level_out * len(self.levels))()
            for i, o in enumerate(level_outs):
                lo[i] = ps_level_out(
                    _dev(o["depth"], torch.float32, "depth") if o.get("depth") is not None else None,
                    _dev(o["c1"], torch.float32, "c1") if o.get("c1") is not None else None,
                    _dev(o["c2"], torch.float32, "c2") if o.get("c2") is not None else None,
                    _dev(o["kstar"], torch.int32, "kstar") if o.get("kstar") is not None else None)
        _check(load().psweep_depth(self.h, ptrs, bx, nb, _dev(out, torch.float32, "out"), lo, _stream_ptr(stream)))
        return out

    def level_outputs(self, outs=None, stream=None):
        """The handle's own level outputs (left by the last psweep_depth without
        level_outs or by the last batch run over this handle), copied out."""
        if outs is None:
            outs = self.alloc_level_outputs()
        lo = (ps_level_out * len(self.levels))()
        for i, o in enumerate(outs):
            lo[i] = ps_level_out(_dev(o["depth"], torch.float32, "depth"), _dev(o["c1"], torch.float32, "c1"),
                                 _dev(o["c2"], torch.float32, "c2"), _dev(o["kstar"], torch.int32, "kstar"))
        _check(load().psweep_level_outputs(self.h, lo, _stream_ptr(stream)))
        return outs

    def alloc_records(self, device="cuda"):
        """Per level, a (7, H_l, W_l) float32 buffer for a plane-range record."""
        return [torch.empty((N_RECORD, h, w), dtype=torch.float32, device=device) for (h, w) in self.level_shapes()]

    def n_planes(self):
        return [lv.n_planes for lv in self.levels]

    def depth_planes(self, images: Sequence[torch.Tensor], plane_lo, plane_hi, records=None, stream=None):
        """Sweep planes [plane_lo[l], plane_hi[l]) of each level; per level a
        (7, H_l, W_l) record of that range (psweep_depth_planes)."""
        n = 1 + len(self.rig.cams)
        if len(images) != n:
            raise ValueError(f"expected {n} images")
        nl = len(self.levels)
        if len(plane_lo) != nl or len(plane_hi) != nl:
            raise ValueError(f"plane_lo / plane_hi need {nl} entries")
        if records is None:
            records = self.alloc_records(images[0].device)
        for r, (h, w) in zip(records, self.level_shapes()):
            if tuple(r.shape) != (N_RECORD, h, w):
                raise ValueError(f"a record buffer must be ({N_RECORD}, {h}, {w})")
        ptrs = (C.c_void_p * n)(*[_dev(im, torch.uint8, f"images[{i}]") for i, im in enumerate(images)])
        lo = (C.c_int32 * nl)(*[int(v) for v in plane_lo])
        hi = (C.c_int32 * nl)(*[int(v) for v in plane_hi])
        rp = (C.c_void_p * nl)(*[_dev(r, torch.float32, "records") for r in records])
        _check(load().psweep_depth_planes(self.h, ptrs, lo, hi, rp, _stream_ptr(stream)))
        return records

    def merge_records(self, part_lo, records, boxes=None, out: Optional[torch.Tensor] = None, level_outs=None,
                      stream=None, device=None) -> torch.Tensor:
        """psweep_merge_records: part_lo[p][l] = first plane of part p at level l
        (part 0 at 0); records[p][l] = that part's (7, H_l, W_l) record."""
        nl = len(self.levels)
        n_parts = len(part_lo)
        if not 1 <= n_parts <= MAX_PARTS or len(records) != n_parts:
            raise ValueError(f"need 1..{MAX_PARTS} parts with one record list each")
        for p in range(n_parts):
            if len(records[p]) != nl:
                raise ValueError(f"part {p} needs {nl} record buffers")
            for r, (h, w) in zip(records[p], self.level_shapes()):
                if tuple(r.shape) != (N_RECORD, h, w) or r.dtype != torch.float32 or not r.is_contiguous():
                    raise ValueError(f"part {p}: a record buffer must be contiguous float32 ({N_RECORD}, {h}, {w})")
        lo = (C.c_int32 * (n_parts * nl))(*[int(part_lo[p][l]) for p in range(n_parts) for l in range(nl)])
        rp = (C.c_void_p * (n_parts * nl))(*[_dev(records[p][l], torch.float32, "records")
                                             for p in range(n_parts) for l in range(nl)])
        if out is None:
            out = torch.empty((self.rig.ref.height, self.rig.ref.width), dtype=torch.float32,
                              device=device or records[0][0].device)
        bx, nb = boxes_array(boxes)
        lvo = None
        if level_outs is not None:
            lvo = (ps_level_out * nl)()
            for i, o in enumerate(level_outs):
                lvo[i] = ps_level_out(
                    _dev(o["depth"], torch.float32, "depth") if o.get("depth") is not None else None,
                    _dev(o["c1"], torch.float32, "c1") if o.get("c1") is not None else None,
                    _dev(o["c2"], torch.float32, "c2") if o.get("c2") is not None else None,
                    _dev(o["kstar"], torch.int32, "kstar") if o.get("kstar") is not None else None)
        _check(load().psweep_merge_records(self.h, n_parts, lo, rp, bx, nb, _dev(out, torch.float32, "out"), lvo,
                                           _stream_ptr(stream)))
        return out

    def frame_host(self, host_images: Sequence[np.ndarray], boxes=None, tsdf: "Tsdf" = None, world_to_ref=None,
                   local_center=None, depth_out: Optional[np.ndarray] = None, stream=None):
        """One frame from host memory: H2D copies, depth, optional fusion, D2H depth (synchronous)."""
        n = 1 + len(self.rig.cams)
        arrs = [np.ascontiguousarray(a, dtype=np.uint8) if isinstance(a, np.ndarray) else a for a in host_images]
        ptrs = (C.c_void_p * n)(*[a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr() for a in arrs])
        bx, nb = boxes_array(boxes)
        pz = pose(world_to_ref) if world_to_ref is not None else None
        lc = None if local_center is None else (C.c_double * 3)(*local_center)
        dptr = None
        if depth_out is not None:
            dptr = depth_out.ctypes.data if isinstance(depth_out, np.ndarray) else depth_out.data_ptr()
        _check(load().psweep_frame_host(self.h, tsdf.h if tsdf is not None else None, ptrs, bx, nb,
                                        C.byref(pz) if pz is not None else None, lc, dptr, _stream_ptr(stream)))
        return depth_out


class Pipeline:
    """Host frames through copy-in / compute (sweep, then fusion) / copy-out
    streams, two frames in flight (ps_pipe_*).  push() returns at once; the depth map of a frame
    lands in its host buffer by the time the push two calls later, or
    flush(), returns."""

    def __init__(self, sweep: Sweep, tsdf: Optional["Tsdf"] = None):
        h = C.c_void_p()
        _check(load().ps_pipe_create(sweep.h, tsdf.h if tsdf is not None else None, C.byref(h)))
        self.h = h
        self.sweep, self.tsdf = sweep, tsdf
        self._keep = [None, None]   # host buffers of the frames in flight
        self._n = 0

    def close(self):
        if getattr(self, "h", None):
            load().ps_pipe_destroy(self.h)
            self.h = None

    __del__ = close

    def push(self, host_images: Sequence[np.ndarray], boxes=None, world_to_ref=None, local_center=None,
             depth_out: Optional[np.ndarray] = None):
        n = 1 + len(self.sweep.rig.cams)
        arrs = [np.ascontiguousarray(a, dtype=np.uint8) if isinstance(a, np.ndarray) else a for a in host_images]
        ptrs = (C.c_void_p * n)(*[a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr() for a in arrs])
        bx, nb = boxes_array(boxes)
        pz = pose(world_to_ref) if world_to_ref is not None else None
        lc = None if local_center is None else (C.c_double * 3)(*local_center)
        dptr = None
        if depth_out is not None:
            dptr = depth_out.ctypes.data if isinstance(depth_out, np.ndarray) else depth_out.data_ptr()
        _check(load().ps_pipe_push(self.h, ptrs, bx, nb, C.byref(pz) if pz is not None else None, lc, dptr))
        self._keep[self._n & 1] = depth_out
        self._n += 1
        return depth_out

    def flush(self):
        _check(load().ps_pipe_flush(self.h))
        self._keep = [None, None]


BATCH_SHORTEST_FIRST, BATCH_GIVEN_ORDER = 0, 1
QUEUE_KINDS = ("ref", "quad", "stats", "sweep", "merge", "continuity")


def batch_opts(tile_h: int = 24, kp: int = 2, plane_chunk: int = 32, order: int = BATCH_SHORTEST_FIRST,
               use_graph: bool = False, grid: int = 0, wait_limit_ms: int = 2000,
               drill_unmet_wait: bool = False) -> ps_batch_opts:
    return ps_batch_opts(int(tile_h), int(kp), int(plane_chunk), int(order), 1 if use_graph else 0, int(grid),
                         int(wait_limit_ms), 1 if drill_unmet_wait else 0)


class _BatchArgs:
    """C arrays of one batch run: images, boxes and outputs of every sweep."""

    def __init__(self, sweeps, images, boxes, outs):
        if len(images) != len(sweeps) or len(outs) != len(sweeps):
            raise ValueError("one image list and one output per sweep")
        flat = []
        for i, (sw, ims) in enumerate(zip(sweeps, images)):
            if len(ims) != 1 + len(sw.rig.cams):
                raise ValueError(f"sweep {i}: expected {1 + len(sw.rig.cams)} images")
            flat += [_dev(im, torch.uint8, f"images[{i}]") for im in ims]
        self.images = (C.c_void_p * len(flat))(*flat)
        boxes = boxes if boxes is not None else [None] * len(sweeps)
        allb = [np.zeros((0, 4), np.int32) if b is None else np.ascontiguousarray(b, dtype=np.int32).reshape(-1, 4)
                for b in boxes]
        self.n_boxes = (C.c_int32 * len(sweeps))(*[len(b) for b in allb])
        cat = np.concatenate(allb, axis=0) if allb else np.zeros((0, 4), np.int32)
        self.boxes, _ = boxes_array(cat)
        self.outs = (C.c_void_p * len(sweeps))(*[_dev(o, torch.float32, f"out[{i}]") for i, o in enumerate(outs)])


class Batch:
    """Depth maps of many sweeps in one persistent launch (psbatch_*)."""

    def __init__(self, sweeps: Sequence[Sweep], opts: Optional[ps_batch_opts] = None, **kw):
        L = load()
        self.sweeps = list(sweeps)
        self.opts = opts if opts is not None else batch_opts(**kw)
        hs = (C.c_void_p * len(self.sweeps))(*[s.h for s in self.sweeps])
        h = C.c_void_p()
        _check(L.psbatch_create(hs, len(self.sweeps), C.byref(self.opts), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().psbatch_destroy(self.h)
            self.h = None

    __del__ = close

    def alloc_outputs(self, device="cuda"):
        return [torch.empty((s.rig.ref.height, s.rig.ref.width), dtype=torch.float32, device=device)
                for s in self.sweeps]

    def run(self, images, boxes=None, outs=None, stream=None):
        """images: per sweep a list [ref, cam_1, ...] of uint8 CUDA tensors; boxes: per sweep (n, 4) or None."""
        if outs is None:
            outs = self.alloc_outputs(images[0][0].device)
        a = _BatchArgs(self.sweeps, images, boxes, outs)
        _check(load().psbatch_run(self.h, a.images, a.boxes, a.n_boxes, a.outs, _stream_ptr(stream)))
        return outs

    def timing(self):
        """(per-sweep ms from kernel start to its depth map, ms to the last one) of the last run."""
        done = (C.c_double * len(self.sweeps))()
        span = C.c_double()
        _check(load().psbatch_timing(self.h, done, C.byref(span)))
        return list(done), span.value

    def status(self) -> int:
        return load().psbatch_status(self.h)

    def sync_status(self, stream=None) -> int:
        """ps_sync_status on this batch handle (the last run's outcome)."""
        return load().ps_sync_status(self.h, _stream_ptr(stream))

    def queue_stats(self):
        c = (C.c_int32 * 6)()
        _check(load().psbatch_queue_stats(self.h, c))
        return dict(zip(QUEUE_KINDS, list(c)))


def batch_autotune(sweeps: Sequence[Sweep], images, candidates: Sequence[ps_batch_opts], boxes=None, outs=None,
                   reps: int = 3, stream=None):
    """Time every candidate option set on these inputs; (best index, median ms per candidate)."""
    if outs is None:
        outs = [torch.empty((s.rig.ref.height, s.rig.ref.width), dtype=torch.float32, device="cuda")
                for s in sweeps]
    a = _BatchArgs(sweeps, images, boxes, outs)
    hs = (C.c_void_p * len(sweeps))(*[s.h for s in sweeps])
    cand = (ps_batch_opts * len(candidates))(*candidates)
    best = C.c_int32()
    ms = (C.c_double * len(candidates))()
    _check(load().psbatch_autotune(hs, len(sweeps), a.images, a.boxes, a.n_boxes, a.outs, cand, len(candidates),
                                   int(reps), C.byref(best), ms, _stream_ptr(stream)))
    return best.value, list(ms)


class Tsdf:
    """TSDF volume of voxel blocks (tsdf_create / tsdf_integrate / tsdf_extract)."""

    def __init__(self, params, cam):
        L = load()
        p = params
        d = ps_tsdf_desc(cam=camera(cam), voxel_size=p.voxel_size, mu=p.mu, w_max=p.w_max, block_dim=p.block_dim,
                         hash_slots=p.hash_slots, pool_blocks=p.pool_blocks)
        if p.dense_dim is not None:
            for i in range(3):
                d.dense_dim[i] = p.dense_dim[i]
        for i in range(3):
            d.origin[i] = p.origin[i]
            d.local_half[i] = p.local_half[i] if p.local_half is not None else 0.0
        h = C.c_void_p()
        _check(L.tsdf_create(C.byref(d), C.byref(h)))
        self.h = h
        self.params = p

    def close(self):
        if getattr(self, "h", None):
            load().tsdf_destroy(self.h)
            self.h = None

    __del__ = close

    def integrate(self, depth: torch.Tensor, world_to_cam, local_center=None, stream=None):
        pz = pose(world_to_cam)
        lc = None if local_center is None else (C.c_double * 3)(*local_center)
        _check(load().tsdf_integrate(self.h, _dev(depth, torch.float32, "depth"), C.byref(pz), lc,
                                     _stream_ptr(stream)))

    def profile(self, capacity: int):
        """Record stage events for the next `capacity` integrate calls (0 = off)."""
        _check(load().tsdf_profile(self.h, int(capacity)))

    def profile_read(self):
        """(summed ms per stage [depth max, alloc, visible, integrate], calls recorded)."""
        ms = (C.c_double * 4)()
        n = C.c_int32()
        _check(load().tsdf_profile_read(self.h, ms, C.byref(n)))
        return list(ms), n.value

    def count(self, stream=None) -> int:
        n = C.c_int64()
        _check(load().tsdf_count(self.h, C.byref(n), _stream_ptr(stream)))
        return n.value

    def listed(self, stream=None) -> int:
        """Blocks on the last integrate call's visible-block list (tsdf_listed)."""
        n = C.c_int64()
        _check(load().tsdf_listed(self.h, C.byref(n), _stream_ptr(stream)))
        return n.value

    def status(self, stream=None) -> int:
        return load().tsdf_status(self.h, _stream_ptr(stream))

    def sync_status(self, stream=None) -> int:
        """ps_sync_status on this handle (same outcome as status())."""
        return load().ps_sync_status(self.h, _stream_ptr(stream))

    def set_partition(self, n_parts: int, part: int):
        """Allocate only the blocks whose key hashes to `part` of n_parts (tsdf_set_partition)."""
        _check(load().tsdf_set_partition(self.h, int(n_parts), int(part)))

    def swap_out(self, local_center, capacity: int = None, device="cuda", stream=None):
        """Move the blocks outside the local map out of the map: (keys, D, W) CUDA tensors."""
        device = _cuda_device(device, "swap_out")
        cap = self.count(stream) if capacity is None else int(capacity)
        keys = torch.empty((max(cap, 1), 3), dtype=torch.int32, device=device)
        D = torch.empty((max(cap, 1), 512), dtype=torch.float32, device=device)
        W = torch.empty((max(cap, 1), 512), dtype=torch.float32, device=device)
        m = C.c_int64()
        lc = (C.c_double * 3)(*local_center)
        _check(load().tsdf_swap_out(self.h, lc, keys.data_ptr(), D.data_ptr(), W.data_ptr(), cap, C.byref(m),
                                    _stream_ptr(stream)))
        return keys[:m.value], D[:m.value], W[:m.value]

    def load_blocks(self, keys: torch.Tensor, D: torch.Tensor, W: torch.Tensor, stream=None):
        """Insert or overwrite blocks (checkpoint resume, swap-in)."""
        n = keys.shape[0]
        _check(load().tsdf_load(self.h, _dev(keys.contiguous(), torch.int32, "keys"),
                                _dev(D.contiguous(), torch.float32, "D"), _dev(W.contiguous(), torch.float32, "W"),
                                n, _stream_ptr(stream)))

    def extract(self, min_weight: float = 0.0, device="cuda", stream=None):
        """(keys (n, 3) int32, D (n, 512), W (n, 512)) as CUDA tensors, in pool order."""
        device = _cuda_device(device, "extract")
        n = self.count(stream)
        keys = torch.empty((max(n, 1), 3), dtype=torch.int32, device=device)
        D = torch.empty((max(n, 1), 512), dtype=torch.float32, device=device)
        W = torch.empty((max(n, 1), 512), dtype=torch.float32, device=device)
        m = C.c_int64()
        _check(load().tsdf_extract(self.h, float(min_weight), keys.data_ptr(), D.data_ptr(), W.data_ptr(), n,
                                   C.byref(m), _stream_ptr(stream)))
        return keys[:m.value], D[:m.value], W[:m.value]


def _tsdf_points(self, min_weight: float = 3.0, device="cuda", stream=None):
    """Surface points (m, 3) float32 and edges (m, 4) int32 (voxel index, axis) as CUDA tensors."""
    device = _cuda_device(device, "points")
    m = C.c_int64()
    st = load().tsdf_extract_points(self.h, float(min_weight), None, None, 0, C.byref(m), _stream_ptr(stream))
    if st not in (PS_OK, PS_ERR_CAPACITY):
        _check(st)
    n = m.value
    pts = torch.empty((max(n, 1), 3), dtype=torch.float32, device=device)
    edges = torch.empty((max(n, 1), 4), dtype=torch.int32, device=device)
    _check(load().tsdf_extract_points(self.h, float(min_weight), pts.data_ptr(), edges.data_ptr(), n, C.byref(m),
                                      _stream_ptr(stream)))
    return pts[:m.value], edges[:m.value]


Tsdf.points = _tsdf_points

STATIC_MAX_BLOCKS = 65536


def tsdf_integrate_dense_static(voxels: torch.Tensor, dims, origin, voxel_size: float, mu: float, w_max: float,
                                depth: torch.Tensor, cam, world_to_cam, stream=None):
    """Fuse one depth map into a caller-owned dense grid without any
    allocation by the library (for callers that cannot allocate while they
    run; the working memory is a fixed static device array).  voxels:
    contiguous CUDA float32 tensor of n_blocks x 512 x 2 ({D, w} pairs);
    depth: float32 cam.height x cam.width.  The C library only sees
    pointers, so the sizes are checked here: a short tensor would be read
    and written past its end."""
    dims = [int(v) for v in dims]
    if len(dims) != 3 or any(v <= 0 or v % 8 for v in dims):
        raise ValueError(f"dims must be three positive multiples of 8, got {dims}")
    n_blocks = (dims[0] // 8) * (dims[1] // 8) * (dims[2] // 8)
    if voxels.numel() != n_blocks * 1024:
        raise ValueError(f"voxels holds {voxels.numel()} floats; dims {dims} need {n_blocks} x 512 x 2")
    if depth.numel() != int(cam.width) * int(cam.height):
        raise ValueError(f"depth holds {depth.numel()} values; the camera is {cam.width} x {cam.height}")
    d = (C.c_int32 * 3)(*dims)
    o = (C.c_double * 3)(*[float(v) for v in origin])
    cz = camera(cam)
    pz = pose(world_to_cam)
    _check(load().tsdf_integrate_dense_static(_dev(voxels, torch.float32, "voxels"), d, o, float(voxel_size),
                                              float(mu), float(w_max), _dev(depth, torch.float32, "depth"),
                                              C.byref(cz), C.byref(pz), _stream_ptr(stream)))


CHECK_BITS = {1: "image gather outside the image", 2: "pixel index outside the image",
              4: "pool slot outside the pool", 8: "work item outside its level or queue"}


def check_read() -> int:
    """Bounds-check failures recorded since the last read (always 0 in the normal build)."""
    b = C.c_uint32()
    _check(load().ps_check_read(C.byref(b)))
    return b.value


def version() -> str:
    return load().ps_version().decode()


# ----------------------------------------------------------------- differentiable forms

def se3_exp_left(xi, p):
    """exp([w]x, v) applied on the left of pose p (R, t): rotation Exp(w) R,
    translation Exp(w) t + v; xi = (w, v)."""
    xi = np.asarray(xi, dtype=np.float64).reshape(6)
    w, v = xi[:3], xi[3:]
    th = float(np.linalg.norm(w))
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    Rw = np.eye(3) if th == 0.0 else np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K
    R = np.asarray(p.R, dtype=np.float64).reshape(3, 3)
    t = np.asarray(p.t, dtype=np.float64).reshape(3)

    class _P:
        pass
    o = _P()
    o.R, o.t = Rw @ R, Rw @ t + v
    return o


class SoftSweep:
    """Soft-argmin depth of one full-resolution level and its gradient
    (psdiff_*): images are float32 CUDA tensors (reference first), poses the
    matching cameras' ref_to_cam."""

    def __init__(self, rig, lv, temperature: float = 0.05):
        L = load()
        self.rig, self.level, self.T = rig, lv, float(temperature)
        self._cams = (ps_camera * len(rig.cams))(*[camera(c) for c in rig.cams])
        d = ps_diff_desc(ref=camera(rig.ref), n_cams=len(rig.cams), cams=self._cams, level=level(lv),
                         temperature=self.T)
        h = C.c_void_p()
        _check(L.psdiff_create(C.byref(d), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().psdiff_destroy(self.h)
            self.h = None

    __del__ = close

    def _args(self, images, poses):
        n = 1 + len(self.rig.cams)
        if len(images) != n:
            raise ValueError(f"expected {n} images")
        ims = (C.c_void_p * n)(*[_dev(im, torch.float32, f"images[{i}]") for i, im in enumerate(images)])
        poses = self.rig.ref_to_cam if poses is None else poses
        ps = (ps_pose * len(poses))(*[pose(p) for p in poses])
        return ims, ps

    def forward(self, images, poses=None, want_aux: bool = True, stream=None):
        """(range, soft-minimum cost, aux) maps; aux feeds backward()."""
        ims, ps = self._args(images, poses)
        H, W = self.rig.ref.height, self.rig.ref.width
        dev = images[0].device
        rng = torch.empty((H, W), dtype=torch.float32, device=dev)
        cost = torch.empty((H, W), dtype=torch.float32, device=dev)
        aux = torch.empty((H, W, 3), dtype=torch.float32, device=dev) if want_aux else None
        _check(load().psdiff_forward(self.h, ims, ps, rng.data_ptr(), cost.data_ptr(),
                                     aux.data_ptr() if aux is not None else None, _stream_ptr(stream)))
        return rng, cost, aux

    def backward(self, images, poses, aux, g_range=None, g_cost=None, stream=None):
        """(per-image gradients, (n_cams, 6) float64 pose gradients (w, v))."""
        ims, ps = self._args(images, poses)
        gi = [torch.zeros_like(im) for im in images]
        gptr = (C.c_void_p * len(gi))(*[g.data_ptr() for g in gi])
        gp = torch.zeros((len(self.rig.cams), 6), dtype=torch.float64, device=images[0].device)
        gr = _dev(g_range.contiguous(), torch.float32, "g_range") if g_range is not None else None
        gc = _dev(g_cost.contiguous(), torch.float32, "g_cost") if g_cost is not None else None
        _check(load().psdiff_backward(self.h, ims, ps, _dev(aux, torch.float32, "aux"), gr, gc, gptr,
                                      gp.data_ptr(), _stream_ptr(stream)))
        return gi, gp


class _SoftDepthFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sweep, base_poses, delta, *images):
        d = delta.detach().cpu().double().numpy().reshape(len(base_poses), 6)
        poses = [se3_exp_left(d[j], p) for j, p in enumerate(base_poses)]
        ims = [im.contiguous() for im in images]
        rng, cost, aux = sweep.forward(ims, poses)
        ctx.sweep, ctx.poses, ctx.delta_meta = sweep, poses, (delta.dtype, delta.device)
        ctx.save_for_backward(aux, *ims)
        return rng, cost

    @staticmethod
    def backward(ctx, g_range, g_cost):
        aux, *ims = ctx.saved_tensors
        gi, gp = ctx.sweep.backward(ims, ctx.poses, aux, g_range, g_cost)
        dt, dev = ctx.delta_meta
        return (None, None, gp.to(dtype=dt, device=dev)) + tuple(gi)


def soft_depth(sweep: SoftSweep, images, delta: Optional[torch.Tensor] = None, base_poses=None):
    """Differentiable (range, soft-minimum cost) maps.  delta: (n_cams, 6)
    left perturbation (w, v) of base_poses (default: the rig's ref_to_cam);
    its gradient is exact at delta = 0 (update the base pose and reset delta
    between steps).  The images receive gradients when they require them."""
    base = list(sweep.rig.ref_to_cam if base_poses is None else base_poses)
    if delta is None:
        delta = torch.zeros((len(base), 6), dtype=torch.float64)
    return _SoftDepthFn.apply(sweep, base, delta, *images)


def tsdf_dense_fuse_backward(voxels_in, dims, origin, voxel_size, mu, w_max, depth, cam, world_to_cam, g_D_out,
                             want_depth: bool = True, want_pose: bool = True, stream=None):
    """(dL/dD_in per voxel, dL/ddepth, (6,) float64 pose gradient) of one fusion step."""
    gD = _dev(g_D_out.contiguous(), torch.float32, "g_D_out")
    gin = torch.empty(g_D_out.shape, dtype=torch.float32, device=voxels_in.device)
    gd = torch.zeros(depth.shape, dtype=torch.float32, device=depth.device) if want_depth else None
    gp = torch.zeros(6, dtype=torch.float64, device=depth.device) if want_pose else None
    dims_a = (C.c_int32 * 3)(*[int(v) for v in dims])
    org = (C.c_double * 3)(*[float(v) for v in origin])
    _check(load().tsdf_dense_fuse_backward(_dev(voxels_in, torch.float32, "voxels_in"), dims_a, org,
                                           float(voxel_size), float(mu), float(w_max),
                                           _dev(depth, torch.float32, "depth"), C.byref(camera(cam)),
                                           C.byref(pose(world_to_cam)), gD, gin.data_ptr(),
                                           gd.data_ptr() if gd is not None else None,
                                           gp.data_ptr() if gp is not None else None, _stream_ptr(stream)))
    return gin, gd, gp


class _DenseFuseFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, grid, base_pose, delta, vox_in, depth):
        dims, origin, vs, mu, w_max, cam = grid
        d = delta.detach().cpu().double().numpy().reshape(6)
        p = se3_exp_left(d, base_pose)
        vin = vox_in.contiguous()
        dep = depth.contiguous()
        out = vin.clone()
        tsdf_integrate_dense_static(out, dims, origin, vs, mu, w_max, dep, cam, p)
        ctx.grid, ctx.pose, ctx.delta_meta = grid, p, (delta.dtype, delta.device)
        ctx.save_for_backward(vin, dep)
        return out

    @staticmethod
    def backward(ctx, g_out):
        vin, dep = ctx.saved_tensors
        dims, origin, vs, mu, w_max, cam = ctx.grid
        gin, gd, gp = tsdf_dense_fuse_backward(vin, dims, origin, vs, mu, w_max, dep, cam, ctx.pose,
                                               g_out[..., 0])
        g_vox = torch.zeros_like(vin)
        g_vox[..., 0] = gin            # weights are observation counts: no gradient
        dt, dev = ctx.delta_meta
        return None, None, gp.to(dtype=dt, device=dev), g_vox, gd


def dense_fuse(voxels: torch.Tensor, depth: torch.Tensor, params, cam, world_to_cam,
               delta: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Differentiable fusion of one depth map into a dense (n_blocks, 512, 2)
    {D, w} grid (params: TsdfParams with dense_dim); out of place.  delta:
    (6,) left perturbation (w, v) of world_to_cam, exact at 0."""
    grid = (tuple(params.dense_dim), tuple(params.origin), params.voxel_size, params.mu, params.w_max, cam)
    if delta is None:
        delta = torch.zeros(6, dtype=torch.float64)
    return _DenseFuseFn.apply(grid, world_to_cam, delta, voxels, depth)
