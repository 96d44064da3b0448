"""FP64 CPU oracle of the fisheye plane-sweep + TSDF fusion path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg, never by the product package.  It
shares no code with the CUDA library; both consume the same seeded inputs
from ``scenes``.

The arithmetic lives in ``oracle.cpp`` (plain double-precision C++ loops,
each function citing the step of the paper it restates).  This module
compiles it on first use (g++, no CUDA) and marshals arguments with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain g++ -O2, IEEE double arithmetic), with
    OpenMP when the compiler has it (the per-pixel arithmetic is the same
    either way; only independent loops are shared among threads)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        base = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-fno-fast-math", _SRC, "-o", tmp]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's independent loops (n <= 0: leave as is);
    returns the count in effect (1 without OpenMP)."""
    return int(lib().orc_set_threads(int(n)))


class OrCamera(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("xi", "fx", "fy", "cx", "cy", "k1", "k2", "p1", "p2", "r2_max")] + \
               [("width", C.c_int32), ("height", C.c_int32)]


class OrPose(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3)]


class OrPlaneSet(C.Structure):
    _fields_ = [("family", C.c_int32), ("count", C.c_int32), ("a", C.c_double), ("b", C.c_double),
                ("n", C.c_double * 3)]


class OrLevel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("factor", C.c_int32), ("crop_w", C.c_int32), ("crop_h", C.c_int32),
                ("window", C.c_int32), ("n_sets", C.c_int32), ("sets", OrPlaneSet * 4)]


class OrFilter(C.Structure):
    _fields_ = [("alpha_upper", C.c_double), ("alpha_lower", C.c_double), ("split_row", C.c_double),
                ("ratio_min", C.c_double), ("gamma", C.c_double), ("delta", C.c_double), ("window", C.c_int32)]


class OrTsdfDesc(C.Structure):
    _fields_ = [("voxel_size", C.c_double), ("mu", C.c_double), ("w_max", C.c_double),
                ("block_dim", C.c_int32), ("dense_dim", C.c_int32 * 3), ("origin", C.c_double * 3),
                ("local_half", C.c_double * 3)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_set_threads.argtypes = [C.c_int32]
            L.orc_set_threads.restype = C.c_int32
            L.orc_project.argtypes = [C.POINTER(OrCamera), _D, _D]
            L.orc_unproject.argtypes = [C.POINTER(OrCamera), C.c_double, C.c_double, _D]
            L.orc_distort.argtypes = [C.POINTER(OrCamera), C.c_double, C.c_double, _D]
            L.orc_undistort.argtypes = [C.POINTER(OrCamera), C.c_double, C.c_double, _D]
            L.orc_zncc.argtypes = [_D, _D, C.c_int32, _D]
            L.orc_level_planes.argtypes = [C.POINTER(OrLevel), _D, _D, _P, _P]
            L.orc_level_planes.restype = C.c_int32
            L.orc_level_ref.argtypes = [C.POINTER(OrCamera), C.POINTER(OrLevel), _P, C.POINTER(OrCamera), _D]
            L.orc_warped_sample.argtypes = [C.POINTER(OrCamera), C.c_int32, C.POINTER(OrCamera),
                                            C.POINTER(OrPose), C.POINTER(OrLevel), _P, C.c_int32, C.c_int32,
                                            C.c_int32, C.c_int32, _D]
            L.orc_sweep_level.argtypes = [C.POINTER(OrCamera), C.c_int32, C.POINTER(OrCamera), C.POINTER(OrPose),
                                          C.POINTER(OrLevel), _P, C.c_int64, _P, _D, _D, _D, _P, _D]
            L.orc_sweep_level.restype = C.c_int64
            L.orc_wta.argtypes = [_D, C.c_int32, C.c_int32, _P, _P, _D]
            L.orc_merge.argtypes = [C.c_int32, C.c_int32, _D, C.c_int32, _D, C.c_int32, C.c_int32, _P,
                                    C.c_int32, _D]
            L.orc_filter_frame.argtypes = [C.c_int32, C.c_int32, _D, _D, _D, C.c_int32, _D, _D, _D, C.c_int32,
                                           C.c_int32, C.POINTER(OrFilter), _P, C.c_int32, _D, _P]
            L.orc_tsdf_new.argtypes = [C.POINTER(OrTsdfDesc)]
            L.orc_tsdf_new.restype = C.c_void_p
            L.orc_tsdf_free.argtypes = [_P]
            L.orc_tsdf_set_bands.argtypes = [_P, C.c_double, C.c_double, C.c_double, C.c_double]
            L.orc_tsdf_integrate.argtypes = [_P, _P, C.POINTER(OrCamera), C.POINTER(OrPose), _D]
            L.orc_tsdf_count.argtypes = [_P]
            L.orc_tsdf_count.restype = C.c_int64
            L.orc_tsdf_dump.argtypes = [_P, _P, _D, _D, _P]
            L.orc_tsdf_alloc_counts.argtypes = [_P, _P, _P]
            L.orc_tsdf_alloc_sets.argtypes = [_P, _P, _P]
            L.orc_tsdf_swap_out.argtypes = [_P, _D, _P, _D, _D, _P, _P]
            L.orc_tsdf_swap_out.restype = C.c_int64
            L.orc_tsdf_load.argtypes = [_P, C.c_int64, _P, _D, _D]
            L.orc_tsdf_ever_maybe.argtypes = [_P, _P]
            L.orc_tsdf_ever_maybe.restype = C.c_int64
            L.orc_tsdf_points.argtypes = [C.c_int64, _P, _D, _D, C.c_double, _D, C.c_double, C.c_int64, _D, _P]
            L.orc_tsdf_points.restype = C.c_int64
            L.orc_project_jacobian.argtypes = [C.POINTER(OrCamera), _D, _D]
            L.orc_soft_argmin.argtypes = [_D, _D, C.c_int32, C.c_double, _D, _D, _D]
            L.orc_soft_depth.argtypes = [C.POINTER(OrCamera), C.c_int32, C.POINTER(OrCamera), C.POINTER(OrPose),
                                         C.POINTER(OrLevel), _P, C.c_double, _D, _D]
            L.orc_soft_depth_grad.argtypes = [C.POINTER(OrCamera), C.c_int32, C.POINTER(OrCamera),
                                              C.POINTER(OrPose), C.POINTER(OrLevel), _P, C.c_double, _D, _D, _P,
                                              _D]
            L.orc_soft_depth_ties.argtypes = [C.POINTER(OrCamera), C.c_int32, C.POINTER(OrCamera),
                                              C.POINTER(OrPose), C.POINTER(OrLevel), _P, C.c_double, C.c_double,
                                              _P]
            L.orc_dense_fuse.argtypes = [_P, _D, C.c_double, C.c_double, C.c_double, _D, _P, C.POINTER(OrCamera),
                                         C.POINTER(OrPose), _D]
            L.orc_dense_fuse_grad.argtypes = [_P, _D, C.c_double, C.c_double, C.c_double, _D, _P,
                                              C.POINTER(OrCamera), C.POINTER(OrPose), _D, _D, _D, _D]
            _lib = L
    return _lib


# ----------------------------------------------------------------- marshalling

def camera(c) -> OrCamera:
    return OrCamera(xi=c.xi, fx=c.fx, fy=c.fy, cx=c.cx, cy=c.cy, k1=c.k1, k2=c.k2, p1=c.p1, p2=c.p2,
                    r2_max=min(c.r2_max, 1e300), width=c.width, height=c.height)


def pose(p) -> OrPose:
    o = OrPose()
    for i, v in enumerate(np.asarray(p.R, dtype=np.float64).reshape(-1)):
        o.R[i] = v
    for i, v in enumerate(np.asarray(p.t, dtype=np.float64).reshape(-1)):
        o.t[i] = v
    return o


def level(lv) -> OrLevel:
    o = OrLevel(kind=lv.kind, factor=lv.factor, crop_w=lv.crop_w, crop_h=lv.crop_h, window=lv.window,
                n_sets=len(lv.sets))
    assert len(lv.sets) <= 4
    for i, s in enumerate(lv.sets):
        o.sets[i].family = s.family
        o.sets[i].count = s.count
        o.sets[i].a = s.a
        o.sets[i].b = s.b
        for k in range(3):
            o.sets[i].n[k] = s.n[k]
    return o


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _images(imgs: Sequence[np.ndarray]):
    arrs = [np.ascontiguousarray(np.asarray(i, dtype=np.uint8)) for i in imgs]
    ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return arrs, ptrs


# ----------------------------------------------------------------- camera

def project(cam, X) -> Optional[np.ndarray]:
    X = np.ascontiguousarray(X, dtype=np.float64)
    uv = np.zeros(2)
    ok = lib().orc_project(C.byref(camera(cam)), _dptr(X), _dptr(uv))
    return uv if ok else None


def unproject(cam, u: float, v: float) -> Optional[np.ndarray]:
    r = np.zeros(3)
    ok = lib().orc_unproject(C.byref(camera(cam)), u, v, _dptr(r))
    return r if ok else None


def distort(cam, x: float, y: float) -> np.ndarray:
    o = np.zeros(2)
    lib().orc_distort(C.byref(camera(cam)), x, y, _dptr(o))
    return o


def undistort(cam, xd: float, yd: float) -> Optional[np.ndarray]:
    o = np.zeros(2)
    ok = lib().orc_undistort(C.byref(camera(cam)), xd, yd, _dptr(o))
    return o if ok else None


def zncc(a, b) -> Optional[float]:
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    out = np.zeros(1)
    ok = lib().orc_zncc(_dptr(a), _dptr(b), a.size, _dptr(out))
    return float(out[0]) if ok else None


# ----------------------------------------------------------------- sweep

def level_planes(lv):
    K = lv.n_planes
    n = np.zeros((K, 3))
    d = np.zeros(K)
    s = np.zeros(K, dtype=np.int32)
    loc = np.zeros(K, dtype=np.int32)
    lib().orc_level_planes(C.byref(level(lv)), _dptr(n), _dptr(d), s.ctypes.data, loc.ctypes.data)
    return n, d, s, loc


def level_ref(ref_cam, lv, ref_img):
    """(level camera as OrCamera, level reference image float64 in [0,1])."""
    if lv.kind == 0:
        W, H = ref_cam.width // lv.factor, ref_cam.height // lv.factor
    else:
        W, H = lv.crop_w, lv.crop_h
    out = np.zeros((H, W))
    oc = OrCamera()
    img = np.ascontiguousarray(ref_img, dtype=np.uint8)
    lib().orc_level_ref(C.byref(camera(ref_cam)), C.byref(level(lv)), img.ctypes.data, C.byref(oc), _dptr(out))
    return oc, out


def level_shape(rig, lv):
    if lv.kind == 0:
        return rig.ref.height // lv.factor, rig.ref.width // lv.factor
    return lv.crop_h, lv.crop_w


def warped_sample(rig, lv, imgs, j: int, k: int, qx: int, qy: int) -> Optional[float]:
    cams = (OrCamera * len(rig.cams))(*[camera(c) for c in rig.cams])
    poses = (OrPose * len(rig.cams))(*[pose(p) for p in rig.ref_to_cam])
    arrs, ptrs = _images(imgs)
    w = np.zeros(1)
    ok = lib().orc_warped_sample(C.byref(camera(rig.ref)), len(rig.cams), cams, poses, C.byref(level(lv)),
                                 C.cast(ptrs, C.c_void_p), j, k, qx, qy, _dptr(w))
    return float(w[0]) if ok else None


def sweep_level(rig, lv, imgs, pix: Optional[np.ndarray] = None, want_costs: bool = False):
    """Sweep one level.  pix: (n, 2) int (x, y) level coordinates or None for
    all pixels.  Returns dict(depth, c1, c2, kstar[, costs]) shaped (H, W)
    for the whole level or (n,) for a pixel list."""
    H, W = level_shape(rig, lv)
    n = H * W if pix is None else int(len(pix))
    K = lv.n_planes
    depth = np.zeros(n)
    c1 = np.zeros(n)
    c2 = np.zeros(n)
    ks = np.zeros(n, dtype=np.int32)
    costs = np.zeros((n, K)) if want_costs else None
    cams = (OrCamera * len(rig.cams))(*[camera(c) for c in rig.cams])
    poses = (OrPose * len(rig.cams))(*[pose(p) for p in rig.ref_to_cam])
    arrs, ptrs = _images(imgs)
    pixa = None if pix is None else np.ascontiguousarray(pix, dtype=np.int32)
    lib().orc_sweep_level(C.byref(camera(rig.ref)), len(rig.cams), cams, poses, C.byref(level(lv)),
                          C.cast(ptrs, C.c_void_p), n, None if pixa is None else pixa.ctypes.data,
                          _dptr(depth), _dptr(c1), _dptr(c2), ks.ctypes.data,
                          _dptr(costs) if costs is not None else None)
    out = dict(depth=depth, c1=c1, c2=c2, kstar=ks)
    if costs is not None:
        out["costs"] = costs
    if pix is None:
        out = {k: (v.reshape(H, W) if k != "costs" else v.reshape(H, W, K)) for k, v in out.items()}
    return out


def wta(costs, counts):
    """Winner-take-all + parabola step alone: (kstar, c1, c2, delta)."""
    Cc = np.ascontiguousarray(costs, dtype=np.float64)
    cn = np.ascontiguousarray(counts, dtype=np.int32)
    ks = np.zeros(1, dtype=np.int32)
    out = np.zeros(3)
    lib().orc_wta(_dptr(Cc), Cc.size, cn.size, cn.ctypes.data, ks.ctypes.data, _dptr(out))
    return int(ks[0]), float(out[0]), float(out[1]), float(out[2])


def merge(W: int, H: int, low: Optional[np.ndarray], s: int, crop: Optional[np.ndarray], crop_w: int, crop_h: int,
          boxes: Optional[np.ndarray]) -> np.ndarray:
    out = np.zeros((H, W))
    lo = None if low is None else np.ascontiguousarray(low, dtype=np.float64)
    cr = None if crop is None else np.ascontiguousarray(crop, dtype=np.float64)
    bx = np.ascontiguousarray(boxes if boxes is not None else np.zeros((0, 4)), dtype=np.int32)
    lib().orc_merge(W, H, _dptr(lo) if lo is not None else None, s, _dptr(cr) if cr is not None else None,
                    crop_w, crop_h, bx.ctypes.data, len(bx), _dptr(out))
    return out


def filter_params(f) -> OrFilter:
    return OrFilter(alpha_upper=f.alpha_upper, alpha_lower=f.alpha_lower, split_row=f.split_row,
                    ratio_min=f.ratio_min, gamma=f.gamma, delta=f.delta, window=f.window)


def filter_frame(W, H, low=None, s=1, crop=None, crop_w=0, crop_h=0, params=None, boxes=None):
    """Depth filtering, merge and masks at full resolution.  low / crop: dicts
    with depth, c1, c2 arrays of their level.  Returns (depth, ambiguous)."""
    out = np.zeros((H, W))
    amb = np.zeros((H, W), dtype=np.uint8)
    f = filter_params(params)

    def arrs(d):
        if d is None:
            return None, None, None
        return tuple(np.ascontiguousarray(d[k], dtype=np.float64) for k in ("depth", "c1", "c2"))

    ld, l1, l2 = arrs(low)
    cd, k1, k2 = arrs(crop)
    bx = np.ascontiguousarray(boxes if boxes is not None else np.zeros((0, 4)), dtype=np.int32)
    p = lambda a: _dptr(a) if a is not None else None  # noqa: E731
    lib().orc_filter_frame(W, H, p(ld), p(l1), p(l2), s, p(cd), p(k1), p(k2), crop_w, crop_h, C.byref(f),
                           bx.ctypes.data, len(bx), _dptr(out), amb.ctypes.data)
    return out, amb.astype(bool)


def depth_frame(wl, imgs, boxes=None):
    """Whole-frame depth of a workload (every level swept at every pixel,
    then merged and masked): dict(depth (H, W), levels [per-level dicts])."""
    rig = wl.rig
    levels = [sweep_level(rig, lv, imgs) for lv in wl.levels]
    low = crop = None
    s = 1
    cw = ch = 0
    for lv, res in zip(wl.levels, levels):
        if lv.kind == 0:
            low, s = res["depth"], lv.factor
        else:
            crop, cw, ch = res["depth"], lv.crop_w, lv.crop_h
    D = merge(rig.ref.width, rig.ref.height, low, s, crop, cw, ch, boxes)
    out = dict(depth=D, levels=levels)
    flt = getattr(wl, "filters", None)
    if flt is not None and flt.enable:
        lo = cr = None
        for lv, res in zip(wl.levels, levels):
            if lv.kind == 0:
                lo = res
            else:
                cr = res
        out["filtered"], out["filtered_amb"] = filter_frame(rig.ref.width, rig.ref.height, lo, s, cr, cw, ch, flt,
                                                             boxes)
    return out


# ----------------------------------------------------------------- TSDF

class Tsdf:
    """FP64 TSDF map (brute-force integration over every allocated voxel)."""

    def __init__(self, params, bands=None):
        p = params
        d = OrTsdfDesc(voxel_size=p.voxel_size, mu=p.mu, w_max=p.w_max, block_dim=p.block_dim)
        if p.dense_dim is not None:
            for i in range(3):
                d.dense_dim[i] = p.dense_dim[i]
        for i in range(3):
            d.origin[i] = p.origin[i]
            d.local_half[i] = p.local_half[i] if p.local_half is not None else 0.0
        self.params = p
        self.h = lib().orc_tsdf_new(C.byref(d))
        if bands is not None:
            lib().orc_tsdf_set_bands(self.h, *bands)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_tsdf_free(self.h)
            self.h = None

    def integrate(self, depth: np.ndarray, cam, world_to_cam, local_center=None):
        dep = np.ascontiguousarray(depth, dtype=np.float32)
        lc = None if local_center is None else np.ascontiguousarray(local_center, dtype=np.float64)
        lib().orc_tsdf_integrate(self.h, dep.ctypes.data, C.byref(camera(cam)), C.byref(pose(world_to_cam)),
                                 _dptr(lc) if lc is not None else None)

    def dump(self):
        """(keys (n, 3) int64 sorted, D (n, B^3), W (n, B^3), amb (n, B^3) bool)."""
        n = lib().orc_tsdf_count(self.h)
        B3 = self.params.block_dim ** 3
        keys = np.zeros((n, 3), dtype=np.int64)
        D = np.zeros((n, B3))
        W = np.zeros((n, B3))
        amb = np.zeros((n, B3), dtype=np.uint8)
        lib().orc_tsdf_dump(self.h, keys.ctypes.data, _dptr(D), _dptr(W), amb.ctypes.data)
        return keys, D, W, amb.astype(bool)

    def alloc_sets(self):
        ns = np.zeros(1, dtype=np.int64)
        nm = np.zeros(1, dtype=np.int64)
        lib().orc_tsdf_alloc_counts(self.h, ns.ctypes.data, nm.ctypes.data)
        s = np.zeros((int(ns[0]), 3), dtype=np.int64)
        m = np.zeros((int(nm[0]), 3), dtype=np.int64)
        lib().orc_tsdf_alloc_sets(self.h, s.ctypes.data, m.ctypes.data)
        return s, m

    def swap_out(self, local_center):
        """Remove the blocks outside the local map: (keys, D, W, ambiguous keys)."""
        lc = np.ascontiguousarray(local_center, dtype=np.float64)
        n = lib().orc_tsdf_count(self.h)
        B3 = self.params.block_dim ** 3
        keys = np.zeros((n, 3), dtype=np.int64)
        D = np.zeros((n, B3))
        W = np.zeros((n, B3))
        na = np.zeros(1, dtype=np.int64)
        amb = np.zeros((n, 3), dtype=np.int64)
        m = lib().orc_tsdf_swap_out(self.h, _dptr(lc), keys.ctypes.data, _dptr(D), _dptr(W), na.ctypes.data,
                                    amb.ctypes.data)
        return keys[:m], D[:m], W[:m], amb[:int(na[0])]

    def load(self, keys, D, W):
        keys = np.ascontiguousarray(keys, dtype=np.int64)
        D = np.ascontiguousarray(D, dtype=np.float64)
        W = np.ascontiguousarray(W, dtype=np.float64)
        lib().orc_tsdf_load(self.h, len(keys), keys.ctypes.data, _dptr(D), _dptr(W))

    def ever_maybe(self):
        n = lib().orc_tsdf_ever_maybe(self.h, None)
        k = np.zeros((n, 3), dtype=np.int64)
        lib().orc_tsdf_ever_maybe(self.h, k.ctypes.data)
        return k


# ----------------------------------------------------------------- differentiable forms

def project_jacobian(cam, X) -> np.ndarray:
    """d(u, v)/dX of the unified projection with distortion (2 x 3)."""
    J = np.zeros(6)
    X = np.ascontiguousarray(X, dtype=np.float64)
    lib().orc_project_jacobian(C.byref(camera(cam)), _dptr(X), _dptr(J))
    return J.reshape(2, 3)


def soft_argmin(costs, rho, T: float):
    """(weights s, E = sum s rho, soft minimum S) of one pixel; None when no cost is finite."""
    c = np.ascontiguousarray(costs, dtype=np.float64)
    r = np.ascontiguousarray(rho, dtype=np.float64)
    s = np.zeros(len(c))
    E, S = C.c_double(), C.c_double()
    ok = lib().orc_soft_argmin(_dptr(c), _dptr(r), len(c), T, _dptr(s), C.byref(E), C.byref(S))
    return (s, E.value, S.value) if ok else None


def _real_images(images):
    arrs = [np.ascontiguousarray(i, dtype=np.float64) for i in images]
    ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return arrs, ptrs


def soft_depth(rig, lv, images, T: float = 0.05, poses=None, with_cost: bool = False):
    """Soft-argmin range map of one full-resolution level of real-valued images
    (and the soft-minimum cost map with with_cost)."""
    poses = rig.ref_to_cam if poses is None else poses
    cams = (OrCamera * len(rig.cams))(*[camera(c) for c in rig.cams])
    ps = (OrPose * len(rig.cams))(*[pose(p) for p in poses])
    arrs, ptrs = _real_images(images)
    out = np.zeros((rig.ref.height, rig.ref.width))
    cost = np.zeros_like(out)
    lib().orc_soft_depth(C.byref(camera(rig.ref)), len(rig.cams), cams, ps, C.byref(level(lv)), ptrs, T,
                         _dptr(out), _dptr(cost))
    return (out, cost) if with_cost else out


def soft_depth_grad(rig, lv, images, g, T: float = 0.05, poses=None, g_cost=None):
    """Gradient of sum(g * range) + sum(g_cost * S): (per-image gradients, (n_cams, 6) pose
    gradients (w, v)).  g may be None."""
    poses = rig.ref_to_cam if poses is None else poses
    cams = (OrCamera * len(rig.cams))(*[camera(c) for c in rig.cams])
    ps = (OrPose * len(rig.cams))(*[pose(p) for p in poses])
    arrs, ptrs = _real_images(images)
    gi = [np.zeros_like(a) for a in arrs]
    gptr = (C.c_void_p * len(gi))(*[a.ctypes.data for a in gi])
    gp = np.zeros((len(rig.cams), 6))
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
    gs = None if g_cost is None else np.ascontiguousarray(g_cost, dtype=np.float64)
    lib().orc_soft_depth_grad(C.byref(camera(rig.ref)), len(rig.cams), cams, ps, C.byref(level(lv)), ptrs, T,
                              None if gg is None else _dptr(gg), None if gs is None else _dptr(gs), gptr, _dptr(gp))
    return gi, gp


def soft_depth_ties(rig, lv, images, tau: float = 1e-5, tau_px: float = 0.0, poses=None) -> np.ndarray:
    """Pixels where some valid plane's two lowest camera costs lie within tau,
    or (tau_px > 0) a winning window sample lies within tau_px of a pixel-grid line."""
    poses = rig.ref_to_cam if poses is None else poses
    cams = (OrCamera * len(rig.cams))(*[camera(c) for c in rig.cams])
    ps = (OrPose * len(rig.cams))(*[pose(p) for p in poses])
    arrs, ptrs = _real_images(images)
    amb = np.zeros((rig.ref.height, rig.ref.width), np.uint8)
    lib().orc_soft_depth_ties(C.byref(camera(rig.ref)), len(rig.cams), cams, ps, C.byref(level(lv)), ptrs, tau,
                              tau_px, amb.ctypes.data)
    return amb.astype(bool)


def dense_fuse(vox, nb, origin, voxel, mu, w_max, depth, cam, w2c) -> np.ndarray:
    """Fusion of one depth map into a dense grid; vox: (n_blocks, 512, 2) {D, w}."""
    vin = np.ascontiguousarray(vox, dtype=np.float64)
    out = np.empty_like(vin)
    nbv = np.ascontiguousarray(nb, dtype=np.int32)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    d = np.ascontiguousarray(depth, dtype=np.float32)
    lib().orc_dense_fuse(nbv.ctypes.data, _dptr(o), voxel, mu, w_max, _dptr(vin), d.ctypes.data,
                         C.byref(camera(cam)), C.byref(pose(w2c)), _dptr(out))
    return out


def dense_fuse_grad(vox, nb, origin, voxel, mu, w_max, depth, cam, w2c, gD):
    """Gradient of sum(gD * D_out): (dD_in (n_blocks, 512), d depth (H, W), pose (6,) as (w, v))."""
    vin = np.ascontiguousarray(vox, dtype=np.float64)
    nbv = np.ascontiguousarray(nb, dtype=np.int32)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    d = np.ascontiguousarray(depth, dtype=np.float32)
    g = np.ascontiguousarray(gD, dtype=np.float64)
    gin = np.zeros(g.shape)
    gd = np.zeros(d.shape)
    gp = np.zeros(6)
    lib().orc_dense_fuse_grad(nbv.ctypes.data, _dptr(o), voxel, mu, w_max, _dptr(vin), d.ctypes.data,
                              C.byref(camera(cam)), C.byref(pose(w2c)), _dptr(g), _dptr(gin), _dptr(gd), _dptr(gp))
    return gin, gd, gp


def tsdf_points(keys, D, W, min_w, origin, voxel):
    """Surface points of a block map: (points (m, 3) float64, edges (m, 4) int32: voxel index, axis)."""
    k = np.ascontiguousarray(keys, dtype=np.int32).reshape(-1, 3)
    d = np.ascontiguousarray(D, dtype=np.float64).reshape(-1, 512)
    w = np.ascontiguousarray(W, dtype=np.float64).reshape(-1, 512)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    L = lib()
    m = L.orc_tsdf_points(len(k), k.ctypes.data, _dptr(d), _dptr(w), float(min_w), _dptr(o), float(voxel), 0, None,
                          None)
    pts = np.zeros((max(m, 1), 3))
    edges = np.zeros((max(m, 1), 4), np.int32)
    L.orc_tsdf_points(len(k), k.ctypes.data, _dptr(d), _dptr(w), float(min_w), _dptr(o), float(voxel), m, _dptr(pts),
                      edges.ctypes.data)
    return pts[:m], edges[:m]
