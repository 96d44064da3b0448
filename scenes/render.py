"""Seeded synthetic fisheye scenes: the inputs that the tests, the oracle checks
and the benchmark all share.

This module synthesises inputs only.  It holds none of the mapping method's
arithmetic (no plane warp, no matching cost, no depth selection, no TSDF
update).  It does need a fisheye camera to render images, and it models that
camera on its own terms so that it can act as an independent check of the
method's back-projection (Eq. 1): a pixel's viewing ray is found here by
bisection on the polar angle of the unified (Mei) sphere model, and lens
distortion is inverted by fixed-point iteration.  Neither step shares code or
formulas with the oracle or with the CUDA library.

Everything is float64 torch tensor code that runs on the CPU or, for the
full-size workloads, on a CUDA device (torch ops only; the product kernels are
not involved).  Random draws come from ``numpy.random.default_rng(seed)``;
texture noise comes from a counter-based integer hash so that it needs no
stored texture.

Conventions: camera frame x right, y down, z forward; world frame likewise
(the ground is the plane y = +height below a camera at y = 0).  A pose (R, t)
maps source coordinates to destination coordinates, X_dst = R X_src + t.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

SKY = 128          # constant (hence featureless) intensity of rays that hit nothing
OUTSIDE = 0        # intensity of pixels that no viewing ray passes through


@dataclass
class Camera:
    """Unified omnidirectional camera with radial-tangential distortion.

    ``r2_max`` bounds the squared radius of undistorted normalised coordinates
    that the camera accepts; it keeps the distortion polynomial on a range
    where it is one-to-one.
    """
    xi: float
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    k1: float = 0.0
    k2: float = 0.0
    p1: float = 0.0
    p2: float = 0.0
    r2_max: float = 1e30


@dataclass
class Pose:
    """Rigid transform X_dst = R X_src + t (R row-major 3x3, t 3-vector)."""
    R: np.ndarray
    t: np.ndarray

    @staticmethod
    def identity() -> "Pose":
        return Pose(np.eye(3), np.zeros(3))

    def inverse(self) -> "Pose":
        Rt = self.R.T
        return Pose(Rt.copy(), -Rt @ self.t)

    def compose(self, other: "Pose") -> "Pose":
        """self after other: X -> self(other(X))."""
        return Pose(self.R @ other.R, self.R @ other.t + self.t)


def rot_xyz(ax: float, ay: float, az: float) -> np.ndarray:
    """Rotation from small angles (radians) about x, then y, then z."""
    cx, sx = math.cos(ax), math.sin(ax)
    cy, sy = math.cos(ay), math.sin(ay)
    cz, sz = math.cos(az), math.sin(az)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


# --------------------------------------------------------------------------
# scene primitives (world frame)
# --------------------------------------------------------------------------

@dataclass
class Plane:
    """Infinite plane n . X = h, textured in the (e1, e2) frame."""
    n: Tuple[float, float, float]
    h: float
    e1: Tuple[float, float, float]
    e2: Tuple[float, float, float]
    texel: float
    tex_id: int


@dataclass
class Rect:
    """Finite rectangle centred at c spanned by unit axes e1, e2 (half sizes a, b)."""
    c: Tuple[float, float, float]
    e1: Tuple[float, float, float]
    e2: Tuple[float, float, float]
    a: float
    b: float
    texel: float
    tex_id: int


@dataclass
class Box:
    """Axis-aligned box [lo, hi]; each face textured with tex_id*8 + face."""
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    texel: float
    tex_id: int


@dataclass
class Scene:
    planes: List[Plane] = field(default_factory=list)
    rects: List[Rect] = field(default_factory=list)
    boxes: List[Box] = field(default_factory=list)
    seed: int = 0


# --------------------------------------------------------------------------
# counter-based texture noise
# --------------------------------------------------------------------------

_M32 = 0xFFFFFFFF


def _hash32(a: torch.Tensor) -> torch.Tensor:
    """32-bit integer finaliser on int64 tensors holding values in [0, 2^32)."""
    a = a & _M32
    a = a ^ (a >> 16)
    a = (a * 0x7FEB352D) & _M32
    a = a ^ (a >> 15)
    a = (a * 0x446CA68B) & _M32
    a = a ^ (a >> 16)
    return a


def _noise(tex_id: torch.Tensor, ix: torch.Tensor, iy: torch.Tensor, seed: int) -> torch.Tensor:
    h = _hash32(tex_id * 0x2545F491 + (seed & _M32))
    h = _hash32(h ^ ((ix & _M32) * 0x1B873593 & _M32))
    h = _hash32(h ^ ((iy & _M32) * 0x5BD1E995 & _M32))
    return (h & 0xFFFFFF).to(torch.float64) / float(1 << 24)


def texture(tex_id: torch.Tensor, s: torch.Tensor, t: torch.Tensor, texel: torch.Tensor,
            seed: int) -> torch.Tensor:
    """Bilinearly interpolated value noise in [0.1, 0.9] at surface coords (s, t)."""
    gs = s / texel - 0.5
    gt = t / texel - 0.5
    i0 = torch.floor(gs)
    j0 = torch.floor(gt)
    fs = gs - i0
    ft = gt - j0
    i0 = i0.to(torch.int64)
    j0 = j0.to(torch.int64)
    n00 = _noise(tex_id, i0, j0, seed)
    n10 = _noise(tex_id, i0 + 1, j0, seed)
    n01 = _noise(tex_id, i0, j0 + 1, seed)
    n11 = _noise(tex_id, i0 + 1, j0 + 1, seed)
    v = (1 - ft) * ((1 - fs) * n00 + fs * n10) + ft * ((1 - fs) * n01 + fs * n11)
    return 0.1 + 0.8 * v


# --------------------------------------------------------------------------
# camera: pixel -> viewing ray, by the renderer's own route
# --------------------------------------------------------------------------

def _undistort_fixed_point(cam: Camera, xd: torch.Tensor, yd: torch.Tensor, iters: int = 80):
    """Invert the radial-tangential model by fixed-point iteration."""
    x = xd.clone()
    y = yd.clone()
    for _ in range(iters):
        r2 = x * x + y * y
        radial = 1 + cam.k1 * r2 + cam.k2 * r2 * r2
        tx = 2 * cam.p1 * x * y + cam.p2 * (r2 + 2 * x * x)
        ty = cam.p1 * (r2 + 2 * y * y) + 2 * cam.p2 * x * y
        x = (xd - tx) / radial
        y = (yd - ty) / radial
    return x, y


def pixel_rays(cam: Camera, u: torch.Tensor, v: torch.Tensor, iters: int = 64):
    """Unit viewing rays (camera frame) of pixel positions (u, v).

    The sphere model maps a direction at polar angle theta to normalised
    radius rho = sin(theta) / (cos(theta) + xi); that map increases on the
    admissible range of theta, so theta is found by bisection.  Returns
    (rays [..., 3], valid [...]).
    """
    u = torch.as_tensor(u).to(torch.float64)
    v = torch.as_tensor(v).to(torch.float64)
    xd = (u - cam.cx) / cam.fx
    yd = (v - cam.cy) / cam.fy
    x, y = _undistort_fixed_point(cam, xd, yd)
    rho = torch.sqrt(x * x + y * y)
    phi = torch.atan2(y, x)
    xi = cam.xi
    lim = min(xi, 1.0 / xi) if xi > 0 else 0.0
    theta_b = math.acos(-lim)
    lo = torch.zeros_like(rho)
    hi = torch.full_like(rho, theta_b)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        g = torch.sin(mid) - rho * (torch.cos(mid) + xi)
        pos = g > 0
        hi = torch.where(pos, mid, hi)
        lo = torch.where(pos, lo, mid)
    theta = 0.5 * (lo + hi)
    valid = torch.ones_like(rho, dtype=torch.bool)
    if xi > 1.0:
        rho_max = math.sin(theta_b) / (math.cos(theta_b) + xi)
        valid &= rho <= rho_max
    valid &= (x * x + y * y) <= cam.r2_max
    st = torch.sin(theta)
    rays = torch.stack([st * torch.cos(phi), st * torch.sin(phi), torch.cos(theta)], dim=-1)
    return rays, valid


def forward_project(cam: Camera, X: np.ndarray) -> Tuple[float, float]:
    """Pixel of camera-frame point X by the textbook sphere model (renderer use only)."""
    Xs = X / np.linalg.norm(X)
    mx = Xs[0] / (Xs[2] + cam.xi)
    my = Xs[1] / (Xs[2] + cam.xi)
    r2 = mx * mx + my * my
    radial = 1 + cam.k1 * r2 + cam.k2 * r2 * r2
    xd = mx * radial + 2 * cam.p1 * mx * my + cam.p2 * (r2 + 2 * mx * mx)
    yd = my * radial + cam.p1 * (r2 + 2 * my * my) + 2 * cam.p2 * mx * my
    return cam.fx * xd + cam.cx, cam.fy * yd + cam.cy


# --------------------------------------------------------------------------
# ray casting
# --------------------------------------------------------------------------

def _vec(t, device):
    return torch.tensor(t, dtype=torch.float64, device=device)


def cast(scene: Scene, origin: torch.Tensor, dirs: torch.Tensor):
    """Nearest hit of rays origin + s*dirs (s > 0).

    Returns (s [N], value [N]) with s = inf and value = SKY/255 where nothing is hit.
    """
    dev = dirs.device
    N = dirs.shape[0]
    best = torch.full((N,), math.inf, dtype=torch.float64, device=dev)
    val = torch.full((N,), SKY / 255.0, dtype=torch.float64, device=dev)
    eps = 1e-9

    def take(s, hit, tex_id, su, sv, texel):
        nonlocal best, val
        upd = hit & (s > eps) & (s < best)
        if not bool(upd.any()):
            return
        idx = upd.nonzero(as_tuple=True)[0]
        tid = tex_id[idx] if torch.is_tensor(tex_id) else torch.full_like(idx, tex_id)
        tx = texel[idx] if torch.is_tensor(texel) else torch.full(
            (idx.numel(),), float(texel), dtype=torch.float64, device=dev)
        best[idx] = s[idx]
        val[idx] = texture(tid, su[idx], sv[idx], tx, scene.seed)

    for pl in scene.planes:
        n = _vec(pl.n, dev)
        nd = dirs @ n
        s = (pl.h - origin @ n) / torch.where(nd.abs() > 1e-15, nd, torch.full_like(nd, 1e-15))
        P = origin[None, :] + s[:, None] * dirs
        take(s, nd.abs() > 1e-15, pl.tex_id, P @ _vec(pl.e1, dev), P @ _vec(pl.e2, dev), pl.texel)

    for rc in scene.rects:
        e1 = _vec(rc.e1, dev)
        e2 = _vec(rc.e2, dev)
        n = torch.linalg.cross(e1, e2)
        c = _vec(rc.c, dev)
        nd = dirs @ n
        ok = nd.abs() > 1e-15
        s = ((c - origin) @ n) / torch.where(ok, nd, torch.full_like(nd, 1e-15))
        P = origin[None, :] + s[:, None] * dirs - c[None, :]
        a = P @ e1
        b = P @ e2
        ok = ok & (a.abs() <= rc.a) & (b.abs() <= rc.b)
        take(s, ok, rc.tex_id, a, b, rc.texel)

    if scene.boxes:
        # all boxes at once: slab test of every ray against every box
        lo = torch.tensor([b.lo for b in scene.boxes], dtype=torch.float64, device=dev)   # (M, 3)
        hi = torch.tensor([b.hi for b in scene.boxes], dtype=torch.float64, device=dev)
        texel = torch.tensor([b.texel for b in scene.boxes], dtype=torch.float64, device=dev)
        tid = torch.tensor([b.tex_id for b in scene.boxes], dtype=torch.int64, device=dev)
        inv = 1.0 / torch.where(dirs.abs() > 1e-15, dirs, torch.full_like(dirs, 1e-15))  # (N, 3)
        t0 = (lo[None, :, :] - origin[None, None, :]) * inv[:, None, :]                    # (N, M, 3)
        t1 = (hi[None, :, :] - origin[None, None, :]) * inv[:, None, :]
        tmin = torch.minimum(t0, t1)
        tmax = torch.maximum(t0, t1)
        del t0, t1
        tenter, axis = tmin.max(dim=2)                                                   # (N, M)
        texit = tmax.min(dim=2).values
        del tmin, tmax
        hit = (tenter <= texit) & (tenter > eps)
        tenter = torch.where(hit, tenter, torch.full_like(tenter, math.inf))
        tb, mb = tenter.min(dim=1)                                                       # nearest box per ray
        ax = axis.gather(1, mb[:, None])[:, 0]
        P = origin[None, :] + tb.clamp(max=1e300)[:, None] * dirs
        su = torch.where(ax == 0, P[:, 2], P[:, 0])
        sv = torch.where(ax == 1, P[:, 2], P[:, 1])
        face = ax * 2 + (dirs.gather(1, ax[:, None])[:, 0] > 0).to(torch.int64)
        take(tb, torch.isfinite(tb), tid[mb] * 8 + face, su, sv, texel[mb])
    return best, val


class Renderer:
    """Caches per-camera subpixel rays and renders views of a scene."""

    def __init__(self, cam: Camera, ss: int = 2, device: str = "cpu", chunk: int = 1 << 18):
        self.cam = cam
        self.ss = ss
        self.device = device
        self.chunk = chunk
        H, W = cam.height, cam.width
        vv, uu = torch.meshgrid(torch.arange(H, dtype=torch.float64, device=device),
                                torch.arange(W, dtype=torch.float64, device=device), indexing="ij")
        offs = (torch.arange(ss, dtype=torch.float64, device=device) + 0.5) / ss - 0.5
        oy, ox = torch.meshgrid(offs, offs, indexing="ij")
        u = uu[:, :, None] + ox.reshape(-1)[None, None, :]
        v = vv[:, :, None] + oy.reshape(-1)[None, None, :]
        self.rays, self.valid = pixel_rays(cam, u.reshape(-1), v.reshape(-1))
        self.center_rays, self.center_valid = pixel_rays(cam, uu.reshape(-1), vv.reshape(-1))

    def render(self, scene: Scene, world_to_cam: Pose, with_range: bool = False):
        """uint8 image (H, W) on the CPU; with_range adds the true range map
        (float64, 0 where the centre ray hits nothing or is not a viewing ray)."""
        cam = self.cam
        dev = self.device
        Rt = torch.tensor(world_to_cam.R.T, dtype=torch.float64, device=dev)
        C = -(Rt @ torch.tensor(world_to_cam.t, dtype=torch.float64, device=dev))
        vals = torch.empty(self.rays.shape[0], dtype=torch.float64, device=dev)
        for s0 in range(0, self.rays.shape[0], self.chunk):
            d = self.rays[s0:s0 + self.chunk] @ Rt.T
            _, v = cast(scene, C, d)
            vals[s0:s0 + self.chunk] = v
        vals = torch.where(self.valid, vals, torch.full_like(vals, OUTSIDE / 255.0))
        img = vals.reshape(cam.height, cam.width, self.ss * self.ss).mean(dim=2)
        img = torch.clamp(torch.round(img * 255.0), 0, 255).to(torch.uint8).cpu()
        if not with_range:
            return img
        rng = torch.empty(self.center_rays.shape[0], dtype=torch.float64, device=dev)
        for s0 in range(0, self.center_rays.shape[0], self.chunk):
            d = self.center_rays[s0:s0 + self.chunk] @ Rt.T
            s, _ = cast(scene, C, d)
            rng[s0:s0 + self.chunk] = s
        rng = torch.where(self.center_valid & torch.isfinite(rng), rng, torch.zeros_like(rng))
        return img, rng.reshape(cam.height, cam.width).cpu()


def random_boxes(rng: np.random.Generator, width: int, height: int, n: int,
                 min_frac: float = 0.05, max_frac: float = 0.2) -> np.ndarray:
    """n axis-aligned half-open pixel rectangles (x0, y0, x1, y1), int32:
    stand-ins for the detector's dynamic-object boxes."""
    out = np.zeros((n, 4), dtype=np.int32)
    for i in range(n):
        w = int(rng.uniform(min_frac, max_frac) * width)
        h = int(rng.uniform(min_frac, max_frac) * height)
        x0 = int(rng.integers(0, max(1, width - w)))
        y0 = int(rng.integers(0, max(1, height - h)))
        out[i] = (x0, y0, x0 + w, y0 + h)
    return out
