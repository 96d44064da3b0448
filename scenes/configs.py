"""Workload descriptions: rigs, sweep levels, plane sets, TSDF settings and
seeded scenes for the two single-GPU workloads.

* ``tiny(seed)`` — 1 reference + 1 matching fisheye camera (xi = 1, fx = fy =
  80, 160x128), textured fronto-parallel planes at 1-15 m, 0.5 m baseline,
  32 fronto-parallel sweep planes uniform in inverse depth over 0.5-20 m,
  5x5 ZNCC window, one dense 64^3 TSDF of 5 cm voxels with 0.2 m truncation.
* ``street(seed)`` — reference + 2 matching cameras (xi ~ U[0.8, 1.2],
  radial-tangential coefficients ~ N(0, 0.02)) at 1280x1024 looking down a
  seeded street (ground plane and boxes); two sweep levels: the whole view
  downsampled 4x to 320x256 with 64 fronto-parallel + 32 ground-parallel
  planes and a 7x7 window, and the central 640x512 crop at full resolution
  with 128 fronto-parallel planes and a 9x9 window; 1-3 dynamic-object boxes
  per frame; voxel-block TSDF (8^3 blocks, 10 cm voxels, 0.5 m truncation,
  60 x 3 x 60 m local map) along a 100-frame straight trajectory at 1 m/frame.

``scale`` shrinks the street rig (image size, focal lengths, crop) for CPU
tests while keeping its structure.

These are plain data: each side (oracle, CUDA library) converts them into its
own structures and derives every quantity of the method (plane depths, level
intrinsics, rays) by itself.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

from .render import Box, Camera, Plane, Pose, Rect, Renderer, Scene, random_boxes, rot_xyz

FRONTO = 0
GROUND = 1
DOWNSAMPLE = 0
CROP = 1


@dataclass
class PlaneSet:
    """family FRONTO: `count` planes n = (0,0,1), inverse depth uniform on
    [1/b, 1/a] with index 0 farthest (a = near, b = far).
    family GROUND: `count` planes n . X = h with h uniform on [a, b],
    index 0 at h = a; n is the ground normal in the reference frame."""
    family: int
    count: int
    a: float
    b: float
    n: Tuple[float, float, float] = (0.0, 0.0, 1.0)


@dataclass
class Level:
    """kind DOWNSAMPLE: all images box-averaged by `factor`; kind CROP: the
    reference image's centred crop_w x crop_h window at full resolution,
    matched against the full-resolution matching images."""
    kind: int
    window: int
    sets: List[PlaneSet]
    factor: int = 1
    crop_w: int = 0
    crop_h: int = 0

    @property
    def n_planes(self) -> int:
        return sum(s.count for s in self.sets)


@dataclass
class Filters:
    """Depth map filtering (best cost, uniqueness, local continuity).  The
    paper gives alpha 0.05 / 0.3 for the upper / lower image part, gamma
    0.5 m and delta 0.3; the ratio threshold and the window are not given."""
    enable: bool = True
    alpha_upper: float = 0.05
    alpha_lower: float = 0.3
    split_row: float = -1.0      # < 0: half the image height
    ratio_min: float = 1.1
    gamma: float = 0.5
    delta: float = 0.3
    window: int = 5


@dataclass
class Rig:
    ref: Camera
    cams: List[Camera]
    ref_to_cam: List[Pose]


@dataclass
class TsdfParams:
    voxel_size: float
    mu: float
    w_max: float = 100.0
    block_dim: int = 8
    dense_dim: Optional[Tuple[int, int, int]] = None   # voxels per axis; None = hashed blocks
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    local_half: Optional[Tuple[float, float, float]] = None  # None = no local-map gate
    local_offset: Tuple[float, float, float] = (0.0, 0.0, 0.0)  # local-map centre - camera centre
    hash_slots: int = 1 << 20
    pool_blocks: int = 1 << 16


@dataclass
class Workload:
    name: str
    rig: Rig
    levels: List[Level]
    tsdf: TsdfParams
    scene: Scene
    world_to_ref: List[Pose]          # trajectory, one pose per frame
    boxes: List[np.ndarray]           # per frame (n, 4) int32 half-open pixel rects
    ss: int = 2                       # supersampling used when rendering
    filters: Optional[Filters] = None  # depth map filtering (None = off)

    @property
    def n_frames(self) -> int:
        return len(self.world_to_ref)

    def local_center(self, frame: int) -> Optional[Tuple[float, float, float]]:
        if self.tsdf.local_half is None:
            return None
        c = self.world_to_ref[frame].inverse().t
        o = self.tsdf.local_offset
        return (c[0] + o[0], c[1] + o[1], c[2] + o[2])

    def pix_planes(self) -> int:
        """Sum over levels of reference pixels x planes."""
        tot = 0
        for lv in self.levels:
            if lv.kind == DOWNSAMPLE:
                w, h = self.rig.ref.width // lv.factor, self.rig.ref.height // lv.factor
            else:
                w, h = lv.crop_w, lv.crop_h
            tot += w * h * lv.n_planes
        return tot


# --------------------------------------------------------------------------
# tiny: 1 + 1 cameras, 160x128, fronto planes, dense TSDF
# --------------------------------------------------------------------------

def tiny(seed: int = 0, n_frames: int = 1) -> Workload:
    rng = np.random.default_rng(1000 + seed)
    cam = Camera(xi=1.0, fx=80.0, fy=80.0, cx=80.0, cy=64.0, width=160, height=128)
    # matching camera 0.5 m to the right of the reference camera
    rig = Rig(ref=cam, cams=[cam], ref_to_cam=[Pose(np.eye(3), np.array([-0.5, 0.0, 0.0]))])
    scene = Scene(seed=seed)
    zb = float(rng.uniform(12.0, 15.0))
    # background: a large fronto-parallel rectangle (about +-63 degrees wide)
    scene.rects.append(Rect(c=(0.0, 0.0, zb), e1=(1, 0, 0), e2=(0, 1, 0), a=2.0 * zb, b=1.6 * zb,
                            texel=0.0375 * zb, tex_id=1))
    n_rect = int(rng.integers(3, 6))
    nearest = None
    for i in range(n_rect):
        z = float(rng.uniform(1.0, 10.0))
        ax = math.radians(rng.uniform(-40, 40))
        ay = math.radians(rng.uniform(-30, 30))
        c = (z * math.tan(ax), z * math.tan(ay), z)
        half = float(rng.uniform(0.15, 0.35)) * z
        scene.rects.append(Rect(c=c, e1=(1, 0, 0), e2=(0, 1, 0), a=half, b=half * 0.8,
                                texel=0.0375 * z, tex_id=10 + i))
        if nearest is None or z < nearest[2]:
            nearest = c
    # dense 64^3 grid of 5 cm voxels (3.2 m cube) centred on the nearest plane's centre
    origin = (nearest[0] - 1.6, nearest[1] - 1.6, nearest[2] - 1.6)
    tsdf = TsdfParams(voxel_size=0.05, mu=0.2, dense_dim=(64, 64, 64), origin=origin)
    levels = [Level(kind=DOWNSAMPLE, factor=1, window=5, sets=[PlaneSet(FRONTO, 32, 0.5, 20.0)])]
    traj = []
    for f in range(n_frames):
        # small sideways drift so that repeated frames see the cube from new poses
        traj.append(Pose(np.eye(3), np.array([-0.05 * f, 0.0, 0.0])))
    boxes = [np.zeros((0, 4), dtype=np.int32) for _ in range(n_frames)]
    return Workload("tiny-160x128-1cam-32planes", rig, levels, tsdf, scene, traj, boxes, ss=4)


# --------------------------------------------------------------------------
# street: 1 + 2 cameras, 1280x1024, multi-resolution, hashed TSDF
# --------------------------------------------------------------------------

def _monotone(k1, k2, p1, p2, r2_max) -> bool:
    """Radial-tangential map one-to-one (Jacobian > 0.2) on the disk r^2 <= r2_max."""
    for s in np.linspace(0, r2_max, 41):
        if 1 + 3 * k1 * s + 5 * k2 * s * s < 0.3:
            return False
    rr = np.sqrt(np.linspace(0, r2_max, 21))
    th = np.linspace(0, 2 * np.pi, 37)
    R, T = np.meshgrid(rr, th)
    x, y = R * np.cos(T), R * np.sin(T)
    r2 = x * x + y * y
    rad = 1 + k1 * r2 + k2 * r2 * r2
    drad = k1 + 2 * k2 * r2           # d rad / d r2
    dxdx = rad + 2 * x * x * drad + 2 * p1 * y + 6 * p2 * x
    dxdy = 2 * x * y * drad + 2 * p1 * x + 2 * p2 * y
    dydx = 2 * x * y * drad + 2 * p1 * x + 2 * p2 * y
    dydy = rad + 2 * y * y * drad + 6 * p1 * y + 2 * p2 * x
    return bool(np.all(dxdx * dydy - dxdy * dydx > 0.2))


def _street_camera(rng, scale: float, r2_max: float = 2.5) -> Camera:
    xi = float(rng.uniform(0.8, 1.2))
    while True:
        k1, k2, p1, p2 = (float(v) for v in rng.normal(0.0, 0.02, size=4))
        if _monotone(k1, k2, p1, p2, r2_max):
            break
    W, H = int(round(1280 * scale)), int(round(1024 * scale))
    f = 640.0 * scale
    return Camera(xi=xi, fx=f, fy=f, cx=W / 2.0, cy=H / 2.0, width=W, height=H,
                  k1=k1, k2=k2, p1=p1, p2=p2, r2_max=r2_max)


def _street_scene(rng, seed: int, height: float) -> Scene:
    """Ground plane, building fronts along both sides of a straight street and
    parked cars by the kerbs (axis-aligned textured boxes)."""
    scene = Scene(seed=seed)
    scene.planes.append(Plane(n=(0, 1, 0), h=height, e1=(1, 0, 0), e2=(0, 0, 1),
                              texel=0.05, tex_id=1))
    tex = 10
    for side in (-1.0, 1.0):
        # building fronts: a run of boxes along the street with small gaps
        z = -40.0
        while z < 240.0:
            zl = float(rng.uniform(4.0, 15.0))
            inner = float(rng.uniform(4.5, 7.0))
            depth = float(rng.uniform(3.0, 8.0))
            h = float(rng.uniform(2.0, 9.0))
            x0, x1 = (inner, inner + depth) if side > 0 else (-inner - depth, -inner)
            scene.boxes.append(Box(lo=(x0, height - h, z), hi=(x1, height, z + zl),
                                   texel=0.05, tex_id=tex))
            tex += 1
            z += zl + float(rng.uniform(0.0, 5.0))
        # parked cars next to the kerb
        z = float(rng.uniform(0.0, 20.0))
        while z < 240.0:
            inner = float(rng.uniform(2.4, 3.0))
            x0, x1 = (inner, inner + 1.8) if side > 0 else (-inner - 1.8, -inner)
            zl = float(rng.uniform(3.8, 4.8))
            scene.boxes.append(Box(lo=(x0, height - 1.5, z), hi=(x1, height, z + zl),
                                   texel=0.04, tex_id=tex))
            tex += 1
            z += zl + float(rng.uniform(6.0, 30.0))
    return scene


def street(seed: int = 0, n_frames: int = 100, scale: float = 1.0) -> Workload:
    rng = np.random.default_rng(2000 + seed)
    ref = _street_camera(rng, scale)
    cams, poses = [], []
    for side in (-1.0, 1.0):
        cams.append(_street_camera(rng, scale))
        yaw, pitch = (math.radians(float(v)) for v in rng.uniform(-1.0, 1.0, size=2))
        R_cr = rot_xyz(pitch, yaw, 0.0)                 # camera axes in the reference frame
        c = np.array([0.5 * side, 0.0, 0.0])            # camera centre in the reference frame
        poses.append(Pose(R_cr.T, -R_cr.T @ c))
    rig = Rig(ref=ref, cams=cams, ref_to_cam=poses)

    height = 1.6
    scene = _street_scene(rng, seed, height)
    W, H = ref.width, ref.height
    s = 4 if scale >= 1.0 else 2
    crop_w, crop_h = int(round(640 * scale)), int(round(512 * scale))
    n_scale = 1.0 if scale >= 1.0 else 0.25
    levels = [
        Level(kind=DOWNSAMPLE, factor=s, window=7,
              sets=[PlaneSet(FRONTO, max(4, int(64 * n_scale)), 0.5, 30.0),
                    PlaneSet(GROUND, max(4, int(32 * n_scale)), height - 0.5, height + 0.5,
                             n=(0.0, 1.0, 0.0))]),
        Level(kind=CROP, window=9, crop_w=crop_w, crop_h=crop_h,
              sets=[PlaneSet(FRONTO, max(4, int(128 * n_scale)), 1.0, 80.0)]),
    ]
    tsdf = TsdfParams(voxel_size=0.1, mu=0.5, local_half=(30.0, 1.5, 30.0),
                      local_offset=(0.0, 0.6, 0.0))
    traj = [Pose(np.eye(3), np.array([0.0, 0.0, -1.0 * f])) for f in range(n_frames)]
    brng = np.random.default_rng(3000 + seed)
    boxes = [random_boxes(brng, W, H, int(brng.integers(1, 4))) for _ in range(n_frames)]
    name = f"street-{W}x{H}-3cam-multires"
    return Workload(name, rig, levels, tsdf, scene, traj, boxes, ss=2)


# --------------------------------------------------------------------------
# rendering helpers
# --------------------------------------------------------------------------

class FrameSource:
    """Renders the frames of a workload: reference + matching images, the
    reference's true range map (for fusion tests) and the boxes."""

    def __init__(self, wl: Workload, device: str = "cpu"):
        self.wl = wl
        self.ref_r = Renderer(wl.rig.ref, ss=wl.ss, device=device)
        self.cam_r = [Renderer(c, ss=wl.ss, device=device) for c in wl.rig.cams]

    def frame(self, f: int, with_range: bool = False):
        wl = self.wl
        w2r = wl.world_to_ref[f]
        out = self.ref_r.render(wl.scene, w2r, with_range=with_range)
        if with_range:
            ref_img, rng = out
        else:
            ref_img, rng = out, None
        imgs = [ref_img]
        for r, p in zip(self.cam_r, wl.rig.ref_to_cam):
            imgs.append(r.render(wl.scene, p.compose(w2r)))
        return imgs, rng


# --------------------------------------------------------------------------
# ring: reference + 3 matching cameras, 1280x1024, 256 full-resolution planes,
# 2 cm voxels along a closed 500 m loop
# --------------------------------------------------------------------------

def ring(seed: int = 0, n_frames: int = 1000, scale: float = 1.0, circumference: float = 500.0) -> Workload:
    """Precision-at-scale workload: a linear rig (matching cameras 0.5 m left,
    0.5 m and 1.0 m right of the reference), one full-resolution sweep level
    of 256 fronto-parallel planes with a 9x9 window, and a TSDF of 2 cm voxels
    (0.1 m truncation, 60 x 3 x 60 m local map, a 32 GB block pool for the
    whole loop) along a closed circular road driven in n_frames steps."""
    rng = np.random.default_rng(4000 + seed)
    ref = _street_camera(rng, scale)
    cams, poses = [], []
    for off in (-0.5, 0.5, 1.0):
        cams.append(_street_camera(rng, scale))
        yaw, pitch = (math.radians(float(v)) for v in rng.uniform(-1.0, 1.0, size=2))
        R_cr = rot_xyz(pitch, yaw, 0.0)
        c = np.array([off, 0.0, 0.0])
        poses.append(Pose(R_cr.T, -R_cr.T @ c))
    rig = Rig(ref=ref, cams=cams, ref_to_cam=poses)
    height = 1.6
    R = circumference / (2 * math.pi)
    scene = Scene(seed=seed)
    scene.planes.append(Plane(n=(0, 1, 0), h=height, e1=(1, 0, 0), e2=(0, 0, 1), texel=0.05, tex_id=1))
    # buildings on both sides of the road, axis-aligned boxes around the ring centre (R, 0, 0)
    tex = 10
    for side, (r0, r1) in ((1, (R + 5.0, R + 12.0)), (-1, (R - 12.0, R - 5.0))):
        ang = 0.0
        while ang < 2 * math.pi:
            rad = float(rng.uniform(r0, r1))
            size = float(rng.uniform(3.0, 8.0))
            h = float(rng.uniform(2.0, 9.0))
            cxw = R - rad * math.cos(ang)
            czw = rad * math.sin(ang)
            scene.boxes.append(Box(lo=(cxw - size / 2, height - h, czw - size / 2),
                                   hi=(cxw + size / 2, height, czw + size / 2), texel=0.05, tex_id=tex))
            tex += 1
            ang += (size + float(rng.uniform(1.0, 5.0))) / rad
    traj = []
    for f in range(n_frames):
        th = 2 * math.pi * f / n_frames
        p = np.array([R - R * math.cos(th), 0.0, R * math.sin(th)])
        R_cw = np.stack([np.array([math.cos(th), 0.0, -math.sin(th)]), np.array([0.0, 1.0, 0.0]),
                         np.array([math.sin(th), 0.0, math.cos(th)])], axis=1)   # camera axes in the world
        traj.append(Pose(R_cw.T, -R_cw.T @ p))
    levels = [Level(kind=DOWNSAMPLE, factor=1, window=9, sets=[PlaneSet(FRONTO, 256, 1.0, 80.0)])]
    # the paper's 60 x 3 x 60 m local map bounds what one frame allocates; the
    # block pool (2^23 blocks of 4 KB, 32 GB) holds the whole loop's map
    tsdf = TsdfParams(voxel_size=0.02, mu=0.1, hash_slots=1 << 25, pool_blocks=1 << 23,
                      local_half=(30.0, 1.5, 30.0), local_offset=(0.0, 0.6, 0.0))
    W, H = ref.width, ref.height
    brng = np.random.default_rng(5000 + seed)
    boxes = [random_boxes(brng, W, H, int(brng.integers(1, 4))) for _ in range(n_frames)]
    name = f"ring-{W}x{H}-4cam-256planes-2cm"
    return Workload(name, rig, levels, tsdf, scene, traj, boxes, ss=2)


# --------------------------------------------------------------------------
# batch mix: many independent single-frame sweeps of uneven size
# --------------------------------------------------------------------------

BATCH_SIZES = ((256, 200), (320, 256), (640, 512), (1024, 768))
BATCH_PLANES = (32, 64, 128, 256)


def batch_mix(seed: int = 0, n: int = 64, sizes=BATCH_SIZES, planes=BATCH_PLANES, max_cams: int = 4,
              ss: int = 1) -> List[Workload]:
    """n one-frame street workloads whose image size, plane count and number
    of matching cameras (1 .. max_cams) are drawn per sweep: each has one
    full-resolution level of fronto-parallel planes on [0.5, 30] m with a 7x7
    window and 0-3 boxes.  Matching cameras sit 0.3-1.0 m left or right of
    the reference with small yaw and pitch."""
    rng = np.random.default_rng(6000 + seed)
    out = []
    for i in range(n):
        W, H = sizes[int(rng.integers(len(sizes)))]
        n_planes = int(planes[int(rng.integers(len(planes)))])
        n_cams = int(rng.integers(1, max_cams + 1))
        scale = W / 1280.0

        def cam():
            c = _street_camera(rng, scale)
            return dataclasses.replace(c, width=W, height=H, cx=W / 2.0, cy=H / 2.0)

        ref = cam()
        cams, poses = [], []
        for j in range(n_cams):
            cams.append(cam())
            side = -1.0 if j % 2 == 0 else 1.0
            off = side * float(rng.uniform(0.3, 1.0))
            yaw, pitch = (math.radians(float(v)) for v in rng.uniform(-1.0, 1.0, size=2))
            R_cr = rot_xyz(pitch, yaw, 0.0)
            c = np.array([off, 0.0, 0.0])
            poses.append(Pose(R_cr.T, -R_cr.T @ c))
        rig = Rig(ref=ref, cams=cams, ref_to_cam=poses)
        height = 1.6
        scene = _street_scene(rng, seed * 1000 + i, height)
        levels = [Level(kind=DOWNSAMPLE, factor=1, window=7, sets=[PlaneSet(FRONTO, n_planes, 0.5, 30.0)])]
        tsdf = TsdfParams(voxel_size=0.1, mu=0.5, local_half=(30.0, 1.5, 30.0), local_offset=(0.0, 0.6, 0.0))
        traj = [Pose(np.eye(3), np.array([0.0, 0.0, -float(rng.uniform(0.0, 100.0))]))]
        boxes = [random_boxes(rng, W, H, int(rng.integers(0, 4)))]
        name = f"mix{i}-{W}x{H}-{1 + n_cams}cam-{n_planes}planes"
        out.append(Workload(name, rig, levels, tsdf, scene, traj, boxes, ss=ss))
    return out


# --------------------------------------------------------------------------
# diff: the small rig of the differentiable forms
# --------------------------------------------------------------------------

def diff(seed: int = 0, width: int = 96, height: int = 80, n_planes: int = 32) -> Workload:
    """Reference + 2 matching cameras (0.4 m left and right, distortion drawn
    as for the street rig) at 96 x 80, f = 0.8 W, looking at 3-5 textured
    fronto-parallel rectangles at 2-7 m in front of a textured background
    at 8-10 m; one full-resolution level of n_planes fronto planes on
    2-12 m with a 5x5 window; a dense 32^3 grid of 10 cm voxels around the
    nearest rectangle."""
    rng = np.random.default_rng(7000 + seed)
    scale = width / 1280.0

    def cam():
        c = _street_camera(rng, scale)
        return dataclasses.replace(c, width=width, height=height, cx=width / 2.0, cy=height / 2.0,
                                   fx=0.8 * width, fy=0.8 * width)

    ref = cam()
    cams, poses = [], []
    for side in (-1.0, 1.0):
        cams.append(cam())
        yaw, pitch = (math.radians(float(v)) for v in rng.uniform(-1.0, 1.0, size=2))
        R_cr = rot_xyz(pitch, yaw, 0.0)
        c = np.array([0.4 * side, 0.0, 0.0])
        poses.append(Pose(R_cr.T, -R_cr.T @ c))
    rig = Rig(ref=ref, cams=cams, ref_to_cam=poses)
    scene = Scene(seed=seed)
    zb = float(rng.uniform(8.0, 10.0))
    scene.rects.append(Rect(c=(0.0, 0.0, zb), e1=(1, 0, 0), e2=(0, 1, 0), a=3.0 * zb, b=2.4 * zb,
                            texel=0.04 * zb, tex_id=1))
    nearest = None
    for i in range(int(rng.integers(3, 6))):
        z = float(rng.uniform(2.0, 7.0))
        ax = math.radians(rng.uniform(-35, 35))
        ay = math.radians(rng.uniform(-25, 25))
        c = (z * math.tan(ax), z * math.tan(ay), z)
        half = float(rng.uniform(0.2, 0.4)) * z
        scene.rects.append(Rect(c=c, e1=(1, 0, 0), e2=(0, 1, 0), a=half, b=half * 0.8, texel=0.04 * z,
                                tex_id=10 + i))
        if nearest is None or z < nearest[2]:
            nearest = c
    origin = (nearest[0] - 1.6, nearest[1] - 1.6, nearest[2] - 1.6)
    tsdf = TsdfParams(voxel_size=0.1, mu=0.3, dense_dim=(32, 32, 32), origin=origin)
    levels = [Level(kind=DOWNSAMPLE, factor=1, window=5, sets=[PlaneSet(FRONTO, n_planes, 2.0, 12.0)])]
    traj = [Pose(np.eye(3), np.zeros(3))]
    boxes = [np.zeros((0, 4), dtype=np.int32)]
    return Workload(f"diff-{width}x{height}-3cam-{n_planes}planes", rig, levels, tsdf, scene, traj, boxes, ss=4)
