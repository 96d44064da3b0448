"""Pins of the oracle's plane-sweep stereo (Sec. III-A).

Checked against things outside the oracle: Pearson correlation from numpy,
the cost endpoints the paper fixes (cost 0 <-> ZNCC 1, cost 1 <-> ZNCC -1),
exact parabola samples, an independent warp chain built from the renderer's
camera code, zero-baseline identities, the analytic depth of rendered
planes, the multi-scale level geometry and the paper's stated sizes.
"""
import copy
import math
import os

import numpy as np
import pytest
import torch

import oracle
import scenes
from scenes.render import Camera, Plane, Pose, Rect, Scene, forward_project, pixel_rays
from scenes.configs import DOWNSAMPLE, CROP, FRONTO, GROUND, Level, PlaneSet, Rig

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ ZNCC

def test_zncc_identities():
    rng = np.random.default_rng(0)
    a = rng.uniform(size=81)
    assert abs(oracle.zncc(a, a) - 1.0) < 1e-14
    assert abs(oracle.zncc(a, 3.0 * a + 0.2) - 1.0) < 1e-14
    assert abs(oracle.zncc(a, -0.5 * a + 0.9) + 1.0) < 1e-14
    assert oracle.zncc(a, np.full(81, 0.3)) is None
    assert oracle.zncc(np.full(25, 0.7), a[:25]) is None


def test_zncc_is_pearson():
    rng = np.random.default_rng(1)
    for n in (9, 25, 49, 81):
        a, b = rng.uniform(size=n), rng.uniform(size=n)
        assert abs(oracle.zncc(a, b) - np.corrcoef(a, b)[0, 1]) < 1e-13


def test_zncc_hand_example():
    # a = 1..9, b = a with the last entry raised from 9 to 12:
    # mean_a = 5, mean_b = 16/3; cov = sum (a-5)(b-16/3) = 60 + 4*(12-9) - 0 = 72... computed below
    # by the textbook sums S_ab - S_a S_b / n over S_aa - S_a^2/n etc.
    a = np.arange(1, 10, dtype=float)
    b = a.copy()
    b[-1] = 12.0
    n = 9
    Sa, Sb = 45.0, 48.0
    Saa = 285.0
    Sbb = 285.0 - 81.0 + 144.0
    Sab = 285.0 - 81.0 + 108.0
    ref = (Sab - Sa * Sb / n) / math.sqrt((Saa - Sa * Sa / n) * (Sbb - Sb * Sb / n))
    assert abs(oracle.zncc(a, b) - ref) < 1e-14


# ------------------------------------------------------------------ planes

def test_plane_families():
    lv = Level(kind=DOWNSAMPLE, window=5, factor=1,
               sets=[PlaneSet(FRONTO, 9, 0.5, 20.0), PlaneSet(GROUND, 5, 1.0, 2.0, n=(0.0, 2.0, 0.0))])
    n, d, s, loc = oracle.level_planes(lv)
    assert list(s) == [0] * 9 + [1] * 5
    assert list(loc) == list(range(9)) + list(range(5))
    inv = 1.0 / d[:9]
    assert abs(d[0] - 20.0) < 1e-12 and abs(d[8] - 0.5) < 1e-12     # index 0 farthest
    assert np.allclose(np.diff(inv), (2.0 - 0.05) / 8, atol=1e-12)   # uniform in inverse depth
    assert np.allclose(n[:9], [0, 0, 1])
    assert np.allclose(d[9:], np.linspace(1.0, 2.0, 5), atol=1e-14)
    assert np.allclose(n[9:], [0, 1, 0])                             # normal normalised


# ------------------------------------------------------------------ WTA

def test_wta_parabola_exact():
    for k0, kexp, dexp in [(7.3, 7, 0.3), (6.8, 7, -0.2), (5.0, 5, 0.0), (12.49, 12, 0.49)]:
        C = 0.02 * (np.arange(20) - k0) ** 2 + 0.1
        ks, c1, c2, delta = oracle.wta(C, [20])
        assert ks == kexp
        assert abs(delta - dexp) < 1e-12
        assert c1 == C[kexp]
        assert c2 == np.sort(C)[1]


def test_wta_ties_ends_and_sets():
    C = np.array([0.5, 0.2, 0.2, 0.7])
    ks, c1, c2, delta = oracle.wta(C, [4])
    assert ks == 1 and c2 == 0.2            # ties go to the lowest index
    # minimum at the end of a set: no neighbour on one side, no fit
    C = np.array([0.9, 0.6, 0.3, 0.1, 0.2, 0.5, 0.8, 0.9])
    ks, c1, c2, delta = oracle.wta(C, [4, 4])
    assert ks == 3 and delta == 0.0         # index 4 belongs to the next set
    ks, c1, c2, delta = oracle.wta(C, [8])
    assert ks == 3 and delta != 0.0
    # invalid neighbour: no fit
    C = np.array([0.9, np.inf, 0.1, 0.3, 0.5])
    ks, c1, c2, delta = oracle.wta(C, [5])
    assert ks == 2 and delta == 0.0 and c2 == 0.3
    # nothing valid
    ks, c1, c2, delta = oracle.wta(np.full(5, np.inf), [5])
    assert ks == -1 and c1 == np.inf and c2 == np.inf
    # flat triple: no fit
    ks, c1, c2, delta = oracle.wta(np.array([0.3, 0.3, 0.3]), [3])
    assert ks == 0 and delta == 0.0


# ------------------------------------------------------------------ warp

def _img(rng, H, W):
    return rng.integers(0, 256, size=(H, W), dtype=np.uint8)


def test_zero_baseline_warp_is_identity():
    cam = Camera(xi=1.0, fx=40, fy=40, cx=31.5, cy=23.5, width=64, height=48)
    rig = Rig(ref=cam, cams=[cam], ref_to_cam=[Pose.identity()])
    lv = Level(kind=DOWNSAMPLE, window=5, factor=1, sets=[PlaneSet(FRONTO, 6, 0.5, 20.0)])
    rng = np.random.default_rng(2)
    ref = _img(rng, 48, 64)
    other = _img(rng, 48, 64)
    for k in (0, 3, 5):
        for (qx, qy) in [(10, 10), (31, 23), (50, 40), (5, 30)]:
            w = oracle.warped_sample(rig, lv, [ref, other], 0, k, qx, qy)
            assert w is not None and abs(w - other[qy, qx] / 255.0) < 1e-10


def test_cost_endpoints_from_sweep():
    # Identical views through a zero baseline: every plane gives ZNCC 1, cost
    # 0.  An inverted copy gives ZNCC -1, cost 1.  (Warped positions carry
    # ~1e-12 px of round-trip rounding, so equal costs are equal to 1e-12 and
    # the outermost samples may fall a hair outside the image.)
    cam = Camera(xi=1.0, fx=40, fy=40, cx=31.5, cy=23.5, width=64, height=48)
    rig = Rig(ref=cam, cams=[cam], ref_to_cam=[Pose.identity()])
    lv = Level(kind=DOWNSAMPLE, window=5, factor=1, sets=[PlaneSet(FRONTO, 6, 0.5, 20.0)])
    rng = np.random.default_rng(3)
    ref = _img(rng, 48, 64)
    res = oracle.sweep_level(rig, lv, [ref, ref], want_costs=True)
    inner = res["costs"][3:-3, 3:-3]
    assert np.isfinite(inner).all()
    assert np.abs(inner).max() < 1e-12
    assert (res["c1"][3:-3, 3:-3] < 1e-12).all()
    inv = (255 - ref).astype(np.uint8)
    res = oracle.sweep_level(rig, lv, [ref, inv], want_costs=True)
    assert np.abs(res["costs"][3:-3, 3:-3] - 1.0).max() < 1e-12
    # pixels closer to the border than the window radius have no depth
    assert (res["kstar"][:2] == -1).all() and (res["kstar"][:, -2:] == -1).all()


def test_warp_matches_independent_chain():
    # Rebuild the warp from the renderer's ray (bisection) and forward
    # projection (textbook sphere model) plus numpy bilinear sampling.
    wl = scenes.street(1, n_frames=1, scale=0.25)
    rig = wl.rig
    lv = wl.levels[0]
    s = lv.factor
    rng = np.random.default_rng(4)
    H, W = rig.ref.height, rig.ref.width
    imgs = [_img(rng, H, W) for _ in range(3)]
    n, d, sets, loc = oracle.level_planes(lv)
    # level cameras: same model with scaled intrinsics (pinned separately below)
    def lvl(c):
        return Camera(xi=c.xi, fx=c.fx / s, fy=c.fy / s, cx=(c.cx - (s - 1) / 2) / s, cy=(c.cy - (s - 1) / 2) / s,
                      width=c.width // s, height=c.height // s, k1=c.k1, k2=c.k2, p1=c.p1, p2=c.p2,
                      r2_max=c.r2_max)
    refl = lvl(rig.ref)
    low = [im.reshape(H // s, s, W // s, s).astype(np.float64).mean(axis=(1, 3)) / 255.0 for im in imgs]
    checked = 0
    for trial in range(300):
        qx, qy = int(rng.integers(0, W // s)), int(rng.integers(0, H // s))
        k = int(rng.integers(0, len(d)))
        j = int(rng.integers(0, 2))
        got = oracle.warped_sample(rig, lv, imgs, j, k, qx, qy)
        r, ok = pixel_rays(refl, torch.tensor([float(qx)]), torch.tensor([float(qy)]))
        r = r.numpy()[0]
        nr = float(n[k] @ r)
        if not ok[0] or nr <= 0:
            assert got is None
            continue
        X = d[k] / nr * r
        P = rig.ref_to_cam[j]
        Xj = P.R @ X + P.t
        cj = lvl(rig.cams[j])
        Xs = Xj / np.linalg.norm(Xj)
        if Xs[2] <= -min(cj.xi, 1 / cj.xi) + 1e-9:
            continue
        mx, my = Xs[0] / (Xs[2] + cj.xi), Xs[1] / (Xs[2] + cj.xi)
        if abs(mx * mx + my * my - cj.r2_max) < 1e-9:
            continue
        if mx * mx + my * my > cj.r2_max:
            assert got is None
            continue
        u, v = forward_project(cj, Xj)
        I = low[1 + j]
        if not (0 <= u <= I.shape[1] - 1 and 0 <= v <= I.shape[0] - 1):
            assert got is None
            continue
        x0, y0 = int(math.floor(u)), int(math.floor(v))
        x1, y1 = min(x0 + 1, I.shape[1] - 1), min(y0 + 1, I.shape[0] - 1)
        ax, ay = u - x0, v - y0
        ref = (1 - ay) * ((1 - ax) * I[y0, x0] + ax * I[y0, x1]) + ay * ((1 - ax) * I[y1, x0] + ax * I[y1, x1])
        assert got is not None and abs(got - ref) < 1e-9
        checked += 1
    assert checked > 100


# ------------------------------------------------------------------ multi-scale geometry

def test_level_geometry_closed_forms():
    cam = Camera(xi=0.9, fx=300, fy=310, cx=321.3, cy=255.2, width=640, height=512,
                 k1=0.01, k2=-0.002, p1=0.001, p2=0.0005, r2_max=2.5)
    rng = np.random.default_rng(5)
    img = _img(rng, 512, 640)
    for s in (2, 4):
        lc, limg = oracle.level_ref(cam, Level(kind=DOWNSAMPLE, window=7, factor=s, sets=[]), img)
        assert (lc.width, lc.height) == (640 // s, 512 // s)
        # block means (numpy reshape) of the uint8 image
        ref = img.reshape(512 // s, s, 640 // s, s).astype(np.float64).mean(axis=(1, 3)) / 255.0
        assert np.abs(limg - ref).max() < 1e-15
        # a level pixel centre sits at full-resolution coordinate s*u' + (s-1)/2
        lcam = Camera(xi=lc.xi, fx=lc.fx, fy=lc.fy, cx=lc.cx, cy=lc.cy, width=lc.width, height=lc.height,
                      k1=lc.k1, k2=lc.k2, p1=lc.p1, p2=lc.p2, r2_max=lc.r2_max)
        for _ in range(50):
            X = np.array([rng.uniform(-3, 3), rng.uniform(-2, 2), rng.uniform(1, 9)])
            uf, ul = oracle.project(cam, X), oracle.project(lcam, X)
            assert uf is not None and ul is not None
            assert np.allclose(s * ul + (s - 1) / 2.0, uf, atol=1e-9)
    lc, limg = oracle.level_ref(cam, Level(kind=CROP, window=9, crop_w=200, crop_h=100, sets=[]), img)
    x0, y0 = (640 - 200) // 2, (512 - 100) // 2
    assert np.array_equal(limg, img[y0:y0 + 100, x0:x0 + 200] / 255.0)
    assert (lc.cx, lc.cy, lc.width, lc.height) == (cam.cx - x0, cam.cy - y0, 200, 100)


def _golden_params():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_parameters.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = [float(x) for x in v.split(",")]
    return vals


def test_paper_sizes():
    # Sec. III-A: 1024x544 images, downsampled to 512x272, centre crop 572x332,
    # 64 fronto-parallel + 30 ground planes, 9x9 (full) and 7x7 (downsampled) windows.
    g = _golden_params()
    W, H = (int(v) for v in g["full_size"])
    cam = Camera(xi=1.0, fx=300, fy=300, cx=W / 2, cy=H / 2, width=W, height=H)
    img = np.zeros((H, W), dtype=np.uint8)
    s = int(round(W / g["low_size"][0]))
    low = Level(kind=DOWNSAMPLE, window=int(g["window_low"][0]), factor=s,
                sets=[PlaneSet(FRONTO, int(g["planes_fronto"][0]), 0.5, 30.0),
                      PlaneSet(GROUND, int(g["planes_ground"][0]), 1.1, 2.1, n=(0, 1, 0))])
    lc, _ = oracle.level_ref(cam, low, img)
    assert [lc.width, lc.height] == [int(v) for v in g["low_size"]]
    assert low.n_planes == 94
    cw, ch = (int(v) for v in g["crop_size"])
    lc, _ = oracle.level_ref(cam, Level(kind=CROP, window=int(g["window_full"][0]), crop_w=cw, crop_h=ch,
                                        sets=[]), img)
    assert (W - cw) // 2 == 226 and (H - ch) // 2 == 106
    assert (lc.cx, lc.cy) == (W / 2 - 226, H / 2 - 106)


def test_merge_toy():
    rng = np.random.default_rng(6)
    W, H, s = 16, 8, 2
    low = rng.uniform(1, 9, size=(H // s, W // s))
    low[1, 2] = 0.0
    crop = rng.uniform(1, 9, size=(4, 6))
    crop[0, 0] = 0.0
    boxes = np.array([[0, 0, 3, 2], [14, 6, 20, 9]], dtype=np.int32)
    out = oracle.merge(W, H, low, s, crop, 6, 4, boxes)
    exp = np.repeat(np.repeat(low, s, axis=0), s, axis=1)
    x0, y0 = (W - 6) // 2, (H - 4) // 2
    sub = exp[y0:y0 + 4, x0:x0 + 6]
    exp[y0:y0 + 4, x0:x0 + 6] = np.where(crop > 0, crop, sub)
    exp[0:2, 0:3] = 0
    exp[6:8, 14:16] = 0
    assert np.array_equal(out, exp)


# ------------------------------------------------------------------ rendered scenes

def _exact_plane_workload(k0):
    wl = scenes.tiny(0)
    n, d, s, loc = oracle.level_planes(wl.levels[0])
    z = d[k0]
    wl.scene = Scene(seed=3)
    wl.scene.rects.append(Rect(c=(0, 0, z), e1=(1, 0, 0), e2=(0, 1, 0), a=3 * z, b=3 * z,
                               texel=0.0375 * z, tex_id=5))
    return wl, d


@pytest.mark.parametrize("k0", [8, 20])
def test_analytic_plane_depth(k0):
    # A textured plane rendered exactly at sweep plane k0 is recovered as k0,
    # with range within half the plane spacing of the true range.
    wl, d = _exact_plane_workload(k0)
    imgs, rng = scenes.FrameSource(wl).frame(0, with_range=True)
    imgs = [i.numpy() for i in imgs]
    rng = rng.numpy()
    res = oracle.sweep_level(wl.rig, wl.levels[0], imgs)
    k = res["kstar"]
    v = k >= 0
    H, W = k.shape
    yy, xx = np.mgrid[0:H, 0:W]
    central = v & (np.abs(xx - 80) < 40) & (np.abs(yy - 64) < 32)
    assert v.mean() > 0.5
    assert (k[v] == k0).mean() > 0.85
    assert (k[central] == k0).mean() >= 0.99
    sel = central & (k == k0) & (rng > 0)
    assert sel.sum() > 4000
    # The true range of the plane z = d_k0 along the pixel's unit ray is
    # d_k0 / r_z (the renderer's ray-cast range), so r_z = d_k0 / range and
    # the recovered plane depth is r_z * range.  The planes are uniform in
    # inverse depth; on every pixel the recovered inverse depth lies within
    # half the plane spacing (the smaller of the two sides) of 1 / d_k0.
    rz = d[k0] / rng[sel]
    dinv = 0.5 * min(abs(1 / d[k0 + 1] - 1 / d[k0]), abs(1 / d[k0] - 1 / d[k0 - 1]))
    einv = np.abs(1 / (rz * res["depth"][sel]) - 1 / d[k0])
    assert (einv <= dinv).all(), (einv / dinv).max()
    # in range: within the far side's half spacing (the two sides' images of
    # half an inverse-depth step differ; the far one is the larger)
    err = np.abs(res["depth"][sel] - rng[sel])
    assert (err * rz <= 0.5 * abs(d[k0] - d[k0 - 1])).all()
    assert np.median(err / rng[sel]) < 0.01


def test_thread_count_does_not_change_results():
    # the OpenMP build shares pixels (and TSDF blocks) among threads; every
    # output must be the same bit for bit as on one thread
    wl = scenes.tiny(2, n_frames=1)
    imgs, _ = scenes.FrameSource(wl).frame(0)
    imgs = [i.numpy() for i in imgs]
    n0 = oracle.set_threads()
    try:
        outs = []
        for n in (1, max(4, n0)):
            oracle.set_threads(n)
            r = oracle.sweep_level(wl.rig, wl.levels[0], imgs)
            T = oracle.Tsdf(wl.tsdf)
            T.integrate(r["depth"].astype(np.float32), wl.rig.ref, wl.world_to_ref[0])
            outs.append((r, T.dump()))
    finally:
        oracle.set_threads(n0)
    (a, ta), (b, tb) = outs
    for key in ("depth", "c1", "c2", "kstar"):
        assert np.array_equal(a[key], b[key]), key
    for x, y in zip(ta, tb):
        assert np.array_equal(x, y)
    assert (a["kstar"] >= 0).mean() > 0.2 and (ta[2] > 0).any()


def test_full_level_invariants():
    wl = scenes.tiny(1)
    imgs, _ = scenes.FrameSource(wl).frame(0)
    imgs = [i.numpy() for i in imgs]
    res = oracle.sweep_level(wl.rig, wl.levels[0], imgs, want_costs=True)
    k, c1, c2, dep, C = res["kstar"], res["c1"], res["c2"], res["depth"], res["costs"]
    v = k >= 0
    assert v.mean() > 0.2
    assert ((dep > 0) == v).all()
    assert (c1[v] >= -1e-15).all() and (c1[v] <= 1 + 1e-15).all() and (c1[v] <= c2[v]).all()
    fin = np.isfinite(C)
    assert (C[fin] >= -1e-15).all() and (C[fin] <= 1 + 1e-15).all()
    assert np.allclose(np.where(np.isfinite(C), C, np.inf).min(axis=2)[v], c1[v])
    rho = wl.levels[0].window // 2
    assert (k[:rho] == -1).all() and (k[-rho:] == -1).all()
    assert (k[:, :rho] == -1).all() and (k[:, -rho:] == -1).all()


def test_ground_family_recovers_ground():
    # A bare ground plane 1.6 m below the cameras: the ground-parallel family
    # (offsets 1.1 .. 2.1 m) should explain most ground pixels.
    wl = scenes.street(2, n_frames=1, scale=0.25)
    wl.scene.boxes = []
    imgs, rng = scenes.FrameSource(wl).frame(0, with_range=True)
    imgs = [i.numpy() for i in imgs]
    rng = rng.numpy()
    lv = wl.levels[0]
    res = oracle.sweep_level(wl.rig, lv, imgs)
    k = res["kstar"]
    s = lv.factor
    truth = rng[::s, ::s][: k.shape[0], : k.shape[1]]
    ground_rows = np.zeros_like(k, dtype=bool)
    ground_rows[int(0.7 * k.shape[0]):] = True
    sel = ground_rows & (k >= 0) & (truth > 0)
    n_fronto = lv.sets[0].count
    assert sel.sum() > 200
    assert (k[sel] >= n_fronto).mean() > 0.8
    rel = np.abs(res["depth"][sel] - truth[sel]) / truth[sel]
    assert np.median(rel) < 0.05
