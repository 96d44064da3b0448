"""Pins of the oracle's TSDF fusion (Sec. III-C, Eq. 2).

Checked against closed forms that need no projection arithmetic (a depth map
of constant range R observes a sphere of radius R around the camera centre,
so eta = R - |X - C| for every voxel in view), repeated and alternating
observations, the weight cap, a hand-computed allocation along an axis ray,
dense point sampling of random ray segments, and the local-map gate.
"""
import math

import numpy as np
import pytest

import oracle
from scenes.configs import TsdfParams
from scenes.render import Camera, Pose, forward_project, rot_xyz

CAM = Camera(xi=1.0, fx=20.0, fy=20.0, cx=20.0, cy=20.0, width=41, height=41)


def _dense(voxel=0.05, mu=0.2, dim=16, origin=(-0.4, -0.4, 0.6), w_max=100.0):
    return TsdfParams(voxel_size=voxel, mu=mu, dense_dim=(dim, dim, dim), origin=origin, w_max=w_max)


def _voxel_centres(p):
    B = p.block_dim
    keys, D, W, amb = oracle.Tsdf(p).dump()
    out = np.zeros((len(keys), B ** 3, 3))
    z, y, x = np.meshgrid(np.arange(B), np.arange(B), np.arange(B), indexing="ij")
    loc = np.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], axis=1)
    for i, k in enumerate(keys):
        out[i] = np.array(p.origin) + (k[None, :] * B + loc + 0.5) * p.voxel_size
    return keys, out


def _expected_sphere(p, centres, R, w2c):
    C = w2c.inverse().t
    dist = np.linalg.norm(centres - C[None, None, :], axis=2)
    eta = R - dist
    inview = np.zeros(dist.shape, dtype=bool)
    for i in range(centres.shape[0]):
        for v in range(centres.shape[1]):
            Xc = w2c.R @ centres[i, v] + w2c.t
            if Xc[2] <= -1.0 + 1e-9:
                continue
            u, vv = forward_project(CAM, Xc)
            pu, pv = math.floor(u + 0.5), math.floor(vv + 0.5)
            inview[i, v] = 0 <= pu < CAM.width and 0 <= pv < CAM.height
    upd = inview & (eta >= -p.mu)
    return np.where(upd, np.minimum(1.0, eta / p.mu), 0.0), upd


@pytest.mark.parametrize("R", [1.0, 0.93])
def test_one_frame_constant_range(R):
    p = _dense()
    keys, centres = _voxel_centres(p)
    w2c = Pose.identity()
    T = oracle.Tsdf(p)
    T.integrate(np.full((41, 41), R, dtype=np.float32), CAM, w2c)
    k2, D, W, amb = T.dump()
    expD, upd = _expected_sphere(p, centres, np.float32(R), w2c)
    assert np.array_equal(k2, keys)
    assert upd.sum() > 1000 and (~upd).sum() > 100            # both outcomes present
    assert np.array_equal(W > 0, upd)
    assert np.abs(D - expD).max() < 1e-12
    # sign convention: positive in front of the surface, negative behind it
    C = np.zeros(3)
    dist = np.linalg.norm(centres - C, axis=2)
    assert (D[upd & (dist < R - 1e-6)] > 0).all()
    assert (D[upd & (dist > R + 1e-6)] < 0).all()
    assert D.max() == 1.0 and D.min() >= -1.0


def test_rotated_camera_constant_range():
    p = _dense(origin=(0.3, -0.4, 0.3))
    keys, centres = _voxel_centres(p)
    R_cw = rot_xyz(0.1, 0.5, -0.05)           # camera axes in world
    C = np.array([0.2, 0.1, -0.3])
    w2c = Pose(R_cw.T, -R_cw.T @ C)
    T = oracle.Tsdf(p)
    T.integrate(np.full((41, 41), 1.2, dtype=np.float32), CAM, w2c)
    _, D, W, _ = T.dump()
    expD, upd = _expected_sphere(p, centres, np.float32(1.2), w2c)
    assert upd.sum() > 500
    assert np.array_equal(W > 0, upd)
    assert np.abs(D - expD).max() < 1e-12


def test_repeated_frames_and_cap():
    p = _dense(w_max=4.0)
    keys, centres = _voxel_centres(p)
    T = oracle.Tsdf(p)
    for n in range(1, 8):
        T.integrate(np.full((41, 41), 1.0, dtype=np.float32), CAM, Pose.identity())
        _, D, W, _ = T.dump()
        expD, upd = _expected_sphere(p, centres, 1.0, Pose.identity())
        assert np.abs(D - expD).max() < 1e-12           # identical frames leave D unchanged
        assert np.array_equal(W[upd], np.full(upd.sum(), min(n, 4.0)))


def test_alternating_frames_average():
    p = _dense()
    keys, centres = _voxel_centres(p)
    T = oracle.Tsdf(p)
    R1, R2 = np.float32(1.0), np.float32(1.1)
    for _ in range(3):
        T.integrate(np.full((41, 41), R1, dtype=np.float32), CAM, Pose.identity())
        T.integrate(np.full((41, 41), R2, dtype=np.float32), CAM, Pose.identity())
    _, D, W, _ = T.dump()
    d1, u1 = _expected_sphere(p, centres, R1, Pose.identity())
    d2, u2 = _expected_sphere(p, centres, R2, Pose.identity())
    both = u1 & u2
    assert both.sum() > 500
    assert np.abs(D[both] - 0.5 * (d1[both] + d2[both])).max() < 1e-12
    assert (W[both] == 6).all()
    only2 = u2 & ~u1                                   # seen only by the farther surface
    assert np.abs(D[only2] - d2[only2]).max() < 1e-12 and (W[only2] == 3).all()


def _hashed(voxel=0.05, mu=0.5, local_half=None):
    return TsdfParams(voxel_size=voxel, mu=mu, origin=(0.0, 0.0, 0.0), local_half=local_half)


def test_allocation_axis_ray():
    # Centre pixel of a pinhole-like camera (xi = 0, no distortion, principal
    # point on a pixel centre) looks along +z; from camera centre (0.05, 0.05,
    # 0) with range 2 and mu 0.5 the segment spans z in [1.5, 2.5] at
    # x = y = 0.05, crossing blocks (0, 0, 3..6) of side 8 * 0.05 = 0.4 m.
    cam = Camera(xi=0.0, fx=20, fy=20, cx=20, cy=20, width=41, height=41)
    depth = np.zeros((41, 41), dtype=np.float32)
    depth[20, 20] = 2.0
    C = np.array([0.05, 0.05, 0.0])
    T = oracle.Tsdf(_hashed())
    T.integrate(depth, cam, Pose(np.eye(3), -C))
    keys, D, W, amb = T.dump()
    assert [tuple(k) for k in keys] == [(0, 0, 3), (0, 0, 4), (0, 0, 5), (0, 0, 6)]
    strict, maybe = T.alloc_sets()
    assert len(strict) == 4 and len(maybe) == 0


def test_allocation_matches_point_sampling():
    rng = np.random.default_rng(11)
    cam = Camera(xi=1.0, fx=20, fy=20, cx=20, cy=20, width=41, height=41)
    depth = np.zeros((41, 41), dtype=np.float32)
    pix = [(int(rng.integers(0, 41)), int(rng.integers(0, 41))) for _ in range(40)]
    for (u, v) in pix:
        depth[v, u] = rng.uniform(0.6, 6.0)
    R_cw = rot_xyz(0.2, -0.3, 0.1)
    C = np.array([0.37, -0.11, 0.23])
    w2c = Pose(R_cw.T, -R_cw.T @ C)
    p = _hashed(voxel=0.05, mu=0.3)
    T = oracle.Tsdf(p)
    T.integrate(depth, cam, w2c)
    keys, _, _, _ = T.dump()
    got = set(map(tuple, keys))
    L = 8 * p.voxel_size
    sampled = set()
    for (u, v) in pix:
        r = oracle.unproject(cam, u, v)
        if r is None:
            continue
        d = float(depth[v, u])
        for s in np.arange(max(0.0, d - p.mu), d + p.mu + 1e-12, 1e-4):
            X = C + s * (R_cw @ r)
            sampled.add(tuple(np.floor(X / L).astype(int)))
    assert sampled <= got                     # every sampled block is allocated
    extra = got - sampled                     # allocated but unsampled: only grazing crossings
    strict, maybe = T.alloc_sets()
    assert len(extra) <= 0.02 * len(got) + 2


def test_local_map_gate():
    rng = np.random.default_rng(12)
    cam = Camera(xi=1.0, fx=20, fy=20, cx=20, cy=20, width=41, height=41)
    depth = rng.uniform(1.0, 12.0, size=(41, 41)).astype(np.float32)
    half = (3.0, 1.0, 3.0)
    centre = (0.5, 0.2, 4.0)
    Tg = oracle.Tsdf(_hashed(voxel=0.1, mu=0.5, local_half=half))
    Tg.integrate(depth, cam, Pose.identity(), local_center=centre)
    Tn = oracle.Tsdf(_hashed(voxel=0.1, mu=0.5))
    Tn.integrate(depth, cam, Pose.identity())
    kg = Tg.dump()[0]
    kn = Tn.dump()[0]
    L = 0.8
    cen = (kn + 0.5) * L
    inside = np.all(np.abs(cen - np.array(centre)) <= np.array(half), axis=1)
    assert len(kg) > 20 and len(kg) < len(kn)
    assert set(map(tuple, kg)) == set(map(tuple, kn[inside]))


def test_dense_and_hashed_agree_on_shared_blocks():
    depth = np.full((41, 41), 1.0, dtype=np.float32)
    pd = _dense(voxel=0.05, mu=0.2, dim=32, origin=(-0.8, -0.8, 0.0))
    ph = TsdfParams(voxel_size=0.05, mu=0.2, origin=(-0.8, -0.8, 0.0))
    Td, Th = oracle.Tsdf(pd), oracle.Tsdf(ph)
    Td.integrate(depth, CAM, Pose.identity())
    Th.integrate(depth, CAM, Pose.identity())
    kd, Dd, Wd, _ = Td.dump()
    kh, Dh, Wh, _ = Th.dump()
    idx = {tuple(k): i for i, k in enumerate(kd)}
    n = 0
    for i, k in enumerate(kh):
        if tuple(k) in idx:
            j = idx[tuple(k)]
            assert np.array_equal(Dh[i], Dd[j]) and np.array_equal(Wh[i], Wd[j])
            n += 1
    assert n > 10


def test_nearest_pixel_lookup():
    # Depth that varies per pixel: each voxel must read the depth of the pixel
    # nearest to its projection, (floor(u + 1/2), floor(v + 1/2)), found here
    # with the renderer's own projection code.
    p = _dense()
    keys, centres = _voxel_centres(p)
    uu, vv = np.meshgrid(np.arange(41), np.arange(41))
    depth = (0.9 + 0.004 * uu + 0.003 * vv).astype(np.float32)
    T = oracle.Tsdf(p)
    T.integrate(depth, CAM, Pose.identity())
    _, D, W, _ = T.dump()
    n = 0
    for i in range(centres.shape[0]):
        for v in range(centres.shape[1]):
            X = centres[i, v]
            u, vy = forward_project(CAM, X)
            if min(abs((u + 0.5) % 1.0 - 0.5), abs((vy + 0.5) % 1.0 - 0.5)) > 0.5 - 1e-6:
                continue
            pu, pv = math.floor(u + 0.5), math.floor(vy + 0.5)
            eta = float(depth[pv, pu]) - np.linalg.norm(X)
            if eta < -p.mu:
                assert W[i, v] == 0
                continue
            assert W[i, v] == 1 and abs(D[i, v] - min(1.0, eta / p.mu)) < 1e-12
            n += 1
    assert n > 1000


def test_swap_out_and_load():
    # blocks whose centre leaves the local map are removed and returned;
    # loading them back restores the map exactly
    rng = np.random.default_rng(13)
    cam = Camera(xi=1.0, fx=20, fy=20, cx=20, cy=20, width=41, height=41)
    depth = rng.uniform(1.0, 12.0, size=(41, 41)).astype(np.float32)
    p = _hashed(voxel=0.1, mu=0.5)
    T = oracle.Tsdf(p)
    T.integrate(depth, cam, Pose.identity())
    k0, D0, W0, _ = T.dump()
    pg = TsdfParams(voxel_size=0.1, mu=0.5, local_half=(2.0, 1.0, 3.0))
    Tg = oracle.Tsdf(pg)
    Tg.load(k0, D0, W0)
    centre = np.array([0.31, -0.17, 5.13])
    ks, Ds, Ws, amb = Tg.swap_out(centre)
    kk, DD, WW, _ = Tg.dump()
    L = 0.8
    cen = (k0 + 0.5) * L
    outside = np.any(np.abs(cen - centre) > np.array(pg.local_half), axis=1)
    assert 0 < outside.sum() < len(k0)
    assert set(map(tuple, ks)) == set(map(tuple, k0[outside]))
    assert set(map(tuple, kk)) == set(map(tuple, k0[~outside]))
    idx = {tuple(k): i for i, k in enumerate(k0)}
    for i, k in enumerate(ks):
        assert np.array_equal(Ds[i], D0[idx[tuple(k)]]) and np.array_equal(Ws[i], W0[idx[tuple(k)]])
    assert len(amb) == 0
    Tg.load(ks, Ds, Ws)
    k2, D2, W2, _ = Tg.dump()
    assert np.array_equal(k2, k0) and np.array_equal(D2, D0) and np.array_equal(W2, W0)
