"""Pins of the oracle's unified fisheye camera model (Sec. III-C, Eq. 1).

Each check compares the oracle with something other than itself: closed
forms of the sphere model, the pinhole special case, the scene renderer's
independent pixel-ray route (bisection on the polar angle), random
directions on the validity boundary, and exact round trips.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from scenes.render import Camera, pixel_rays

CAMS = [
    Camera(xi=0.0, fx=120, fy=110, cx=63.5, cy=47.25, width=128, height=96),
    Camera(xi=0.5, fx=90, fy=95, cx=64.0, cy=48.0, width=128, height=96),
    Camera(xi=0.8, fx=80, fy=80, cx=64.2, cy=47.7, width=128, height=96),
    Camera(xi=1.0, fx=80, fy=80, cx=80, cy=64, width=160, height=128),
    Camera(xi=1.2, fx=60, fy=62, cx=64, cy=48, width=128, height=96),
    Camera(xi=2.0, fx=150, fy=150, cx=64, cy=48, width=128, height=96),
    Camera(xi=1.1, fx=70, fy=70, cx=64, cy=48, width=128, height=96,
           k1=-0.03, k2=0.01, p1=0.004, p2=-0.006, r2_max=2.5),
    Camera(xi=0.9, fx=64, fy=64, cx=64, cy=48, width=128, height=96,
           k1=0.02, k2=-0.005, p1=-0.003, p2=0.002, r2_max=2.5),
]


def test_stereographic_closed_form():
    # xi = 1 without distortion is the stereographic projection: a direction at
    # polar angle theta lands at normalised radius tan(theta / 2).
    cam = Camera(xi=1.0, fx=100, fy=100, cx=50, cy=50, width=100, height=100)
    for theta in (0.1, math.pi / 4, 1.2, 2.0, 2.8):
        for phi in (0.0, 0.7, 2.5, -1.9):
            X = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)]) * 3.7
            uv = oracle.project(cam, X)
            rho = math.tan(theta / 2)
            assert uv is not None
            assert abs(uv[0] - (50 + 100 * rho * math.cos(phi))) < 1e-9
            assert abs(uv[1] - (50 + 100 * rho * math.sin(phi))) < 1e-9
    # theta = 45 deg: tan(22.5 deg) = sqrt(2) - 1
    uv = oracle.project(cam, np.array([1.0, 0.0, 1.0]))
    assert abs(uv[0] - (50 + 100 * (math.sqrt(2) - 1))) < 1e-12


def test_pinhole_special_case():
    # xi = 0 reduces Eq. 1 to the pinhole ray (x, y, 1) / |(x, y, 1)|.
    cam = CAMS[0]
    X = np.array([1.0, 2.0, 4.0])
    uv = oracle.project(cam, X)
    assert abs(uv[0] - (cam.cx + cam.fx * 0.25)) < 1e-12
    assert abs(uv[1] - (cam.cy + cam.fy * 0.5)) < 1e-12
    for u, v in [(0, 0), (10.5, 80), (127, 95), (63.5, 47.25)]:
        r = oracle.unproject(cam, u, v)
        x, y = (u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy
        ref = np.array([x, y, 1.0]) / math.sqrt(x * x + y * y + 1)
        assert np.allclose(r, ref, atol=1e-15)


def test_xi_half_side_direction():
    # xi = 0.5: a direction perpendicular to the axis lands at radius 1 / xi = 2.
    cam = Camera(xi=0.5, fx=10, fy=10, cx=0, cy=0, width=100, height=100)
    uv = oracle.project(cam, np.array([5.0, 0.0, 0.0]))
    assert abs(uv[0] - 20.0) < 1e-12 and abs(uv[1]) < 1e-12


@pytest.mark.parametrize("ci", range(len(CAMS)))
def test_eq1_matches_independent_bisection(ci):
    # The renderer finds each ray by bisection on theta of
    # rho = sin(theta) / (cos(theta) + xi) and inverts distortion by
    # fixed-point iteration; Eq. 1 must give the same unit rays.
    cam = CAMS[ci]
    us = np.arange(0, cam.width, 7, dtype=np.float64)
    vs = np.arange(0, cam.height, 5, dtype=np.float64)
    U, V = np.meshgrid(us, vs)
    rays, valid = pixel_rays(cam, torch.tensor(U.reshape(-1)), torch.tensor(V.reshape(-1)))
    rays = rays.numpy()
    valid = valid.numpy()
    n_checked = 0
    for i, (u, v) in enumerate(zip(U.reshape(-1), V.reshape(-1))):
        r = oracle.unproject(cam, u, v)
        if r is None:
            assert not valid[i], (u, v)
            continue
        assert valid[i], (u, v)
        assert abs(np.linalg.norm(r) - 1) < 1e-14
        assert np.allclose(r, rays[i], atol=1e-10), (u, v, r, rays[i])
        n_checked += 1
    assert n_checked > 100


@pytest.mark.parametrize("ci", range(len(CAMS)))
def test_round_trip(ci):
    cam = CAMS[ci]
    rng = np.random.default_rng(ci)
    n = 0
    for _ in range(400):
        u = rng.uniform(0, cam.width - 1)
        v = rng.uniform(0, cam.height - 1)
        r = oracle.unproject(cam, u, v)
        if r is None:
            continue
        uv = oracle.project(cam, r * rng.uniform(0.3, 40.0))
        assert uv is not None
        assert abs(uv[0] - u) < 1e-9 and abs(uv[1] - v) < 1e-9
        n += 1
    assert n > 150


@pytest.mark.parametrize("xi", [0.0, 0.5, 0.8, 1.0, 1.2, 2.0])
def test_validity_boundary(xi):
    # The forward map is accepted exactly where the sphere point has
    # z_s > -min(xi, 1/xi), and there Eq. 1 inverts it.
    cam = Camera(xi=xi, fx=1, fy=1, cx=0, cy=0, width=1, height=1)
    lim = min(xi, 1 / xi) if xi > 0 else 0.0
    rng = np.random.default_rng(7)
    D = rng.normal(size=(20000, 3))
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    for d in D:
        uv = oracle.project(cam, d)
        inside = d[2] > -lim
        assert (uv is not None) == inside
        if uv is not None and d[2] > -lim + 1e-6:
            r = oracle.unproject(cam, uv[0], uv[1])
            assert r is not None
            assert np.allclose(r, d, atol=1e-7)


def test_distortion_inverse():
    cam = CAMS[6]
    rng = np.random.default_rng(3)
    for _ in range(300):
        x, y = rng.uniform(-1.1, 1.1, size=2)
        xd, yd = oracle.distort(cam, x, y)
        m = oracle.undistort(cam, xd, yd)
        assert m is not None
        assert abs(m[0] - x) < 1e-12 and abs(m[1] - y) < 1e-12
    plain = Camera(xi=1.0, fx=1, fy=1, cx=0, cy=0, width=1, height=1)
    assert np.array_equal(oracle.distort(plain, 0.3, -0.7), [0.3, -0.7])
