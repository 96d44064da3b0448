"""Pins of the oracle's surface-point extraction from a block map: a planar
distance field crossed between two blocks (points exactly on the plane), a
sphere (points within the linear interpolation error), the observation
threshold, a missing neighbour block, and the count against a brute-force
numpy scan of the dense field."""
import numpy as np

import oracle

VOX = 0.1
MU = 0.3


def _blocks(field_fn, nb=(2, 2, 2), w=5.0):
    """Block map (keys, D, W) of a dense field sampled at voxel centres, origin 0."""
    keys, D, W = [], [], []
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                keys.append((bx, by, bz))
                v = np.arange(512)
                g = np.stack([bx * 8 + v % 8, by * 8 + (v // 8) % 8, bz * 8 + v // 64], 1)
                X = (g + 0.5) * VOX
                D.append(field_fn(X))
                W.append(np.full(512, w))
    return np.array(keys, np.int32), np.array(D), np.array(W)


def _dense(keys, D, W, nb=(2, 2, 2)):
    n = 8 * np.array(nb)
    Dd = np.zeros(tuple(n[::-1]))
    Wd = np.zeros(tuple(n[::-1]))
    for k, d, w in zip(keys, D, W):
        v = np.arange(512)
        x, y, z = k[0] * 8 + v % 8, k[1] * 8 + (v // 8) % 8, k[2] * 8 + v // 64
        Dd[z, y, x] = d
        Wd[z, y, x] = w
    return Dd, Wd


def test_plane_crossing_between_blocks():
    z0 = 0.83   # between voxel centres 0.75 (block 0) and 0.85 (block 1)
    keys, D, W = _blocks(lambda X: np.clip((z0 - X[:, 2]) / MU, -1, 1))
    pts, edges = oracle.tsdf_points(keys, D, W, 3.0, (0, 0, 0), VOX)
    assert len(pts) == 16 * 16
    assert (edges[:, 3] == 2).all() and (edges[:, 2] == 7).all()
    assert np.allclose(pts[:, 2], z0, atol=1e-12)
    assert np.allclose(np.sort(np.unique(pts[:, 0])), (np.arange(16) + 0.5) * VOX)


def test_observation_threshold_and_missing_neighbour():
    z0 = 0.83
    keys, D, W = _blocks(lambda X: np.clip((z0 - X[:, 2]) / MU, -1, 1))
    # voxels with x < 0.8 seen only twice: below the threshold of 3
    v = np.arange(512)
    for i, k in enumerate(keys):
        x = k[0] * 8 + v % 8
        W[i, x < 8] = 2.0
    pts, _ = oracle.tsdf_points(keys, D, W, 3.0, (0, 0, 0), VOX)
    assert len(pts) == 8 * 16 and (pts[:, 0] > 0.8).all()
    pts, _ = oracle.tsdf_points(keys, D, W, 2.0, (0, 0, 0), VOX)
    assert len(pts) == 16 * 16
    # unobserved voxels (w = 0) never count, whatever the threshold
    W0 = W.copy()
    W0[:] = 0
    assert len(oracle.tsdf_points(keys, D, W0, 0.0, (0, 0, 0), VOX)[0]) == 0
    # without the upper blocks the crossing has no neighbour
    lower = keys[:, 2] == 0
    pts, _ = oracle.tsdf_points(keys[lower], D[lower], W[lower], 3.0, (0, 0, 0), VOX)
    assert len(pts) == 0


def test_sphere_points_and_brute_force_count():
    c, R = np.array([0.8, 0.8, 0.8]), 0.5
    keys, D, W = _blocks(lambda X: np.clip((R - np.linalg.norm(X - c, axis=1)) / MU, -1, 1))
    pts, edges = oracle.tsdf_points(keys, D, W, 3.0, (0, 0, 0), VOX)
    r = np.linalg.norm(pts - c, axis=1)
    assert len(pts) > 300 and np.abs(r - R).max() < 0.01
    Dd, Wd = _dense(keys, D, W)
    n = 0
    for ax in range(3):   # numpy axes: z, y, x
        a = np.moveaxis(Dd, 2 - ax, 0)
        n += int(((a[:-1] > 0) != (a[1:] > 0)).sum())
    assert n == len(pts)
    # every edge is a sign change between its voxel and the next one along its axis
    for (gx, gy, gz, ax) in edges[:50]:
        nxt = [gx, gy, gz]
        nxt[ax] += 1
        assert (Dd[gz, gy, gx] > 0) != (Dd[nxt[2], nxt[1], nxt[0]] > 0)


def test_exact_zero_and_neighbour_weight():
    # exact binary voxel size: D = 0 exactly at voxel z = 7; zero counts as the
    # non-positive side, so the crossing is on the edge from z = 6, at z = 7's centre
    vox = 0.125
    z0 = 7.5 * vox
    keys, D, W = [], [], []
    for bz in range(2):
        v = np.arange(512)
        g = np.stack([v % 8, (v // 8) % 8, bz * 8 + v // 64], 1)
        keys.append((0, 0, bz))
        D.append(np.clip((z0 - (g[:, 2] + 0.5) * vox) / MU, -1, 1))
        W.append(np.full(512, 5.0))
    keys, D, W = np.array(keys, np.int32), np.array(D), np.array(W)
    assert (D[0][(np.arange(512) // 64) == 7] == 0).all()
    pts, edges = oracle.tsdf_points(keys, D, W, 3.0, (0, 0, 0), vox)
    assert len(pts) == 64 and (edges[:, 2] == 6).all() and np.allclose(pts[:, 2], z0, atol=1e-15)
    # the neighbour's observations count too: a crossing into a voxel seen twice is dropped
    z1 = 7.9 * vox   # crossing between z = 7 (block 0) and z = 8 (block 1)
    D2 = np.array([np.clip((z1 - (np.array([(v // 64) + 8 * b for v in range(512)]) + 0.5) * vox) / MU, -1, 1)
                   for b in range(2)])
    W2 = W.copy()
    W2[1] = 2.0
    assert len(oracle.tsdf_points(keys, D2, W, 3.0, (0, 0, 0), vox)[0]) == 64
    assert len(oracle.tsdf_points(keys, D2, W2, 3.0, (0, 0, 0), vox)[0]) == 0
