"""Pins of the oracle's differentiable forms: the soft-argmin over plane
hypotheses (closed forms), the projection Jacobian (central differences of
the projection), the whole gradient of the soft-argmin range and soft-minimum
cost with respect to images and poses (FP64 central differences of the
forward), and the dense fusion and its gradient (the pinned sparse
integrator, closed forms, central differences)."""
import math

import numpy as np
import pytest

import oracle
import scenes
from scenes.configs import Level, PlaneSet, Rig, FRONTO, DOWNSAMPLE
from scenes.render import Camera, Pose, rot_xyz


# ----------------------------------------------------------------- soft-argmin

def test_soft_argmin_closed_forms():
    T = 0.05
    rho = np.array([0.1, 0.2, 0.5, 1.0])
    # equal costs: plain mean of the inverse ranges, S = C - T log K
    s, E, S = oracle.soft_argmin([0.3] * 4, rho, T)
    assert np.allclose(s, 0.25) and math.isclose(E, rho.mean(), rel_tol=1e-14)
    assert math.isclose(S, 0.3 - T * math.log(4), rel_tol=1e-14)
    # two valid planes: logistic weights; invalid planes get no weight
    s, E, S = oracle.soft_argmin([0.1, np.inf, 0.15, np.inf], rho, T)
    w = 1.0 / (1.0 + math.exp(-(0.15 - 0.1) / T))
    assert math.isclose(s[0], w, rel_tol=1e-14) and s[1] == 0 and s[3] == 0
    assert math.isclose(E, w * 0.1 + (1 - w) * 0.5, rel_tol=1e-14)
    assert math.isclose(S, 0.1 - T * math.log(1 + math.exp(-1.0)), rel_tol=1e-14)
    # a constant added to every cost changes nothing but S
    s2, E2, S2 = oracle.soft_argmin([0.1 + 7, np.inf, 0.15 + 7, np.inf], rho, T)
    assert np.allclose(s2, s, rtol=1e-12) and math.isclose(E2, E, rel_tol=1e-12)
    assert math.isclose(S2, S + 7, rel_tol=1e-12)
    # small temperature: the winner-take-all plane
    s, E, S = oracle.soft_argmin([0.4, 0.2, 0.3, 0.25], rho, 1e-4)
    assert math.isclose(E, 0.2, rel_tol=1e-12) and math.isclose(S, 0.2, rel_tol=1e-9)
    assert oracle.soft_argmin([np.inf] * 4, rho, T) is None


def test_soft_argmin_derivatives_by_central_differences():
    # dE/dC_k = -s_k (rho_k - E) / T and dS/dC_k = s_k, the forms the gradient uses
    rng = np.random.default_rng(0)
    T = 0.05
    C = rng.uniform(0, 0.5, 6)
    rho = rng.uniform(0.05, 1.0, 6)
    s, E, S = oracle.soft_argmin(C, rho, T)
    h = 1e-7
    for k in range(6):
        Cp, Cm = C.copy(), C.copy()
        Cp[k] += h
        Cm[k] -= h
        _, Ep, Sp = oracle.soft_argmin(Cp, rho, T)
        _, Em, Sm = oracle.soft_argmin(Cm, rho, T)
        assert math.isclose((Ep - Em) / (2 * h), -s[k] * (rho[k] - E) / T, rel_tol=1e-6, abs_tol=1e-9)
        assert math.isclose((Sp - Sm) / (2 * h), s[k], rel_tol=1e-6, abs_tol=1e-9)


# ----------------------------------------------------------------- projection Jacobian

@pytest.mark.parametrize("xi,dist", [(0.0, (0, 0, 0, 0)), (1.0, (0, 0, 0, 0)), (0.9, (0.02, -0.01, 0.003, -0.002)),
                                     (1.3, (-0.03, 0.01, -0.004, 0.005))])
def test_projection_jacobian_by_central_differences(xi, dist):
    k1, k2, p1, p2 = dist
    cam = Camera(xi=xi, fx=300.0, fy=310.0, cx=320.0, cy=240.0, width=640, height=480, k1=k1, k2=k2, p1=p1, p2=p2,
                 r2_max=2.5)
    rng = np.random.default_rng(1)
    n = 0
    for _ in range(200):
        X = rng.normal(size=3) * np.array([1.0, 1.0, 0.5]) + np.array([0, 0, 1.5])
        uv = oracle.project(cam, X)
        if uv is None:
            continue
        J = oracle.project_jacobian(cam, X)
        h = 1e-6
        for i in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[i] += h
            Xm[i] -= h
            a, b = oracle.project(cam, Xp), oracle.project(cam, Xm)
            fd = (np.asarray(a) - np.asarray(b)) / (2 * h)
            assert np.allclose(J[:, i], fd, rtol=1e-6, atol=1e-5 * (1 + np.abs(fd).max()))
        n += 1
    assert n > 100


# ----------------------------------------------------------------- whole soft-depth gradient

def _tiny_rig(seed=0, W=28, H=22, n_cams=2):
    """A small textured scene for central differences of the whole chain."""
    wl = scenes.diff(seed, width=W, height=H, n_planes=8)
    rig = Rig(ref=wl.rig.ref, cams=wl.rig.cams[:n_cams], ref_to_cam=wl.rig.ref_to_cam[:n_cams])
    wl.rig = rig
    imgs, _ = scenes.FrameSource(wl).frame(0)
    ims = [i.numpy().astype(np.float64) / 255.0 for i in imgs]
    return wl, ims


def _exp_left(p, w, v):
    """exp([w]x, v) T: rotation Exp(w) R, translation Exp(w) t + v."""
    th = np.linalg.norm(w)
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    Rw = np.eye(3) if th == 0 else np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
    return Pose(Rw @ np.asarray(p.R), Rw @ np.asarray(p.t) + v)


def _loss(wl, ims, g, gs, poses=None, T=0.05):
    r, S = oracle.soft_depth(wl.rig, wl.levels[0], ims, T=T, poses=poses, with_cost=True)
    return float((g * r).sum() + (gs * S).sum())


def test_soft_depth_gradient_by_central_differences():
    wl, ims = _tiny_rig()
    rng = np.random.default_rng(2)
    r0 = oracle.soft_depth(wl.rig, wl.levels[0], ims)
    assert (r0 > 0).mean() > 0.2
    g = rng.normal(size=r0.shape) * (r0 > 0)
    gs = rng.normal(size=r0.shape) * (r0 > 0)
    gi, gp = oracle.soft_depth_grad(wl.rig, wl.levels[0], ims, g, g_cost=gs)
    # poses: left perturbation of each ref_to_cam
    h = 1e-7
    fd = np.zeros_like(gp)
    for j in range(len(wl.rig.cams)):
        for i in range(6):
            e = np.zeros(6)
            e[i] = h
            pp = list(wl.rig.ref_to_cam)
            pm = list(wl.rig.ref_to_cam)
            pp[j] = _exp_left(pp[j], e[:3], e[3:])
            pm[j] = _exp_left(pm[j], -e[:3], -e[3:])
            fd[j, i] = (_loss(wl, ims, g, gs, pp) - _loss(wl, ims, g, gs, pm)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(gp - fd).max() <= 2e-4 * scale, (gp, fd)
    # images: random interior pixels of each image, including the reference
    # (whatever the analytic gradient says there)
    for m in range(len(ims)):
        H, W = ims[m].shape
        assert (np.abs(gi[m]) > 0).sum() > 20, m
        pick = np.stack([rng.integers(3, H - 3, 12), rng.integers(3, W - 3, 12)], 1)
        for (y, x) in pick:
            hp = [a.copy() for a in ims]
            hm = [a.copy() for a in ims]
            hp[m][y, x] += 1e-6
            hm[m][y, x] -= 1e-6
            d = (_loss(wl, hp, g, gs) - _loss(wl, hm, g, gs)) / 2e-6
            assert math.isclose(gi[m][y, x], d, rel_tol=1e-4, abs_tol=1e-5 * np.abs(gi[m]).max()), (m, y, x, d)
    # untouched pixels: no gradient
    g0 = np.zeros_like(g)
    gi0, gp0 = oracle.soft_depth_grad(wl.rig, wl.levels[0], ims, g0, g_cost=g0)
    assert all((a == 0).all() for a in gi0) and (gp0 == 0).all()


def test_soft_depth_min_over_cameras_routes_the_gradient():
    # with one camera the gradient of its pose equals the two-camera gradient
    # restricted to the planes that camera wins; here: a rig whose second
    # camera sees nothing (pointing backwards) gives the one-camera result
    wl, ims = _tiny_rig(n_cams=1)
    rng = np.random.default_rng(3)
    r = oracle.soft_depth(wl.rig, wl.levels[0], ims)
    g = rng.normal(size=r.shape) * (r > 0)
    gi1, gp1 = oracle.soft_depth_grad(wl.rig, wl.levels[0], ims, g)
    back = Pose(rot_xyz(0.0, math.pi, 0.0), np.zeros(3))
    rig2 = Rig(ref=wl.rig.ref, cams=[wl.rig.cams[0], wl.rig.cams[0]], ref_to_cam=[wl.rig.ref_to_cam[0], back])
    wl.rig = rig2
    gi2, gp2 = oracle.soft_depth_grad(wl.rig, wl.levels[0], [ims[0], ims[1], ims[1]], g)
    assert np.allclose(gp2[0], gp1[0], rtol=1e-12, atol=1e-12) and (gp2[1] == 0).all()
    assert np.allclose(gi2[0], gi1[0]) and np.allclose(gi2[1], gi1[1]) and (gi2[2] == 0).all()


# ----------------------------------------------------------------- dense fusion

def _dense_case(seed=0):
    cam = Camera(xi=1.0, fx=40.0, fy=40.0, cx=24.0, cy=20.0, width=48, height=40)
    nb = (2, 2, 2)
    origin = np.array([-0.8, -0.8, 1.2])
    rng = np.random.default_rng(seed)
    vox = np.zeros((8, 512, 2))
    vox[..., 0] = rng.uniform(-1, 1, (8, 512))
    vox[..., 1] = rng.integers(0, 5, (8, 512))
    return cam, nb, origin, vox


def test_dense_fuse_matches_the_pinned_integrator():
    # a fresh dense grid through orc_dense_fuse equals the sparse/dense
    # integrator pinned in test_oracle_tsdf (w = 0 start, two frames)
    from scenes.configs import TsdfParams
    cam, nb, origin, _ = _dense_case()
    p = TsdfParams(voxel_size=0.1, mu=0.3, w_max=100.0, dense_dim=(16, 16, 16), origin=tuple(origin))
    O = oracle.Tsdf(p)
    vox = np.zeros((8, 512, 2))
    rng = np.random.default_rng(4)
    for f in range(2):
        depth = (2.0 + 0.3 * rng.random((40, 48))).astype(np.float32)
        w2c = Pose(rot_xyz(0.02 * f, -0.03 * f, 0.0), np.array([0.05 * f, 0.0, 0.0]))
        vox = oracle.dense_fuse(vox, nb, origin, 0.1, 0.3, 100.0, depth, cam, w2c)
        O.integrate(depth, cam, w2c, None)
    k, D, W, _ = O.dump()
    order = np.lexsort((k[:, 0], k[:, 1], k[:, 2]))   # block b = bx + 2 (by + 2 bz)
    assert np.array_equal(W[order], vox[..., 1])
    assert np.allclose(D[order], vox[..., 0], rtol=0, atol=1e-14)
    assert (vox[..., 1] > 0).sum() > 500


def test_dense_fuse_closed_forms_and_gradient():
    cam, nb, origin, vox = _dense_case()
    w2c = Pose(rot_xyz(0.01, 0.02, 0.0), np.array([0.02, -0.01, 0.03]))
    R = 2.0
    depth = np.full((40, 48), R, np.float32)   # a sphere of range R: eta = R - |X_c|
    out = oracle.dense_fuse(vox, nb, origin, 0.1, 0.3, 4.0, depth, cam, w2c)
    # Eq. 2 by hand: every voxel that projects into the image with eta >= -mu
    b, v = np.nonzero(np.ones((8, 512), bool))
    gx = (b % 2) * 8 + v % 8
    gy = ((b // 2) % 2) * 8 + (v // 8) % 8
    gz = (b // 4) * 8 + v // 64
    X = origin + (np.stack([gx, gy, gz], 1) + 0.5) * 0.1
    Xc = X @ np.asarray(w2c.R).T + np.asarray(w2c.t)
    eta = R - np.linalg.norm(Xc, axis=1)
    inside = np.array([(lambda uv: uv is not None and -0.5 <= uv[0] < 47.5 and -0.5 <= uv[1] < 39.5)(
        oracle.project(cam, x)) for x in Xc])
    upd = inside & (eta >= -0.3)
    w = vox[b, v, 1]
    expD = np.where(upd, (w * vox[b, v, 0] + np.minimum(1.0, eta / 0.3)) / (w + 1), vox[b, v, 0])
    expW = np.where(upd, np.minimum(w + 1, 4.0), w)
    assert 200 < upd.sum() < upd.size
    assert np.allclose(out[b, v, 0], expD, rtol=0, atol=1e-13) and np.array_equal(out[b, v, 1], expW)
    b, v = b[upd], v[upd]
    # gradient against central differences (smooth depth: pixel choice does not matter)
    rng = np.random.default_rng(5)
    gD = rng.normal(size=(8, 512))
    gin, gd, gp = oracle.dense_fuse_grad(vox, nb, origin, 0.1, 0.3, 4.0, depth, cam, w2c, gD)
    L = lambda vx, dp, p: float((gD * oracle.dense_fuse(vx, nb, origin, 0.1, 0.3, 4.0, dp, cam, p)[..., 0]).sum())  # noqa: E731
    h = 1e-7
    fd = np.zeros(6)
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        fd[i] = (L(vox, depth, _exp_left(w2c, e[:3], e[3:])) - L(vox, depth, _exp_left(w2c, -e[:3], -e[3:]))) / (2 * h)
    assert np.allclose(gp, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    for (bb, vv) in [(int(b[0]), int(v[0])), (int(b[len(b) // 2]), int(v[len(v) // 2]))]:
        vp, vm = vox.copy(), vox.copy()
        vp[bb, vv, 0] += 1e-6
        vm[bb, vv, 0] -= 1e-6
        assert math.isclose(gin[bb, vv], (L(vp, depth, w2c) - L(vm, depth, w2c)) / 2e-6, rel_tol=1e-6)
    # depth pixels: a pixel's gradient is the sum over the voxels that read it
    for (y, x) in np.argwhere(gd != 0)[:5]:
        dp = depth.astype(np.float64)
        # float32 depth maps: perturb by an exactly representable step
        hp, hm = depth.copy(), depth.copy()
        hp[y, x] += np.float32(2 ** -10)
        hm[y, x] -= np.float32(2 ** -10)
        d = (L(vox, hp, w2c) - L(vox, hm, w2c)) / (2 * 2 ** -10)
        assert math.isclose(gd[y, x], d, rel_tol=1e-6), (y, x)
        del dp


def test_soft_depth_camera_ties_go_to_the_lowest_index():
    # two identical cameras at the same pose tie on every plane: the whole
    # gradient goes to the first, and equals the one-camera gradient
    wl, ims = _tiny_rig(n_cams=1)
    rng = np.random.default_rng(6)
    r = oracle.soft_depth(wl.rig, wl.levels[0], ims)
    g = rng.normal(size=r.shape) * (r > 0)
    gi1, gp1 = oracle.soft_depth_grad(wl.rig, wl.levels[0], ims, g)
    wl.rig = Rig(ref=wl.rig.ref, cams=[wl.rig.cams[0]] * 2, ref_to_cam=[wl.rig.ref_to_cam[0]] * 2)
    gi2, gp2 = oracle.soft_depth_grad(wl.rig, wl.levels[0], [ims[0], ims[1], ims[1]], g)
    assert np.array_equal(gp2[0], gp1[0]) and (gp2[1] == 0).all() and np.abs(gp1[0]).max() > 0
    assert np.array_equal(gi2[1], gi1[1]) and (gi2[2] == 0).all()


def test_tie_marks():
    # one camera: never tied; two identical cameras: every pixel with a valid plane is tied
    wl, ims = _tiny_rig(n_cams=1)
    assert not oracle.soft_depth_ties(wl.rig, wl.levels[0], ims).any()
    r = oracle.soft_depth(wl.rig, wl.levels[0], ims)
    wl.rig = Rig(ref=wl.rig.ref, cams=[wl.rig.cams[0]] * 2, ref_to_cam=[wl.rig.ref_to_cam[0]] * 2)
    amb = oracle.soft_depth_ties(wl.rig, wl.levels[0], [ims[0], ims[1], ims[1]])
    assert np.array_equal(amb, r > 0)


def test_grid_line_marks():
    # a zero-baseline identity camera samples exactly on the pixel grid: every
    # pixel with a valid plane is marked at any tau_px > 0, none at 0
    wl, ims = _tiny_rig(n_cams=1)
    wl.rig = Rig(ref=wl.rig.ref, cams=[wl.rig.ref], ref_to_cam=[Pose(np.eye(3), np.zeros(3))])
    valid = oracle.soft_depth(wl.rig, wl.levels[0], [ims[0], ims[0] + 0.01 * ims[1]]) > 0
    assert valid.any()
    assert not oracle.soft_depth_ties(wl.rig, wl.levels[0], [ims[0], ims[0] + 0.01 * ims[1]]).any()
    amb = oracle.soft_depth_ties(wl.rig, wl.levels[0], [ims[0], ims[0] + 0.01 * ims[1]], tau_px=1e-6)
    assert np.array_equal(amb, valid)
