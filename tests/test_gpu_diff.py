"""GPU parity of the differentiable forms (psdiff_* and
tsdf_dense_fuse_backward through the C ABI) with the FP64 oracle: the
soft-argmin range and soft-minimum cost maps, their gradients with respect
to the images and the matching cameras' poses, central differences of the
GPU forward, the autograd wiring, and the dense fusion gradient."""
import math

import numpy as np
import pytest
import torch

import oracle
import scenes
from scenes.render import Pose, rot_xyz

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1809_06132_gb300 as P  # noqa: E402


@pytest.fixture(scope="module")
def case():
    wl = scenes.diff(0)                      # 96 x 80, ref + 2 matching cameras, 32 planes, 5 x 5
    imgs, rng = scenes.FrameSource(wl).frame(0, with_range=True)
    ims = [i.numpy().astype(np.float64) / 255.0 for i in imgs]
    dev = [torch.from_numpy(i.astype(np.float32)).cuda() for i in ims]
    # the oracle sees the same float32-rounded intensities
    ims = [d.double().cpu().numpy() for d in dev]
    sw = P.SoftSweep(wl.rig, wl.levels[0], temperature=0.05)
    return wl, ims, dev, sw, rng.numpy()


def test_forward_parity(case):
    wl, ims, dev, sw, _ = case
    r, S, aux = sw.forward(dev)
    torch.cuda.synchronize()
    r, S = r.cpu().numpy(), S.cpu().numpy()
    orr, oS = oracle.soft_depth(wl.rig, wl.levels[0], ims, T=0.05, with_cost=True)
    valid_agree = ((r > 0) == (orr > 0)).mean()
    both = (r > 0) & (orr > 0)
    rel = np.abs(r[both] - orr[both]) / orr[both]
    print("soft forward", dict(valid=float((orr > 0).mean()), agree=float(valid_agree),
                               rel_p50=float(np.median(rel)), rel_p999=float(np.quantile(rel, 0.999)),
                               S_abs_max=float(np.abs(S[both] - oS[both]).max())))
    assert (orr > 0).mean() > 0.8
    assert valid_agree >= 0.995
    assert np.median(rel) <= 1e-5 and (rel <= 1e-3).mean() >= 0.995
    assert (np.abs(S[both] - oS[both]) <= 1e-4).mean() >= 0.995


def _rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_gradient_parity_with_the_oracle(case):
    wl, ims, dev, sw, gt = case
    r, S, aux = sw.forward(dev)
    rng = np.random.default_rng(1)
    # pixels where float rounding decides an integer carry no loss: a plane's
    # camera (costs within 1e-5) or a window sample's bilinear cell (within
    # 3e-5 px of a grid line, where the slope in the pose gradient jumps)
    tied = oracle.soft_depth_ties(wl.rig, wl.levels[0], ims, tau=1e-5, tau_px=3e-5)
    valid = (r > 0).cpu().numpy() & ~tied
    g = (rng.normal(size=valid.shape) * valid).astype(np.float32)
    gs = (rng.normal(size=valid.shape) * valid).astype(np.float32)
    gi, gp = sw.backward(dev, None, aux, torch.from_numpy(g).cuda(), torch.from_numpy(gs).cuda())
    torch.cuda.synchronize()
    ogi, ogp = oracle.soft_depth_grad(wl.rig, wl.levels[0], ims, g.astype(np.float64), T=0.05,
                                      g_cost=gs.astype(np.float64))
    e_pose = [_rel_err(gp[j].cpu().numpy(), ogp[j]) for j in range(len(wl.rig.cams))]
    e_img = [_rel_err(gi[m].cpu().numpy(), ogi[m]) for m in range(len(ims))]
    print("gradient parity: tied pixels", int(tied.sum()), "pose rel err", e_pose, "image rel err", e_img)
    assert tied.mean() < 0.2
    assert max(e_pose) <= 1e-4
    assert max(e_img) <= 1e-4


def test_gradient_by_central_differences_of_the_gpu_forward(case):
    # loss = sum g * range + gs * cost on the GPU, pose steps of 1e-4 (rad, m).
    # One matching camera: the minimum over cameras is not smooth where two
    # cameras' costs cross, and a finite step straddles such crossings.
    wl, ims, dev, _, _ = case
    from scenes.configs import Rig
    rig1 = Rig(ref=wl.rig.ref, cams=wl.rig.cams[:1], ref_to_cam=wl.rig.ref_to_cam[:1])
    sw = P.SoftSweep(rig1, wl.levels[0], temperature=0.05)
    dev = dev[:2]
    rng = np.random.default_rng(2)
    r, _, aux = sw.forward(dev)
    valid = (r > 0).cpu().numpy()
    g = torch.from_numpy((rng.uniform(0.5, 1.5, size=valid.shape) * valid).astype(np.float32)).cuda()
    gs = torch.from_numpy((rng.uniform(0.5, 1.5, size=valid.shape) * valid).astype(np.float32)).cuda()
    _, gp = sw.backward(dev, None, aux, g, gs)
    gp = gp.cpu().numpy()

    def loss(poses):
        rr, SS, _ = sw.forward(dev, poses, want_aux=False)
        return float((g.double() * rr.double()).sum() + (gs.double() * SS.double()).sum())

    h = 1e-4
    fd = np.zeros_like(gp)
    for j in range(len(rig1.cams)):
        for i in range(6):
            e = np.zeros(6)
            e[i] = h
            pp = list(rig1.ref_to_cam)
            pm = list(rig1.ref_to_cam)
            pp[j] = P.se3_exp_left(e, pp[j])
            pm[j] = P.se3_exp_left(-e, pm[j])
            fd[j, i] = (loss(pp) - loss(pm)) / (2 * h)
    print("pose gradient", gp, "central differences", fd)
    assert _rel_err(gp, fd) <= 0.05


def test_autograd_images_and_pose(case):
    wl, ims, dev, sw, gt = case
    imgs = [d.clone().requires_grad_(True) for d in dev]
    delta = torch.zeros((len(wl.rig.cams), 6), dtype=torch.float64, requires_grad=True)
    r, S = P.soft_depth(sw, imgs, delta)
    valid = r.detach() > 0
    loss = (r * valid).sum() + 0.5 * (S * valid).sum()
    loss.backward()
    # the same through the explicit backward
    _, _, aux = sw.forward(dev)
    gi, gp = sw.backward(dev, None, aux, valid.float(), 0.5 * valid.float())
    torch.cuda.synchronize()
    assert torch.allclose(delta.grad, gp.cpu(), rtol=1e-6, atol=1e-9 * gp.abs().max().item())
    for a, b in zip(imgs, gi):
        assert torch.allclose(a.grad, b, rtol=1e-5, atol=1e-6 * b.abs().max().item())
        assert b.abs().max().item() > 0


@pytest.mark.parametrize("window,n_cams,n_planes", [(7, 3, 8), (9, 4, 8), (5, 2, 7)])
def test_wider_windows_and_more_cameras(window, n_cams, n_planes):
    # the other kernel instantiations (window radius 3 and 4), shared-memory
    # layouts (3 and 4 cameras) and an odd plane count (the forward takes
    # planes in pairs) against the oracle: forward maps and gradients
    import dataclasses
    wl = scenes.diff(5, width=64, height=48, n_planes=n_planes)
    cams, poses = list(wl.rig.cams), list(wl.rig.ref_to_cam)
    for k, dy in enumerate((-0.3, 0.3)[:n_cams - 2]):
        R = rot_xyz(math.radians(0.5 * (k + 1)), math.radians(-0.4), 0.0)
        poses.append(Pose(R.T, -R.T @ np.array([0.1, dy, 0.0])))
        cams.append(cams[k])
    wl.rig = dataclasses.replace(wl.rig, cams=cams, ref_to_cam=poses)
    wl.levels = [dataclasses.replace(wl.levels[0], window=window)]
    imgs, _ = scenes.FrameSource(wl).frame(0)
    dev = [torch.from_numpy((i.numpy().astype(np.float64) / 255.0).astype(np.float32)).cuda() for i in imgs]
    ims = [d.double().cpu().numpy() for d in dev]
    sw = P.SoftSweep(wl.rig, wl.levels[0], temperature=0.05)
    r, S, aux = sw.forward(dev)
    orr = oracle.soft_depth(wl.rig, wl.levels[0], ims, T=0.05)
    rc = r.cpu().numpy()
    both = (rc > 0) & (orr > 0)
    assert both.mean() > 0.3 and ((rc > 0) == (orr > 0)).mean() >= 0.99
    assert np.median(np.abs(rc[both] - orr[both]) / orr[both]) <= 1e-5
    tied = oracle.soft_depth_ties(wl.rig, wl.levels[0], ims, tau=1e-5, tau_px=3e-5)
    valid = (rc > 0) & ~tied
    rng = np.random.default_rng(2)
    g = (rng.normal(size=valid.shape) * valid).astype(np.float32)
    gs = (rng.normal(size=valid.shape) * valid).astype(np.float32)
    gi, gp = sw.backward(dev, None, aux, torch.from_numpy(g).cuda(), torch.from_numpy(gs).cuda())
    torch.cuda.synchronize()
    ogi, ogp = oracle.soft_depth_grad(wl.rig, wl.levels[0], ims, g.astype(np.float64), T=0.05,
                                      g_cost=gs.astype(np.float64))
    e_pose = [_rel_err(gp[j].cpu().numpy(), ogp[j]) for j in range(n_cams) if np.abs(ogp[j]).max() > 0]
    e_img = [_rel_err(gi[m].cpu().numpy(), ogi[m]) for m in range(1 + n_cams) if np.abs(ogi[m]).max() > 0]
    print(f"window {window}, {n_cams} cameras, {n_planes} planes: tied", int(tied.sum()), "pose", e_pose,
          "image", e_img)
    assert len(e_pose) >= 2 and len(e_img) >= 3
    assert max(e_pose) <= 1e-4 and max(e_img) <= 1e-4


def _sphere_case():
    cam = scenes.Camera(xi=1.0, fx=40.0, fy=40.0, cx=24.0, cy=20.0, width=48, height=40)
    from scenes.configs import TsdfParams
    p = TsdfParams(voxel_size=0.1, mu=0.3, w_max=4.0, dense_dim=(16, 16, 16), origin=(-0.8, -0.8, 1.2))
    rng = np.random.default_rng(0)
    vox = np.zeros((8, 512, 2), np.float32)
    vox[..., 0] = rng.uniform(-1, 1, (8, 512))
    vox[..., 1] = rng.integers(0, 5, (8, 512))
    depth = (2.0 + 0.05 * np.sin(np.arange(40 * 48).reshape(40, 48) / 50.0)).astype(np.float32)
    w2c = Pose(rot_xyz(0.01, 0.02, 0.0), np.array([0.02, -0.01, 0.03]))
    return cam, p, vox, depth, w2c


def test_dense_fuse_forward_and_gradient_parity():
    cam, p, vox, depth, w2c = _sphere_case()
    rng = np.random.default_rng(7)
    gD = rng.normal(size=(8, 512)).astype(np.float32)
    v = torch.from_numpy(vox).cuda()
    d = torch.from_numpy(depth).cuda()
    out = P.dense_fuse(v, d, p, cam, w2c)
    gin, gd, gp = P.psweep.tsdf_dense_fuse_backward(v, p.dense_dim, p.origin, p.voxel_size, p.mu, p.w_max, d, cam,
                                                     w2c, torch.from_numpy(gD).cuda())
    torch.cuda.synchronize()
    nb = (2, 2, 2)
    o_out = oracle.dense_fuse(vox.astype(np.float64), nb, p.origin, p.voxel_size, p.mu, p.w_max, depth, cam, w2c)
    o_gin, o_gd, o_gp = oracle.dense_fuse_grad(vox.astype(np.float64), nb, p.origin, p.voxel_size, p.mu, p.w_max,
                                               depth, cam, w2c, gD.astype(np.float64))
    out = out.cpu().numpy()
    assert (np.abs(out[..., 0] - o_out[..., 0]) <= 1e-5).mean() >= 0.999
    assert (out[..., 1] == o_out[..., 1]).mean() >= 0.999
    gin, gd, gp = gin.cpu().numpy(), gd.cpu().numpy(), gp.cpu().numpy()
    assert (np.abs(gin - o_gin) <= 1e-5 * np.abs(gD).max()).mean() >= 0.999
    print("dense fuse grad: depth rel err", _rel_err(gd, o_gd), "pose rel err", _rel_err(gp, o_gp))
    assert _rel_err(gd, o_gd) <= 1e-3 and _rel_err(gp, o_gp) <= 1e-3
    # autograd: gradients of the D channel reach voxels, depth and pose
    vv = v.clone().requires_grad_(True)
    dd = d.clone().requires_grad_(True)
    delta = torch.zeros(6, dtype=torch.float64, requires_grad=True)
    o = P.dense_fuse(vv, dd, p, cam, w2c, delta)
    (o[..., 0] * torch.from_numpy(gD).cuda()).sum().backward()
    assert torch.allclose(vv.grad[..., 0].cpu(), torch.from_numpy(gin), atol=1e-7)
    assert (vv.grad[..., 1] == 0).all()
    # float atomics add in any order: equal to rounding
    assert torch.allclose(dd.grad.cpu(), torch.from_numpy(gd), rtol=1e-5, atol=1e-6 * np.abs(gd).max())
    assert torch.allclose(delta.grad, torch.from_numpy(gp), rtol=1e-5, atol=1e-9 * np.abs(gp).max())


def _pose_error(p, true):
    dR = np.asarray(p.R) @ np.asarray(true.R).T
    ang = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(dR) - 1) / 2))))
    return ang, float(np.linalg.norm(np.asarray(p.t) - np.asarray(true.t)))


def test_extrinsic_refinement_from_a_perturbed_pose():
    # 192 x 160 version of the rig, 64 planes, the right camera perturbed by
    # 0.5 degrees and 2 cm; 50 steps of the photometric + range loss
    from paper_1809_06132_gb300.refine import refine_extrinsic
    from scenes.configs import Rig
    wl = scenes.diff(0, width=192, height=160, n_planes=64)
    imgs, rng = scenes.FrameSource(wl, device="cuda").frame(0, with_range=True)
    rig = Rig(ref=wl.rig.ref, cams=wl.rig.cams[1:], ref_to_cam=wl.rig.ref_to_cam[1:])
    dev = [torch.from_numpy(imgs[0].numpy().astype(np.float32) / 255.0).cuda(),
           torch.from_numpy(imgs[2].numpy().astype(np.float32) / 255.0).cuda()]
    gt = torch.from_numpy(rng.numpy().astype(np.float32)).cuda()
    true = rig.ref_to_cam[0]
    r = np.random.default_rng(0)
    ax = r.normal(size=3)
    tv = r.normal(size=3)
    xi0 = np.concatenate([ax / np.linalg.norm(ax) * math.radians(0.5), tv / np.linalg.norm(tv) * 0.02])
    pose0 = P.se3_exp_left(xi0, true)
    sw = P.SoftSweep(rig, wl.levels[0], temperature=0.05)
    poses = refine_extrinsic(sw, dev, gt, pose0, steps=50, lam=0.3, lr=1e-3)
    errs = [_pose_error(p, true) for p in poses]
    print("refinement (deg, m):", [(round(a, 3), round(t, 4)) for a, t in errs[::10] + [errs[-1]]])
    a0, t0 = errs[0]
    a1, t1 = errs[-1]
    assert abs(a0 - 0.5) < 1e-6 and t0 > 0.015
    assert a1 < 0.15 and t1 < 0.008
