"""Extrinsic refinement through the differentiable sweep.

Gradient descent on a left perturbation (w, v) of one matching camera's
ref_to_cam pose, with the loss
    mean over valid pixels of the soft-minimum matching cost
  + lam * mean over valid pixels of |range - range_ref| / range_ref,
where range_ref is a reference range map of the reference camera (a LiDAR
map in the paper's setting).  The photometric term alone cannot fix the
baseline's length (a longer baseline only resamples the same disparities);
the range term does.  Each step evaluates the gradient at the current pose
(delta = 0, where it is exact), lets Adam move delta and folds it into the
pose.  Every evaluation runs psdiff_forward / psdiff_backward.
"""
from __future__ import annotations

from typing import List

import torch

from .psweep import SoftSweep, se3_exp_left, soft_depth


def refine_extrinsic(sweep: SoftSweep, images, range_ref: torch.Tensor, pose0, steps: int = 50, lam: float = 0.3,
                     lr: float = 1e-3) -> List:
    """Poses after each step (pose0 first); the rig of `sweep` has one matching camera."""
    if len(sweep.rig.cams) != 1:
        raise ValueError("refine_extrinsic works on a rig with one matching camera")
    delta = torch.zeros((1, 6), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([delta], lr=lr)
    pose = pose0
    poses = [pose0]
    ref = range_ref
    for _ in range(steps):
        opt.zero_grad()
        rng, cost = soft_depth(sweep, images, delta, [pose])
        valid = (rng.detach() > 0) & (ref > 0)
        n = valid.sum().clamp_min(1)
        rel = (rng - ref) / torch.where(ref > 0, ref, torch.ones_like(ref))
        loss = (cost * valid).sum() / n + lam * (rel.abs() * valid).sum() / n
        loss.backward()
        opt.step()
        with torch.no_grad():
            pose = se3_exp_left(delta.detach().cpu().numpy()[0], pose)
            delta.zero_()
        poses.append(pose)
    return poses
