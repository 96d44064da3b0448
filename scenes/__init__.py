"""Seeded synthetic inputs shared by the tests and the benchmark (input
synthesis only; none of the mapping method's arithmetic lives here)."""
from .render import Camera, Pose, Scene, Renderer, pixel_rays, forward_project, rot_xyz  # noqa: F401
from .configs import (FRONTO, GROUND, DOWNSAMPLE, CROP, PlaneSet, Level, Rig,  # noqa: F401
                      TsdfParams, Workload, FrameSource, Filters, tiny, street, ring, batch_mix, diff)
