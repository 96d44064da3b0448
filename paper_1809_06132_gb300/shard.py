"""Multi-GPU split of one frame's path, one process per GPU
(torch.distributed): host orchestration only, every step runs in the
library's kernels.

* The sweep's plane hypotheses are independent until the winner-take-all
  (Sec. III-A), so each rank sweeps one consecutive plane range of every
  level (psweep_depth_planes), the ranks exchange their per-pixel records
  in one all-gather of plain buffers, and every rank merges all records
  into the frame's depth map (psweep_merge_records), bit-identical to a
  one-GPU psweep_depth.
* TSDF fusion updates each voxel block from the depth map and its own
  state alone (Sec. III-C), so rank r fuses the merged depth map into the
  blocks whose key hashes to part r (tsdf_set_partition); the union of the
  ranks' maps is the one-GPU map.

The exchange moves 7 floats per pixel and level per rank: 7 x (320 x 256
+ 640 x 512) x 4 B = 11.5 MB per rank for the street frame.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import torch
import torch.distributed as dist


def split_planes(n_planes: Sequence[int], world: int) -> List[Tuple[List[int], List[int]]]:
    """Consecutive, balanced plane ranges: for each rank, (lo, hi) lists with
    one entry per level; ranks in order cover every plane exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    out = []
    for r in range(world):
        lo = [k * r // world for k in n_planes]
        hi = [k * (r + 1) // world for k in n_planes]
        out.append((lo, hi))
    return out


def exchange_records(records: Sequence[torch.Tensor], group=None) -> List[List[torch.Tensor]]:
    """All-gather every rank's per-level records (same shapes on every rank):
    result[rank][level], in rank order.  One collective of one flat buffer;
    works on CUDA tensors (NCCL) and CPU tensors (gloo)."""
    world = dist.get_world_size(group)
    flat = torch.cat([r.reshape(-1) for r in records])
    parts = [torch.empty_like(flat) for _ in range(world)]
    dist.all_gather(parts, flat, group=group)
    out = []
    for p in parts:
        per, off = [], 0
        for r in records:
            n = r.numel()
            per.append(p[off:off + n].view(r.shape))
            off += n
        out.append(per)
    return out


class ShardedFrame:
    """One frame on `world` ranks: this rank's plane ranges, the exchange,
    the merge, and the fusion of the merged map into this rank's hash part
    of the map (tsdf may be None: depth only)."""

    def __init__(self, sweep, tsdf=None, group=None):
        self.sw = sweep
        self.T = tsdf
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.ranges = split_planes(sweep.n_planes(), self.world)
        self.part_lo = [lo for lo, _ in self.ranges]
        self.records = None
        if tsdf is not None:
            tsdf.set_partition(self.world, self.rank)

    def step(self, images, boxes=None, world_to_ref=None, local_center=None, out=None, level_outs=None,
             stream=None):
        lo, hi = self.ranges[self.rank]
        if self.records is None:
            self.records = self.sw.alloc_records(images[0].device)
        self.sw.depth_planes(images, lo, hi, records=self.records, stream=stream)
        if stream is not None:
            stream.synchronize()  # the collective runs on the process group's own stream
        gathered = exchange_records(self.records, self.group)
        depth = self.sw.merge_records(self.part_lo, gathered, boxes=boxes, out=out, level_outs=level_outs,
                                      stream=stream)
        if self.T is not None and world_to_ref is not None:
            self.T.integrate(depth, world_to_ref, local_center, stream=stream)
        return depth
