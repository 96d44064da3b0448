"""Comparison of the CUDA library's outputs with the FP64 oracle's.

Criteria (all computed on the same seeded inputs):
  * winning plane: identical on >= 99.9% of pixels whose oracle margin
    (second-best minus best cost) exceeds 1e-3;
  * depth: |gpu - oracle| <= 1e-4 * oracle on >= 99.9% of those pixels
    where the plane agrees (the rest is bounded by one plane spacing);
  * validity (a depth at all): identical on >= 99.9% of pixels; a
    mismatch needs a warped sample or a window variance within float
    rounding of a validity threshold;
  * TSDF: |D_gpu - D_oracle| <= 1e-5 and W identical on every voxel whose
    history the oracle does not mark rounding-sensitive.
"""
import numpy as np

MARGIN = 1e-3
DEPTH_REL = 1e-4
FRAC = 0.999
TSDF_ABS = 1e-5


def sweep_stats(o, g):
    """o, g: dicts with depth, c1, c2, kstar (same shape)."""
    ok, gk = o["kstar"], g["kstar"]
    ov, gv = ok >= 0, gk >= 0
    n = ok.size
    gated = ov & gv & ((o["c2"] - o["c1"]) > MARGIN)
    agree = gated & (ok == gk)
    od = o["depth"][agree]
    rel = np.abs(g["depth"][agree] - od) / np.maximum(od, 1e-30)
    c1err = np.abs(g["c1"][agree] - o["c1"][agree])
    return dict(
        n=int(n),
        n_valid_oracle=int(ov.sum()),
        valid_mismatch=float((ov != gv).mean()),
        n_gated=int(gated.sum()),
        index_agree=float(agree.sum() / max(1, gated.sum())),
        depth_ok=float((rel <= DEPTH_REL).mean()) if rel.size else 1.0,
        depth_rel_p50=float(np.median(rel)) if rel.size else 0.0,
        depth_rel_p999=float(np.quantile(rel, 0.999)) if rel.size else 0.0,
        depth_rel_max=float(rel.max()) if rel.size else 0.0,
        c1_abs_max=float(c1err.max()) if c1err.size else 0.0,
        c1_abs_p50=float(np.median(c1err)) if c1err.size else 0.0,
    )


def assert_sweep_parity(o, g, min_gated=50):
    s = sweep_stats(o, g)
    assert s["n_gated"] >= min_gated, s
    assert s["valid_mismatch"] <= 1 - FRAC, s
    assert s["index_agree"] >= FRAC, s
    assert s["depth_ok"] >= FRAC, s
    return s


def tsdf_compare(o_keys, o_D, o_W, o_amb, g_keys, g_D, g_W):
    """Match blocks by key; compare voxels not marked ambiguous."""
    gi = {tuple(int(v) for v in k): i for i, k in enumerate(g_keys)}
    common = [(i, gi[tuple(int(v) for v in k)]) for i, k in enumerate(o_keys) if tuple(int(v) for v in k) in gi]
    if not common:
        return dict(n_common=0)
    oi = np.array([a for a, _ in common])
    gj = np.array([b for _, b in common])
    amb = o_amb[oi]
    clean = ~amb
    dD = np.abs(g_D[gj] - o_D[oi])[clean]
    wW = (g_W[gj] != o_W[oi])[clean]
    return dict(n_common=len(common), n_voxels=int(clean.sum()), n_amb=int(amb.sum()),
                D_abs_max=float(dD.max()) if dD.size else 0.0, W_mismatch=int(wW.sum()),
                n_updated=int((o_W[oi][clean] > 0).sum()))
