"""Pins of the oracle's depth map filtering (Sec. III-A, "Depth map filtering"):
best-cost threshold per image part, first/second-best uniqueness ratio, and
local depth continuity, on small maps whose outcome is worked out by hand."""
import numpy as np

import oracle
from scenes.configs import Filters

OFF = dict(alpha_upper=10.0, alpha_lower=10.0, ratio_min=0.0, gamma=1e9, delta=0.0)


def _lvl(d, c1, c2):
    return dict(depth=np.asarray(d, float), c1=np.asarray(c1, float), c2=np.asarray(c2, float))


def test_best_cost_threshold_by_image_part():
    # alpha = 0.05 above the middle row, 0.3 below (the paper's values)
    W = H = 8
    f = Filters(alpha_upper=0.05, alpha_lower=0.3, ratio_min=0.0, gamma=1e9, delta=0.0)
    lvl = _lvl(np.full((H, W), 2.0), np.full((H, W), 0.1), np.full((H, W), 1.0))
    out, amb = oracle.filter_frame(W, H, low=lvl, s=1, params=f)
    assert (out[:4] == 0).all() and (out[4:] == 2.0).all()
    # a 2x downsampled level: level row 1 has its centre at full row 2.5 (upper),
    # level row 2 at 4.5 (lower)
    lvl = _lvl(np.full((4, 4), 3.0), np.full((4, 4), 0.1), np.full((4, 4), 1.0))
    out, _ = oracle.filter_frame(W, H, low=lvl, s=2, params=f)
    assert (out[:4] == 0).all() and (out[4:] == 3.0).all()
    # exactly at the threshold: kept (an outlier is a cost *larger* than alpha)
    lvl = _lvl(np.full((H, W), 2.0), np.full((H, W), 0.05), np.full((H, W), 1.0))
    out, amb = oracle.filter_frame(W, H, low=lvl, s=1, params=f)
    assert (out == 2.0).all()
    assert amb[:4].all() and not amb[6:].any()      # c1 on the upper threshold; window reaches 2 rows


def test_uniqueness_ratio():
    W, H = 4, 2
    f = Filters(alpha_upper=1.0, alpha_lower=1.0, ratio_min=1.1, gamma=1e9, delta=0.0)
    c1 = np.full((H, W), 0.01)
    c2 = np.array([[0.0105, 0.0111, 0.02, np.inf], [0.01, 0.0109, 0.012, 0.5]])
    out, _ = oracle.filter_frame(W, H, low=_lvl(np.ones((H, W)), c1, c2), s=1, params=f)
    assert out.tolist() == [[0, 1, 1, 1], [0, 0, 1, 1]]


def test_local_continuity():
    # 7x7 map of depth 2 with one outlier at (3, 3): the outlier has no
    # consistent neighbour; every other pixel loses at most one of its
    # window neighbours to it
    W = H = 7
    d = np.full((H, W), 2.0)
    d[3, 3] = 10.0
    f = Filters(alpha_upper=1.0, alpha_lower=1.0, ratio_min=0.0, gamma=0.5, delta=0.3, window=5)
    lvl = _lvl(d, np.zeros((H, W)), np.ones((H, W)))
    out, _ = oracle.filter_frame(W, H, low=lvl, s=1, params=f)
    exp = d.copy()
    exp[3, 3] = 0.0
    assert np.array_equal(out, exp)
    # a pixel with exactly delta of its neighbours consistent survives:
    # corner (0, 0) has 8 in-image neighbours in a 5x5 window; make 5 of them
    # inconsistent -> 3/8 = 0.375 >= 0.3 kept; 6 inconsistent -> 2/8 = 0.25 dropped
    d = np.full((H, W), 2.0)
    nb = [(0, 1), (0, 2), (1, 0), (1, 1), (1, 2), (2, 0), (2, 1), (2, 2)]
    for (y, x) in nb[:5]:
        d[y, x] = 5.0
    out, _ = oracle.filter_frame(W, H, low=_lvl(d, np.zeros((H, W)), np.ones((H, W))), s=1, params=f)
    assert out[0, 0] == 2.0
    d[nb[5]] = 5.0
    out, _ = oracle.filter_frame(W, H, low=_lvl(d, np.zeros((H, W)), np.ones((H, W))), s=1, params=f)
    assert out[0, 0] == 0.0
    # pixels without depth count as inconsistent neighbours and stay empty
    d = np.zeros((H, W))
    d[3, 3] = 2.0
    out, _ = oracle.filter_frame(W, H, low=_lvl(d, np.zeros((H, W)), np.ones((H, W))), s=1, params=f)
    assert (out == 0).all()


def test_crop_falls_back_and_boxes_come_last():
    W, H = 8, 8
    f = Filters(alpha_upper=0.2, alpha_lower=0.2, ratio_min=0.0, gamma=0.5, delta=0.3, window=3)
    low = _lvl(np.full((4, 4), 4.0), np.full((4, 4), 0.1), np.ones((4, 4)))
    c1 = np.full((4, 4), 0.1)
    c1[0, 0] = 0.5                                     # fails alpha: the low level shows through
    crop = _lvl(np.full((4, 4), 4.2), c1, np.ones((4, 4)))
    boxes = np.array([[0, 0, 2, 8]], dtype=np.int32)   # columns 0..1 masked after the filters
    out, _ = oracle.filter_frame(W, H, low=low, s=2, crop=crop, crop_w=4, crop_h=4, params=f, boxes=boxes)
    exp = np.full((H, W), 4.0)
    exp[2:6, 2:6] = 4.2
    exp[2, 2] = 4.0
    exp[:, 0:2] = 0.0
    assert np.array_equal(out, exp)


def test_disabled_filters_equal_merge():
    rng = np.random.default_rng(0)
    W, H = 16, 12
    d = rng.uniform(1, 5, (H // 2, W // 2))
    lvl = _lvl(d, rng.uniform(0, 1, d.shape), rng.uniform(1, 2, d.shape))
    f = Filters(**OFF, window=3)
    out, amb = oracle.filter_frame(W, H, low=lvl, s=2, params=f)
    assert np.array_equal(out, oracle.merge(W, H, d, 2, None, 0, 0, None))
