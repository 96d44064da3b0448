"""CPU checks of the parity helpers the GPU tests rely on: the bound on the
sub-plane fit's response to cost rounding must hold against the oracle's
own winner-take-all + parabola step, and the statistics must ignore
invalid pixels without arithmetic on infinities."""
import warnings

import numpy as np

import oracle
from scenes.configs import DOWNSAMPLE, FRONTO, GROUND, Level, PlaneSet
from tests.parity import fit_sensitivity, sweep_stats


def _param(S, i):
    t = i / (S.count - 1)
    if S.family == 0:
        return 1.0 / (1.0 / S.b + t * (1.0 / S.a - 1.0 / S.b))
    return S.a + t * (S.b - S.a)


def test_fit_sensitivity_bounds_the_parabola_response():
    lv = Level(kind=DOWNSAMPLE, factor=1, window=5,
               sets=[PlaneSet(FRONTO, 24, 0.5, 30.0), PlaneSet(GROUND, 9, 1.1, 2.1, n=(0.0, 1.0, 0.0))])
    planes = oracle.level_planes(lv)
    _, _, s_of, loc = planes
    K = lv.n_planes
    counts = [S.count for S in lv.sets]
    rng = np.random.default_rng(0)
    eps = 1e-5
    n_checked = 0
    for trial in range(400):
        k = int(rng.integers(1, K - 1))
        if not (0 < loc[k] < lv.sets[s_of[k]].count - 1):
            continue
        C = rng.uniform(0.3, 0.9, K)
        C[k] = rng.uniform(0.0, 0.2)
        C[k - 1] = C[k] + rng.uniform(1e-3, 0.05)
        C[k + 1] = C[k] + rng.uniform(1e-3, 0.05)
        bound = fit_sensitivity(C[None, :], np.array([k]), lv, planes, eps)[0]
        ks, _, _, d0 = oracle.wta(C, counts)
        assert ks == k
        S = lv.sets[s_of[k]]
        p0 = _param(S, loc[k] + d0)
        worst = 0.0
        for _ in range(20):
            Cp = C.copy()
            Cp[k - 1:k + 2] += rng.uniform(-eps, eps, 3)
            _, _, _, d1 = oracle.wta(Cp, counts)
            worst = max(worst, abs(_param(S, loc[k] + d1) - p0) / p0)
        # first-order bound: allow the second-order remainder
        assert worst <= bound * 1.05 + 1e-12, (trial, worst, bound)
        n_checked += 1
    assert n_checked > 200


def test_sweep_stats_on_invalid_pixels_is_quiet():
    inf = np.inf
    o = dict(kstar=np.array([-1, 3, 4, 5]), c1=np.array([inf, 0.1, 0.2, 0.1]), c2=np.array([inf, inf, 0.5, 0.3]),
             depth=np.array([0.0, 2.0, 3.0, 4.0]))
    g = dict(kstar=np.array([-1, 3, 4, 6]), c1=np.array([inf, 0.1, 0.2, 0.1]), c2=np.array([inf, inf, 0.5, 0.3]),
             depth=np.array([0.0, 2.0, 3.0001, 4.0]))
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        s = sweep_stats(o, g)
    # pixel 1 has a single valid plane (c2 = inf): gated; pixel 3 disagrees
    assert s["n_gated"] == 3 and s["n_index_disagree"] == 1 and s["n_depth_over"] == 0
