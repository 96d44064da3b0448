"""Batched sweeps (psbatch_* through the C ABI): many uneven depth maps in one
persistent launch give the same maps as psweep_depth on each sweep, for
every queue order, plane chunk, grid size and pass width, and within float
rounding for the 16-row tile shape; graph replay picks up new inputs; the
bounded dependency wait reports a timeout and leaves the context usable."""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1809_06132_gb300 as P  # noqa: E402

PREP_ROWS = MERGE_ROWS = 16


def _cdiv(a, b):
    return -(-a // b)


@pytest.fixture(scope="module")
def mix():
    """Uneven sweeps: drawn sizes / plane counts / 1-4 matching cameras, a
    two-level street rig with the depth filters, the same rig with FP16
    matching images, and the one-camera tiny rig."""
    wls = scenes.batch_mix(1, n=7, sizes=((256, 200), (320, 256), (640, 512)), planes=(32, 64, 128))
    st = scenes.street(0, n_frames=1, scale=0.25)
    wls += [st, st, scenes.tiny(0)]
    filt = [None] * 7 + [scenes.Filters(), None, None]
    half = [False] * 8 + [True, False]
    sweeps, images, boxes, single = [], [], [], []
    for wl, f, hf in zip(wls, filt, half):
        imgs, _ = scenes.FrameSource(wl, device="cuda").frame(0)
        dev = [torch.from_numpy(np.ascontiguousarray(i.numpy())).cuda() for i in imgs]
        sw = P.Sweep(wl.rig, wl.levels, filters=f, image_half=hf)
        sweeps.append(sw)
        images.append(dev)
        boxes.append(wl.boxes[0])
        single.append(sw.depth(dev, boxes=wl.boxes[0]).clone())
    torch.cuda.synchronize()
    return dict(wls=wls, sweeps=sweeps, images=images, boxes=boxes, single=single, filt=filt)


def _run(mix, **kw):
    b = P.Batch(mix["sweeps"], **kw)
    outs = b.run(mix["images"], boxes=mix["boxes"])
    torch.cuda.synchronize()
    assert b.status() == P.PS_OK
    return b, outs


def test_batch_equals_single_sweeps(mix):
    b, outs = _run(mix)
    for i, (o, s) in enumerate(zip(outs, mix["single"])):
        assert (s > 0).float().mean().item() > 0.2, i
        assert torch.equal(o, s), f"sweep {i}: {(o != s).sum().item()} pixels differ"


@pytest.mark.parametrize("kw", [dict(kp=1), dict(plane_chunk=8), dict(plane_chunk=4096), dict(plane_chunk=5, kp=1),
                                dict(order=P.BATCH_GIVEN_ORDER), dict(grid=5)])
def test_batch_options_keep_results(mix, kw):
    # one or two planes per pass, any plane chunk, queue order or grid size:
    # the same arithmetic per pixel and plane, so the same maps
    _, outs = _run(mix, **kw)
    for i, (o, s) in enumerate(zip(outs, mix["single"])):
        assert torch.equal(o, s), f"{kw} sweep {i}: {(o != s).sum().item()} pixels differ"


@pytest.mark.parametrize("kp", [1, 2])
def test_batch_16_row_tiles(mix, kp):
    # 16-row tiles slide the vertical window sums from other starting rows:
    # the maps agree to float rounding (ties of nearly equal planes aside)
    _, outs = _run(mix, tile_h=16, kp=kp, plane_chunk=16)
    for i, (o, s) in enumerate(zip(outs, mix["single"])):
        o, s = o.cpu().numpy(), s.cpu().numpy()
        assert ((o > 0) != (s > 0)).mean() < 0.005, i
        both = (o > 0) & (s > 0)
        rel = np.abs(o[both] - s[both]) / s[both]
        assert (rel <= 1e-4).mean() >= 0.995, (i, float((rel <= 1e-4).mean()))


def test_batch_queue_and_timing(mix):
    b, _ = _run(mix)
    q = b.queue_stats()
    exp = dict(ref=0, quad=0, stats=0, sweep=0, merge=0, continuity=0)
    for sw, f in zip(mix["sweeps"], mix["filt"]):
        for (h, w), lv in zip(sw.level_shapes(), sw.levels):
            exp["ref"] += _cdiv(h, PREP_ROWS)
            exp["stats"] += _cdiv(h, PREP_ROWS)
            exp["quad"] += sum(_cdiv(c.height // (lv.factor if lv.kind == 0 else 1), PREP_ROWS) for c in sw.rig.cams)
            n_chunks = _cdiv(lv.n_planes, 32)
            exp["sweep"] += _cdiv(w, 64) * _cdiv(h, 24) * n_chunks
        exp["merge"] += _cdiv(sw.rig.ref.height, MERGE_ROWS)
        if f is not None:
            exp["continuity"] += _cdiv(sw.rig.ref.height, MERGE_ROWS)
    assert q == exp
    done, span = b.timing()
    assert all(0 < d <= span for d in done)
    assert span == max(done)


def test_batch_graph_replay_takes_new_inputs(mix):
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = P.Batch(mix["sweeps"], use_graph=True)
        for rep in range(3):                      # both staging slots, then a replay of the first
            outs = b.run(mix["images"], boxes=mix["boxes"], stream=s)
            s.synchronize()
            assert all(torch.equal(o, x) for o, x in zip(outs, mix["single"])), rep
        # other boxes and other output buffers through the same graphs
        H, W = mix["single"][0].shape
        nb = [np.array([[0, 0, W // 2, H]], np.int32)] + [None] * (len(mix["sweeps"]) - 1)
        outs2 = b.run(mix["images"], boxes=nb, stream=s)
        s.synchronize()
    ref0 = mix["sweeps"][0].depth(mix["images"][0], boxes=nb[0])
    torch.cuda.synchronize()
    assert torch.equal(outs2[0], ref0)
    assert (outs2[0][:, : W // 2] == 0).all()
    for i in range(1, len(outs2)):
        ref = mix["sweeps"][i].depth(mix["images"][i])
        torch.cuda.synchronize()
        assert torch.equal(outs2[i], ref), i
    assert b.status() == P.PS_OK


def test_bounded_wait_reports_timeout_and_context_stays_usable(mix):
    # failure drill: every merge waits for a tile that never comes; the first
    # wait gives up after 100 ms, the rest of the batch is skipped
    sw = mix["sweeps"][:3]
    b = P.Batch(sw, wait_limit_ms=100, drill_unmet_wait=True)
    b.run(mix["images"][:3], boxes=mix["boxes"][:3])
    assert b.sync_status() == P.PS_ERR_TIMEOUT      # through the handle-generic call
    assert b.status() == P.PS_ERR_TIMEOUT
    with pytest.raises(P.PsError) as e:
        b.timing()
    assert e.value.status == P.PS_ERR_TIMEOUT
    b.close()
    # the context is fine: a normal batch on the same handles still matches
    b2 = P.Batch(sw)
    outs = b2.run(mix["images"][:3], boxes=mix["boxes"][:3])
    torch.cuda.synchronize()
    assert b2.status() == P.PS_OK
    assert all(torch.equal(o, x) for o, x in zip(outs, mix["single"][:3]))


def test_autotune_picks_a_candidate(mix):
    cands = [P.batch_opts(tile_h=t, kp=k, plane_chunk=c) for t in (16, 24) for k in (1, 2) for c in (16, 64)]
    best, ms = P.batch_autotune(mix["sweeps"], mix["images"], cands, boxes=mix["boxes"], reps=2)
    assert 0 <= best < len(cands)
    assert all(m > 0 for m in ms) and ms[best] == min(ms)


def test_rejects_bad_runs(mix):
    b = P.Batch(mix["sweeps"][:2])
    with pytest.raises(ValueError):
        b.run(mix["images"][:1])
    with pytest.raises(P.PsError) as e:
        b.run(mix["images"][:2], boxes=[np.zeros((300, 4), np.int32), None])
    assert e.value.status == P.PS_ERR_ARG
    with pytest.raises(P.PsError) as e:
        P.Batch(mix["sweeps"][:2], use_graph=True).run(mix["images"][:2], stream=torch.cuda.default_stream())
    assert e.value.status == P.PS_ERR_ARG


def test_same_results_with_duplicate_rig_shapes():
    # two handles of one rig in one batch: separate buffers, same maps
    wl = scenes.tiny(2)
    imgs, _ = scenes.FrameSource(wl, device="cuda").frame(0)
    dev = [torch.from_numpy(np.ascontiguousarray(i.numpy())).cuda() for i in imgs]
    a, c = P.Sweep(wl.rig, wl.levels), P.Sweep(wl.rig, wl.levels)
    ref = a.depth(dev).clone()
    outs = P.Batch([a, c]).run([dev, dev])
    torch.cuda.synchronize()
    assert torch.equal(outs[0], ref) and torch.equal(outs[1], ref)


@pytest.fixture(scope="module")
def oracle_mix():
    """Five uneven sweeps for the oracle comparison: drawn sizes, plane
    counts and 1-3 matching cameras, plus one with 4 matching cameras."""
    wls = scenes.batch_mix(5, n=12, sizes=((256, 200), (320, 256), (640, 512)), planes=(32, 64, 128))
    four = next(w for w in scenes.batch_mix(11, n=40, sizes=((320, 256),), planes=(64,), max_cams=4)
                if len(w.rig.cams) == 4)
    wls = wls[:4] + [four]
    sweeps, images, host = [], [], []
    for wl in wls:
        imgs, _ = scenes.FrameSource(wl, device="cuda").frame(0)
        host.append([np.ascontiguousarray(i.numpy()) for i in imgs])
        images.append([torch.from_numpy(h).cuda() for h in host[-1]])
        sweeps.append(P.Sweep(wl.rig, wl.levels))
    return dict(wls=wls, sweeps=sweeps, images=images, host=host)


@pytest.mark.parametrize("tile_h,kp", [(24, 2), (24, 1), (16, 2), (16, 1)])
def test_batch_level_maps_against_the_oracle(oracle_mix, tile_h, kp):
    # every tile shape and pass width of the batched launch, each sweep's
    # level maps against the FP64 oracle at 2,500 sampled pixels, at the
    # spec thresholds
    import os

    import oracle
    from tests.parity import assert_sweep_parity
    oracle.set_threads(os.cpu_count() or 1)
    m = oracle_mix
    b = P.Batch(m["sweeps"], tile_h=tile_h, kp=kp, plane_chunk=32)
    b.run(m["images"], boxes=[w.boxes[0] for w in m["wls"]])
    torch.cuda.synchronize()
    assert b.sync_status() == P.PS_OK
    cams = set()
    for i, (wl, sw) in enumerate(zip(m["wls"], m["sweeps"])):
        g = {k: v.cpu().numpy() for k, v in sw.level_outputs()[0].items()}
        lv = wl.levels[0]
        H, W = g["kstar"].shape
        rho = lv.window // 2
        rng = np.random.default_rng(100 + i)
        flat = rng.choice((H - 2 * rho) * (W - 2 * rho), 2500, replace=False)
        pix = np.stack([rho + flat % (W - 2 * rho), rho + flat // (W - 2 * rho)], axis=1).astype(np.int32)
        o = oracle.sweep_level(wl.rig, lv, m["host"][i], pix=pix)
        s = assert_sweep_parity(o, {k: v[pix[:, 1], pix[:, 0]] for k, v in g.items()}, min_gated=300,
                                src=(wl.rig, lv, m["host"][i], pix))
        print(f"batch th={tile_h} kp={kp} sweep {i} ({W}x{H}, {lv.n_planes} planes, {len(wl.rig.cams)} cams)", s)
        cams.add(len(wl.rig.cams))
    assert 4 in cams and len(cams) >= 2
