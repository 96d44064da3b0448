"""Host logic of the multi-GPU split of one frame (plane ranges per rank,
the all-gather of the ranks' records, the merge rule), on CPU ranks over
gloo.  The records each rank contributes are built from the FP64 oracle's
per-plane costs by the record definition, so the merge of the gathered
records must reproduce the oracle's winner-take-all over all planes."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INF = np.inf


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def record_from_costs(C, lo, hi):
    """(7, n) record of planes [lo, hi) from (n, K) costs: best, second best,
    the best plane's neighbour costs inside the range, first and last cost,
    best index (-1 = none; ties keep the lowest plane)."""
    n = C.shape[0]
    rec = np.full((7, n), INF)
    rec[6] = -1
    if hi <= lo:
        return rec
    S = C[:, lo:hi]
    fin = np.isfinite(S)
    k = np.where(fin.any(axis=1), np.argmin(np.where(fin, S, INF), axis=1), -1)
    for i in range(n):
        rec[4, i], rec[5, i] = S[i, 0], S[i, -1]
        if k[i] < 0:
            continue
        kk = lo + k[i]
        rec[0, i] = C[i, kk]
        others = np.delete(S[i], k[i])
        rec[1, i] = others.min() if others.size else INF
        rec[2, i] = C[i, kk - 1] if kk - 1 >= lo else INF
        rec[3, i] = C[i, kk + 1] if kk + 1 < hi else INF
        rec[6, i] = kk
    return rec


def merge_records(recs, los, K):
    """The merge rule of psweep_merge_records (parts in plane order)."""
    n = recs[0].shape[1]
    out = dict(c1=np.full(n, INF), c2=np.full(n, INF), k=np.full(n, -1), cm=np.full(n, INF), cp=np.full(n, INF))
    his = list(los[1:]) + [K]
    live = [p for p in range(len(recs)) if his[p] > los[p]]
    for i in range(n):
        wc, b1 = -1, INF
        for p in live:
            if recs[p][0, i] < b1:
                b1, wc = recs[p][0, i], p
        if wc < 0:
            continue
        b2 = min([recs[wc][1, i]] + [recs[p][0, i] for p in live if p != wc])
        k = int(recs[wc][6, i])
        j = live.index(wc)
        cm = recs[wc][2, i] if k > los[wc] else (recs[live[j - 1]][5, i] if j > 0 else INF)
        cp = recs[wc][3, i] if k < his[wc] - 1 else (recs[live[j + 1]][4, i] if j + 1 < len(live) else INF)
        out["c1"][i], out["c2"][i], out["k"][i], out["cm"][i], out["cp"][i] = b1, b2, k, cm, cp
    return out


def _tiny_costs():
    sys.path.insert(0, ROOT)
    import oracle
    import scenes
    wl = scenes.tiny(0)
    imgs, _ = scenes.FrameSource(wl).frame(0)
    imgs = [i.numpy() for i in imgs]
    rng = np.random.default_rng(4)
    pix = np.stack([rng.integers(2, 158, 600), rng.integers(2, 126, 600)], axis=1).astype(np.int32)
    o = oracle.sweep_level(wl.rig, wl.levels[0], imgs, pix=pix, want_costs=True)
    return o, wl.levels[0].n_planes


def test_split_planes_is_a_consecutive_cover():
    from paper_1809_06132_gb300.shard import split_planes
    for K in ([96, 128], [32], [5, 1], [0, 7]):
        for world in (1, 2, 3, 4, 8):
            r = split_planes(K, world)
            assert len(r) == world
            for l, k in enumerate(K):
                assert r[0][0][l] == 0 and r[-1][1][l] == k
                for a, b in zip(r, r[1:]):
                    assert a[1][l] == b[0][l]
                sizes = [hi[l] - lo[l] for lo, hi in r]
                assert max(sizes) - min(sizes) <= 1


def test_merge_rule_reproduces_the_whole_range_on_oracle_costs():
    o, K = _tiny_costs()
    C = o["costs"]
    full = record_from_costs(C, 0, K)
    for los in ([0], [0, 16], [0, 5, 5, 31], [0, 1, 2, 30]):
        recs = [record_from_costs(C, lo, hi) for lo, hi in zip(los, los[1:] + [K])]
        m = merge_records(recs, los, K)
        assert np.array_equal(m["k"], full[6].astype(int)), los
        assert np.array_equal(m["k"], o["kstar"])
        assert np.array_equal(m["c1"], full[0]) and np.array_equal(m["c2"], full[1])
        assert np.array_equal(m["cm"], full[2]) and np.array_equal(m["cp"], full[3])


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1809_06132_gb300.shard import exchange_records, split_planes
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        o, K = _tiny_costs()
        ranges = split_planes([K], world)
        lo, hi = ranges[rank]
        mine = torch.from_numpy(record_from_costs(o["costs"], lo[0], hi[0]).astype(np.float32))
        extra = torch.full((3, 5), float(rank))           # a second "level" of another shape
        got = exchange_records([mine, extra])
        los = [r[0][0] for r in ranges]
        recs = [g[0].numpy().astype(np.float64) for g in got]
        m = merge_records(recs, los, K)
        out.put((rank, [int(g[1][0, 0]) for g in got], np.array_equal(m["k"], o["kstar"]),
                 bool(np.array_equal(got[rank][0].numpy(), mine.numpy()))))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_records_exchange_on_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=150) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, order, same_k, own in res:
        assert order == [0, 1]          # gathered in rank order, every level split back out
        assert same_k and own
