"""Serving loop: requests of mixed sizes and settings arrive over time from
another thread; every container must equal the one compressed alone (and
the oracle's), whatever batch it was admitted in."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest
import torch

import oracle
import phantom

pytestmark = pytest.mark.gpu


def test_server_mix_equals_alone():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15917_gb300 as roix
    proj_cfg = dict(eb=4, cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100)
    vol_cfg = dict(eb=1e-3, eb_mode="rel", threshold=0.1, dilate=1)
    reqs = []
    rng = np.random.default_rng(3)
    for i in range(40):
        if i % 4 == 3:
            x = phantom.ellipsoids(shape=tuple(int(v) for v in rng.integers(8, 40, 3)),
                                   seed=100 + i)
            cfg = vol_cfg
        else:
            x = phantom.projection(int(rng.integers(40, 300)), i, seed=11)
            cfg = proj_cfg
        xd = x.cuda()
        out = torch.empty(x.numel() * x.element_size() + 65536, dtype=torch.uint8, device="cuda")
        reqs.append((i, x.numpy(), xd, out, cfg))
    torch.cuda.synchronize()
    srv = roix.RoixServer(0, hbm_budget=2 << 30, lanes=3, max_batch=16)

    def client():
        # a burst (queues up behind the busy lanes, so batches form), then
        # arrivals spread out in time
        for k, (tag, _, xd, out, cfg) in enumerate(reqs):
            assert srv.submit(tag, xd, out, **cfg) == 0
            if k >= 24:
                time.sleep(float(rng.exponential(0.002)))

    th = threading.Thread(target=client)
    th.start()
    th.join()
    assert srv.drain(60.0) == 0
    done = {}
    while True:
        got = srv.poll()
        if not got:
            break
        for c in got:
            done[c["tag"]] = c
    stats = srv.stats()
    srv.close()
    assert len(done) == len(reqs) and stats["completed"] == len(reqs)
    assert stats["batches"] < len(reqs)  # requests were batched together
    alone = roix.Roix(0)
    for tag, x, xd, out, cfg in reqs:
        c = done[tag]
        assert c["status"] == 0 and c["t_submit"] <= c["t_admit"] <= c["t_done"]
        got = out[:c["size"]].cpu().numpy()
        ref = alone.compress_bytes(xd, **cfg).cpu().numpy()
        assert np.array_equal(got, ref)
        if tag % 8 == 0:
            assert np.array_equal(got, oracle.compress(x, **cfg))
    alone.close()


def test_server_refuses_request_larger_than_the_budget():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15917_gb300 as roix
    srv = roix.RoixServer(0, hbm_budget=64 << 20, lanes=2, max_batch=8)
    # 64 MiB input: its pixel section alone fills the 64 MiB arena
    x = torch.zeros((256, 256, 256), dtype=torch.float32, device="cuda")
    out = torch.empty(x.numel() * 4 + 65536, dtype=torch.uint8, device="cuda")
    assert srv.submit(1, x, out, eb=1e-3) == 2  # ROIX_ENOMEM: never fits
    srv.close()


def test_server_large_request_waits_for_memory_then_runs():
    """Two requests that each need most of the arena: the second waits until
    the first has returned its workspace (and the requests behind it wait
    too, in arrival order), then runs; every container equals the one
    compressed alone, and the arena is empty at the end."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15917_gb300 as roix
    cfg = dict(eb=1e-3, eb_mode="rel", threshold=0.1, dilate=1)
    small = [phantom.ellipsoids(shape=(24, 40, 40), seed=50 + i) for i in range(8)]
    bigs = [phantom.ellipsoids(shape=(160, 160, 160), seed=77 + i) for i in range(2)]
    xs = small[:4] + bigs + small[4:]
    alone = roix.Roix(0)
    refs = [alone.compress_bytes(x.cuda(), **cfg).cpu().numpy() for x in xs]
    need_big = alone.workspace_size(bigs[0].shape, torch.float32, bigs[0].numel() * 4 + 65536,
                                    **cfg)
    alone.close()
    budget = int(need_big * 1.3)  # one big request at a time
    srv = roix.RoixServer(0, hbm_budget=budget, lanes=3, max_batch=4)
    outs = []
    for tag, x in enumerate(xs):
        xd = x.cuda()
        out = torch.empty(x.numel() * 4 + 65536, dtype=torch.uint8, device="cuda")
        outs.append((xd, out))
        assert srv.submit(tag, xd, out, **cfg) == 0
    assert srv.drain(60.0) == 0
    got = {}
    while True:
        cs = srv.poll()
        if not cs:
            break
        for c in cs:
            got[c["tag"]] = c
    assert sorted(got) == list(range(len(xs)))
    for tag, ref in enumerate(refs):
        c = got[tag]
        assert c["status"] == 0
        buf = outs[tag][1][:c["size"]].cpu().numpy()
        assert np.array_equal(buf, ref), tag
    # the second big request was admitted only after the first had completed
    assert got[5]["t_admit"] >= got[4]["t_done"]
    stats = srv.stats()
    assert stats["in_use_bytes"] == 0 and stats["budget_bytes"] == budget
    srv.close()
