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


def test_server_refuses_request_larger_than_a_lane():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15917_gb300 as roix
    srv = roix.RoixServer(0, hbm_budget=64 << 20, lanes=2, max_batch=8)
    # 32 MiB input: its pixel section alone fills a 32 MiB lane
    x = torch.zeros((128, 256, 256), dtype=torch.float32, device="cuda")
    out = torch.empty(x.numel() * 4 + 65536, dtype=torch.uint8, device="cuda")
    assert srv.submit(1, x, out, eb=1e-3) == 2  # ROIX_ENOMEM: never fits 32 MiB
    srv.close()
