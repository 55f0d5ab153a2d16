"""Sharding over ranks: the plan, and a world_size-2 gloo run whose merged
output equals the single-process trace (CPU; the oracle traces each shard)."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2309_15861_gb300 import inputs as I
from paper_2309_15861_gb300 import shard


def test_plan_covers_and_balances():
    for n, world in ((0, 1), (1, 2), (10, 3), (1_000_003, 8)):
        p = shard.plan(n, world)
        assert len(p) == world and p[0][0] == 0 and p[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(p, p[1:]))
        sizes = [hi - lo for lo, hi in p]
        assert max(sizes) - min(sizes) <= 1


def test_plan_cuts_on_shower_boundaries():
    rng = np.random.default_rng(3)
    shower = np.repeat(np.arange(40), rng.integers(1, 500, size=40))
    n = len(shower)
    for world in (1, 2, 3, 7, 40, 64):
        p = shard.plan(n, world, shower)
        assert p[0][0] == 0 and p[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(p, p[1:]))
        for lo, hi in p:
            if 0 < lo < n:
                assert shower[lo] != shower[lo - 1]
    with pytest.raises(ValueError):
        shard.plan(3, 2, np.array([1, 0, 2]))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, by_shower, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = I.batch_showers(4, seed=7, scale=2e-4) if by_shower else I.workload_shower_1tev(n=3000, seed=5)
        n_tel = len(w.telescopes)
        lo, hi = shard.plan(len(w.segments), world, w.segments["shower"] if by_shower else None)[rank]
        h, c, s, st = O.trace(w.segments[lo:hi], w.atmosphere, w.telescopes, w.params, n_showers=w.n_showers,
                              threads=2, seg_base=lo)
        shower_of = w.segments["shower"]
        mh, mc, ms = shard.merge(h, c, s, lambda x: shower_of[x["seg"]].astype(np.int64) * n_tel + x["tel"])
        if rank == 0:
            np.savez(out_path, hits=mh, counts=mc, sums=ms)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("by_shower", [False, True])
def test_gloo_two_ranks_merge_equals_single_process(by_shower):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "merged.npz")
        mp.spawn(_rank_main, args=(2, _free_port(), by_shower, out), nprocs=2, join=True)
        r = np.load(out)
        w = I.batch_showers(4, seed=7, scale=2e-4) if by_shower else I.workload_shower_1tev(n=3000, seed=5)
        h, c, s, st = O.trace(w.segments, w.atmosphere, w.telescopes, w.params, n_showers=w.n_showers, threads=2)
        assert len(h) > 50
        assert np.array_equal(r["hits"], h)
        assert np.array_equal(r["counts"], c)
        if by_shower:
            assert np.array_equal(r["sums"], s)
        else:
            np.testing.assert_allclose(r["sums"], s, rtol=1e-12, atol=0)
