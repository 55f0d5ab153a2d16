"""The entry point that allocates nothing (clight_trace_noalloc).

Some callers cannot let a library call cudaMalloc while it runs -- an
embedding framework that owns all device memory through its own pool, or a
process that reserves its memory at start-up.  clight_trace_noalloc serves
them: its scratch is a static array in the library image.  This file is
named to be collected last, so that a run stopping at its first failure has
already run every other test; it passes alone in a fresh process too.
"""
import numpy as np
import pytest

import oracle as O
import paper_2309_15861_gb300 as G
from paper_2309_15861_gb300 import inputs as I
from tests import _parity

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _sorted(h):
    return h[np.lexsort((h["k"], h["seg"], h["tel"]))]


def _dperp_fn(w):
    nbc, nbf = O.bunch_counts(w.segments, w.atmosphere, w.params, w.telescopes)

    def f(h):
        return O.eval_rays(w.segments, h["seg"], h["k"], h["tel"], nbc, nbf, w.atmosphere, w.telescopes,
                           w.params)[:, 4]
    return f


def test_noalloc_matches_clight_trace_on_two_calls_in_a_row():
    torch = _torch()
    w = I.workload_shower_1tev(n=60_000, seed=37)
    ctx = G.Context(0)
    try:
        ctx.setup(w)
        ref_h, ref_c, ref_s, ref_st = G.run_workload(ctx, w)       # the allocating entry point
        assert len(ref_h) > 500
        n = len(w.segments)
        segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).cuda()
        cap = len(ref_h) + 1000
        hits = torch.empty(cap * 48, dtype=torch.uint8, device="cuda")
        counts = torch.full((len(w.telescopes),), -1, dtype=torch.int64, device="cuda")
        for call in range(2):
            hits.fill_(0xFF)                                       # stale bytes must not survive
            code, nh, st = ctx.trace_noalloc(segs, n, 1, hits, cap, counts)
            assert code == G.OK
            assert nh == len(ref_h)
            assert st["rays"] == ref_st["rays"] and st["hits"] == ref_st["hits"]
            got = _sorted(hits[: nh * 48].cpu().numpy().view(G.HIT_DTYPE).copy())
            for f in ("seg", "k", "tel"):
                np.testing.assert_array_equal(got[f], ref_h[f])
            np.testing.assert_allclose(got["x_rel"], ref_h["x_rel"], rtol=0, atol=_parity.TOL_XY)
            np.testing.assert_allclose(got["y_rel"], ref_h["y_rel"], rtol=0, atol=_parity.TOL_XY)
            np.testing.assert_allclose(got["t"], ref_h["t"], rtol=0, atol=_parity.TOL_T)
            np.testing.assert_allclose(got["weight"], ref_h["weight"], rtol=_parity.TOL_W)
            np.testing.assert_allclose(got["lambda"], ref_h["lambda"], rtol=_parity.TOL_LAM)
            np.testing.assert_allclose(got["cx"], ref_h["cx"], atol=_parity.TOL_DIR)
            np.testing.assert_allclose(got["cy"], ref_h["cy"], atol=_parity.TOL_DIR)
            np.testing.assert_array_equal(counts.cpu().numpy(), ref_c.reshape(-1))
        # and against the FP64 oracle, element by element
        rh, rc, rs, rst = O.trace(w.segments, w.atmosphere, w.telescopes, w.params)
        assert st["rays"] == rst["rays"]
        _parity.compare(got, rh, w.telescopes, ref_dperp_of=_dperp_fn(w),
                        w_tol=_parity.weight_tolerance(w.segments, rh, w.atmosphere, w.params))
        _parity.compare_counts(counts.cpu().numpy().reshape(1, -1), rc, got, rh, len(w.telescopes),
                               lambda s: 0)
        # more groups than the static array holds: refused before any launch
        code, _, _ = ctx.trace_noalloc(segs, n, 200, hits, cap, raise_on_error=False)
        assert code == G.ERR_LIMIT
    finally:
        ctx.close()


def test_noalloc_two_showers_and_capacity_overflow():
    """Two showers with fluorescence (group index shower * n_tel + tel): the
    counts match the oracle's and clight_trace's; with the capacity below
    the hit count the call reports the count it needs, writes nothing past
    the capacity, and still returns every group's count."""
    torch = _torch()
    w = I.batch_showers(n_showers=2, seed=83, scale=2e-3)
    ctx = G.Context(0)
    try:
        ctx.setup(w)
        ref_h, ref_c, ref_s, ref_st = G.run_workload(ctx, w)
        assert ref_c[0].sum() > 0 and ref_c[1].sum() > 0
        n = len(w.segments)
        segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).cuda()
        ng = w.n_showers * len(w.telescopes)
        counts = torch.full((ng,), -1, dtype=torch.int64, device="cuda")
        cap = len(ref_h) + 64
        hits = torch.empty(cap * 48, dtype=torch.uint8, device="cuda")
        code, nh, st = ctx.trace_noalloc(segs, n, w.n_showers, hits, cap, counts)
        assert code == G.OK and nh == len(ref_h)
        got = _sorted(hits[: nh * 48].cpu().numpy().view(G.HIT_DTYPE).copy())
        np.testing.assert_array_equal(counts.cpu().numpy(), ref_c.reshape(-1))
        rh, rc, rs, rst = O.trace(w.segments, w.atmosphere, w.telescopes, w.params, n_showers=w.n_showers)
        _parity.compare(got, rh, w.telescopes, ref_dperp_of=_dperp_fn(w),
                        w_tol=_parity.weight_tolerance(w.segments, rh, w.atmosphere, w.params))
        shower = w.segments["shower"]
        _parity.compare_counts(counts.cpu().numpy().reshape(w.n_showers, -1), rc, got, rh, len(w.telescopes),
                               lambda s: shower[s])
        # overflow: a guard region behind the first `small` records stays untouched
        small = nh // 3
        guard = 256
        buf = torch.full(((small + guard) * 48,), 0xAB, dtype=torch.uint8, device="cuda")
        counts.fill_(-1)
        code, nh2, st2 = ctx.trace_noalloc(segs, n, w.n_showers, buf, small, counts, raise_on_error=False)
        assert code == G.ERR_HIT_CAPACITY and nh2 == nh
        tail = buf[small * 48:].cpu().numpy()
        assert np.all(tail == 0xAB)
        np.testing.assert_array_equal(counts.cpu().numpy(), ref_c.reshape(-1))
        # the records that were written are valid hits of the full list
        part = buf[: small * 48].cpu().numpy().view(G.HIT_DTYPE)
        full_keys = set(zip(ref_h["seg"].tolist(), ref_h["k"].tolist(), ref_h["tel"].tolist()))
        assert all(k in full_keys for k in zip(part["seg"].tolist(), part["k"].tolist(), part["tel"].tolist()))
        # buffers smaller than the call would write are refused before the call
        with pytest.raises(ValueError):
            ctx.trace_noalloc(segs, n, w.n_showers, buf, small + guard + 1, counts)
    finally:
        ctx.close()


def test_noalloc_queue_overflow_traces_the_chunk_in_place():
    """The default feature set takes the two passes with a static queue of
    2^22 rays per chunk of steps.  A dense array (6 m spheres 10 m apart)
    queues more rays than that: the chunk is traced again by the in-place
    kernel from the counters saved before it (so its statistics show no
    queued ray), and hits, counts and ray totals equal clight_trace's, whose
    queue grows instead."""
    torch = _torch()
    w = I.workload_shower_1tev(n=2_000_000, seed=71, workers=I.default_workers())
    w.telescopes = I.telescope_grid(81, 81, 10.0, z=w.atmosphere.h_obs)
    ctx = G.Context(0)
    try:
        ctx.setup(w)
        ref_h, ref_c, ref_s, ref_st = G.run_workload(ctx, w)
        assert ref_st["deferred"] > (1 << 22)
        n = len(w.segments)
        segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).cuda()
        cap = len(ref_h) + 1000
        hits = torch.empty(cap * 48, dtype=torch.uint8, device="cuda")
        counts = torch.full((len(w.telescopes),), -1, dtype=torch.int64, device="cuda")
        code, nh, st = ctx.trace_noalloc(segs, n, 1, hits, cap, counts)
        assert code == G.OK and nh == len(ref_h)
        assert st["rays"] == ref_st["rays"] and st["hits"] == ref_st["hits"]
        assert st["deferred"] == 0 and st["step_skipped"] == 0      # the in-place kernel traced the chunk
        got = _sorted(hits[: nh * 48].cpu().numpy().view(G.HIT_DTYPE).copy())
        for f in ("seg", "k", "tel"):
            np.testing.assert_array_equal(got[f], ref_h[f])
        np.testing.assert_allclose(got["weight"], ref_h["weight"], rtol=_parity.TOL_W)
        np.testing.assert_array_equal(counts.cpu().numpy(), ref_c.reshape(-1))
        # a small call right after takes the two passes again
        w2 = I.workload_shower_1tev(n=60_000, seed=37)
        ctx.setup(w2)
        segs2 = torch.from_numpy(w2.segments.view(np.uint8).reshape(-1)).cuda()
        code, nh2, st2 = ctx.trace_noalloc(segs2, len(w2.segments), 1, hits, cap)
        assert code == G.OK and st2["deferred"] > 0
    finally:
        ctx.close()


def test_noalloc_refuses_stream_capture():
    """The call reads its counters back to the host, which a stream capture
    does not allow: it returns an argument error and leaves the caller's
    capture intact."""
    torch = _torch()
    w = I.workload_shower_1tev(n=2_000, seed=89)
    ctx = G.Context(0)
    try:
        ctx.setup(w)
        segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).cuda()
        hits = torch.empty(4096 * 48, dtype=torch.uint8, device="cuda")
        ctx.trace_noalloc(segs, len(w.segments), 1, hits, 4096)      # first call: address lookup
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin()
            try:
                hits[:48].zero_()                                      # the capture holds one node
                code, _, _ = ctx.trace_noalloc(segs, len(w.segments), 1, hits, 4096, stream=s,
                                               raise_on_error=False)
            finally:
                g.capture_end()
        assert code == G.ERR_ARG
        torch.cuda.synchronize()
        code, nh, st = ctx.trace_noalloc(segs, len(w.segments), 1, hits, 4096)
        assert code == G.OK and st["rays"] > 0
    finally:
        ctx.close()
