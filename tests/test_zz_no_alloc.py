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

import paper_2309_15861_gb300 as G
from paper_2309_15861_gb300 import inputs as I
from tests import _parity

pytestmark = pytest.mark.gpu


def _sorted(h):
    return h[np.lexsort((h["k"], h["seg"], h["tel"]))]


def test_noalloc_matches_clight_trace_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
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
        # more groups than the static array holds: refused before any launch
        code, _, _ = ctx.trace_noalloc(segs, n, 200, hits, cap, raise_on_error=False)
        assert code == G.ERR_LIMIT
    finally:
        ctx.close()
