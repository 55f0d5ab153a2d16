"""The autotuner of the batched forward path: it picks a setting from its
candidate set, the context keeps it, and the tuned path still matches the
oracle run at the chosen bunch size."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import paper_2309_15861_gb300 as G
from paper_2309_15861_gb300 import inputs as I
from tests import _parity

pytestmark = pytest.mark.gpu


def test_autotune_batch_then_parity_at_chosen_bunch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = I.batch_showers(n_showers=8, seed=31, scale=2e-3)
    ctx = G.Context(0)
    try:
        ctx.setup(w)
        segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).cuda()
        cap = 1 << 20
        hits = torch.empty(cap * 48, dtype=torch.uint8, device="cuda")
        n = len(w.segments)
        # a sample of a third of the steps, in blocks spread over every shower
        t = ctx.autotune(segs, n, n // 3, w.n_showers, hits, cap, bunch_max=5.0, reps=5)
        assert (t["block"], t["ctas_per_sm"]) in {(256, 0), (256, 4), (256, 3), (128, 8), (128, 6), (64, 16)}
        assert t["cell_width"] in (1.0, 1.5) and t["work_chunk"] in (1, 2, 4)
        assert t["bunch"] in (1.0, 2.0, 5.0)
        # defaults, bunch 1 and 2, five shapes, two chunks, one cell width
        assert t["n_tried"] == 1 + 2 + 5 + 2 + 1
        assert 0 < t["n_sample"] <= n // 3 + 64 * 32
        # the defaults compete: the choice is never slower by the tuner's own timing
        assert 0 < t["best_ms"] <= t["default_ms"]
        # the context traces with the chosen settings; the oracle runs at the chosen bunch size
        par = dataclasses.replace(w.params, bunch=t["bunch"])
        tuned = I.Workload(w.name, w.segments, w.atmosphere, w.telescopes, par, n_showers=w.n_showers)
        gh, gc, gs, gst = G.run_workload(ctx, tuned)
        rh, rc, rs, rst = O.trace(w.segments, w.atmosphere, w.telescopes, par, n_showers=w.n_showers)
        assert gst["rays"] == rst["rays"]
        nbc, nbf = O.bunch_counts(w.segments, w.atmosphere, par)

        def dp(h):
            return O.eval_rays(w.segments, h["seg"], h["k"], h["tel"], nbc, nbf, w.atmosphere, w.telescopes,
                               par)[:, 4]
        _parity.compare(gh, rh, w.telescopes, ref_dperp_of=dp,
                        w_tol=_parity.weight_tolerance(w.segments, rh, w.atmosphere, par))
        shower = w.segments["shower"]
        _parity.compare_counts(gc, rc, gh, rh, len(w.telescopes), lambda s: shower[s])
    finally:
        ctx.close()


def test_autotune_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = I.workload_shower_1tev(n=1000, seed=3)
    ctx = G.Context(0)
    try:
        ctx.setup(w)
        segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).cuda()
        hits = torch.empty(1024 * 48, dtype=torch.uint8, device="cuda")
        for kw in ({"bunch_max": 0.0}, {"bunch_max": 5.0, "reps": 0}):
            with pytest.raises(G.ClightError):
                ctx.autotune(segs, 1000, 1000, 1, hits, 1024, **kw)
        with pytest.raises(G.ClightError):
            ctx.autotune(segs, 1000, 0, 1, hits, 1024, bunch_max=5.0)
        with pytest.raises(G.ClightError):
            ctx.autotune(segs, 0, 100, 1, hits, 1024, bunch_max=5.0)
    finally:
        ctx.close()
