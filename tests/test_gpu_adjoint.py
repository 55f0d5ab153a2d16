"""The adjoint against central finite differences of the FP64 oracle.

theta = (c_1..c_5, K, L0).  Loss: sum over the hits of gx x_rel + gy y_rel +
gt t plus sum over telescopes of gY Y, with seeded upstream gradients; Y is
the soft-edged (sigma = 0.5 m, cut 20 m) absorption-weighted yield.  Bunch
counts and random numbers are held at their nominal values on both sides.
The oracle's loss is evaluated at theta (1 +- 1e-4) per component.
Agreement: 1e-4 relative, component by component (a component that is
exactly zero in the oracle, a layer no ray reaches, must be zero on the GPU
too).  Hits of steps within kappa = (delta + eps) / (beta n - 1) = 1e3 of
the Cherenkov threshold get no upstream gradient in the central-difference
check (their cone angle, ~ sqrt(beta n - 1), makes their arrival points
non-smooth on the FD scale); they stay in a second comparison with the
oracle's dual-number gradient.  The GPU carries the tangents in binary32 and sums them over every hit,
whose upstream gradients have random signs, so its relative error is of the
order of 1e-5; the central difference's own error is about 1e-8.
"""
import numpy as np
import pytest

import oracle as O
import paper_2309_15861_gb300 as G
from paper_2309_15861_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _oracle_loss(w, atm, hits, gx, gy, gt, gY, nbc, nbf, s=0.5, W=20.0):
    ev = O.eval_rays(w.segments, hits["seg"], hits["k"], hits["tel"], nbc, nbf, atm, w.telescopes, w.params)
    Y = O.soft_yield(w.segments, nbc, nbf, atm, w.telescopes, w.params, n_showers=w.n_showers, s=s, W=W)
    return float(np.sum(gx * ev[:, 0]) + np.sum(gy * ev[:, 1]) + np.sum(gt * ev[:, 2]) + np.sum(gY * Y.ravel()))


def _kappa_of_hits(w, hits):
    """(delta + eps) / (beta n - 1) of each hit's step (0 for fluorescence hits)."""
    kap = np.zeros(len(hits))
    cache = {}
    for i, h in enumerate(hits):
        s = int(h["seg"])
        if s not in cache:
            y = O.yield_of(w.segments[s], w.atmosphere, w.params)
            g1 = 1.0 / y["cos_tc"] - 1.0 if y["n_c"] > 0 else 0.0
            cache[s] = (y["n_c"], (y["delta"] + float(w.segments[s]["eps"])) / g1 if g1 > 0 else 0.0)
        nc, k = cache[s]
        kap[i] = k if h["k"] < nc else 0.0
    return kap


def _check(n_segs, seed, rel=1e-4, zenith_deg=0.0, h=1e-4):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_15861_gb300.autograd import atmosphere_at
    if zenith_deg:
        atm = I.atmosphere_layered()
        w = I.workload_shower_1tev(n=n_segs, seed=seed, zenith_deg=zenith_deg,
                                   telescopes=I.telescope_grid(21, 21, 20.0, z=atm.h_obs),
                                   workers=I.default_workers())
    else:
        w = I.workload_shower_1tev(n=n_segs, seed=seed, workers=I.default_workers())
    ctx = G.Context(0)
    try:
        ctx.setup(w)
        hits, counts, sums, st = G.run_workload(ctx, w)
        rng = np.random.default_rng(seed)
        gx = rng.normal(size=len(hits)).astype(np.float32)
        gy = rng.normal(size=len(hits)).astype(np.float32)
        gt = rng.normal(size=len(hits)).astype(np.float32)
        gY = rng.normal(size=len(w.telescopes))
        # A step within kappa ~ 1e3 of the Cherenkov threshold has a cone
        # angle ~ sqrt(beta n - 1): the FD step (1e-4 of delta) moves beta n - 1
        # by more than 5% of itself, so its arrival points are not smooth on
        # the FD scale.  Such hits get no upstream gradient in the FD check.
        far = _kappa_of_hits(w, hits) < 1e3
        dev = "cuda"
        d_segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).to(dev)
        d_hits = torch.from_numpy(hits.view(np.uint8).reshape(-1).copy()).to(dev)
        tg = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        nbc, nbf = O.bunch_counts(w.segments, w.atmosphere, w.params)
        gsoft = O.grad_soft(w.segments, nbc, nbf, w.atmosphere, w.telescopes, w.params, gY, s=0.5, W=20.0)
        if not far.all():
            # every hit, near-threshold ones included, against the dual numbers
            ga = ctx.trace_adjoint(d_segs, len(w.segments), 1, d_hits, len(hits), tg(gx), tg(gy), tg(gt), tg(gY))[:7]
            gda = O.grad_rays(w.segments, hits["seg"], hits["k"], hits["tel"], nbc, nbf, w.atmosphere,
                              w.telescopes, w.params, gx, gy, gt) + gsoft
            erra = np.where(gda == 0.0, np.abs(ga), np.abs(ga - gda) / np.where(gda == 0.0, 1.0, np.abs(gda)))
            print("all hits: adjoint", ga, "\ndual ", gda, "\nrel  ", erra, "\nnear-threshold hits", int((~far).sum()))
            assert np.all(erra < rel), (ga, gda, erra)
        gx, gy, gt = gx * far, gy * far, gt * far
        grad = ctx.trace_adjoint(d_segs, len(w.segments), 1, d_hits, len(hits), tg(gx), tg(gy), tg(gt), tg(gY))[:7]
        # central differences of the FP64 oracle at h relative
        theta = np.array(list(w.atmosphere.c) + [w.atmosphere.K, w.atmosphere.L0])
        fd = np.zeros(7)
        for p in range(7):
            hp = h * theta[p]
            tp, tm = theta.copy(), theta.copy()
            tp[p] += hp
            tm[p] -= hp
            lp = _oracle_loss(w, atmosphere_at(w.atmosphere, tp), hits, gx, gy, gt, gY, nbc, nbf)
            lm = _oracle_loss(w, atmosphere_at(w.atmosphere, tm), hits, gx, gy, gt, gY, nbc, nbf)
            fd[p] = (lp - lm) / (2 * hp)
        zero = fd == 0.0
        assert np.all(grad[zero] == 0.0), (grad, fd)
        err = np.where(zero, 0.0, np.abs(grad - fd) / np.where(zero, 1.0, np.abs(fd)))
        print("adjoint", grad, "\nfd     ", fd, "\nrel    ", err)
        assert np.all(err < rel), (grad, fd, err)
        # and the oracle's FP64 gradient by dual numbers
        gd = (O.grad_rays(w.segments, hits["seg"], hits["k"], hits["tel"], nbc, nbf, w.atmosphere, w.telescopes,
                          w.params, gx, gy, gt) + gsoft)
        errd = np.where(gd == 0.0, np.abs(grad), np.abs(grad - gd) / np.where(gd == 0.0, 1.0, np.abs(gd)))
        print("dual   ", gd, "\nrel    ", errd)
        assert np.all(errd < rel), (grad, gd, errd)
        return grad, fd
    finally:
        ctx.close()


def test_adjoint_matches_oracle_finite_differences_small():
    _check(20_000, seed=41)


def test_adjoint_matches_oracle_finite_differences_large():
    """3x10^5 steps of the 1 TeV vertical shower."""
    _check(300_000, seed=1)


def test_adjoint_matches_oracle_at_the_differentiation_size():
    """10^6 steps of the 1 TeV vertical generator: the size the
    differentiation workload is stated at.  Among 10^6 steps some sit so
    close to the Cherenkov threshold that their cone angle, ~ sqrt(beta n - 1),
    moves by a large fraction under a 1e-4 change of the refractivity: the
    soft yield is then not smooth on that scale (the oracle's own h = 1e-4
    central differences miss its exact dual-number derivative by 2-5e-4, at
    h = 1e-6 by 1e-6 to 1e-5), so the differences here take h = 1e-6."""
    _check(1_000_000, seed=2, h=1e-6)


def test_adjoint_matches_oracle_at_60_degrees():
    """An inclined shower (60 deg zenith, 21 x 21 telescopes at 20 m): long
    slanted paths through every layer, against the oracle's central
    differences and its dual-number gradient."""
    _check(20_000, seed=3, zenith_deg=60.0)


def test_adjoint_is_bitwise_reproducible():
    """Two adjoint calls on the same inputs give the same gradient and the
    same soft yields to the last bit (the candidate rays are sorted before
    the tangent kernels; the yield is summed in fixed point)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = I.workload_shower_1tev(n=200_000, seed=53, workers=I.default_workers())
    ctx = G.Context(0)
    try:
        ctx.setup(w)
        with pytest.raises(G.ClightError):                 # no adjoint call yet
            ctx.last_adjoint()
        hits, counts, sums, st = G.run_workload(ctx, w)
        dev = "cuda"
        d_segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).to(dev)
        d_hits = torch.from_numpy(hits.view(np.uint8).reshape(-1).copy()).to(dev)
        rng = np.random.default_rng(53)
        tg = lambda a: torch.from_numpy(a).to(dev)
        gx = tg(rng.normal(size=len(hits)).astype(np.float32))
        gY = tg(rng.normal(size=len(w.telescopes)))
        outs = []
        for _ in range(3):
            Y = torch.full((len(w.telescopes),), -1.0, dtype=torch.float64, device=dev)
            g = ctx.trace_adjoint(d_segs, len(w.segments), 1, d_hits, len(hits), gx=gx, gY=gY, d_yield=Y)[:7]
            outs.append((g.copy(), Y.cpu().numpy().copy()))
        for g, Y in outs[1:]:
            assert np.array_equal(g.view(np.int64), outs[0][0].view(np.int64))
            assert np.array_equal(Y.view(np.int64), outs[0][1].view(np.int64))
        assert np.all(np.isfinite(outs[0][0])) and outs[0][1].sum() > 0
        # the fixed-point yield against the oracle's soft yield (binary32 weights)
        nbc, nbf = O.bunch_counts(w.segments, w.atmosphere, w.params)
        Yr = O.soft_yield(w.segments, nbc, nbf, w.atmosphere, w.telescopes, w.params, s=0.5, W=20.0).ravel()
        np.testing.assert_allclose(outs[0][1], Yr, rtol=1e-4, atol=1e-3)
        # the last call's counts and phase times
        info = ctx.last_adjoint()
        assert info["hits"] == len(hits) and info["candidates"] >= len(hits) // 2 > 0
        assert min(info["candidate_ms"], info["sort_ms"], info["tangent_ms"]) >= 0.0 and info["tangent_ms"] > 0.0
    finally:
        ctx.close()


def test_autograd_function_backward_equals_adjoint():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_15861_gb300.autograd import AtmosphereResponse, Engine, theta_of
    w = I.workload_shower_1tev(n=20_000, seed=43)
    ctx = G.Context(0)
    try:
        ctx.setup(w)
        d_segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).cuda()
        eng = Engine(ctx=ctx, workload=w, d_segs=d_segs)
        theta = theta_of(w.atmosphere).requires_grad_(True)
        x, y, t, Y = AtmosphereResponse.apply(theta, eng)
        assert x.numel() > 100 and Y.numel() == len(w.telescopes)
        gen = torch.Generator().manual_seed(5)
        ax = torch.randn(x.shape, generator=gen).cuda()
        aY = torch.randn(Y.shape, generator=gen, dtype=torch.float64).cuda()
        loss = (ax * x).sum().double() + (aY * Y).sum()
        loss.backward()
        direct = ctx.trace_adjoint(d_segs, len(w.segments), 1, eng.hits, x.numel(), gx=ax, gY=aY)[:7]
        np.testing.assert_allclose(theta.grad.numpy(), direct, rtol=1e-12)
        assert np.all(np.isfinite(direct)) and np.any(direct != 0)
    finally:
        ctx.close()


def test_adjoint_refuses_what_its_tangents_do_not_cover():
    """The tangents are those of the exact propagator without dispersion:
    with the straight-line propagator or dispersion on, the adjoint returns
    CLIGHT_ERR_ARG instead of a gradient of another model."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = I.workload_shower_1tev(n=2_000, seed=47)
    ctx = G.Context(0)
    try:
        d_segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).cuda()
        d_hits = torch.zeros(48, dtype=torch.uint8, device="cuda")
        gY = torch.ones(len(w.telescopes), dtype=torch.float64, device="cuda")
        ctx.setup(w, propagator=G.PROP_STRAIGHT)
        with pytest.raises(G.ClightError) as e:
            ctx.trace_adjoint(d_segs, len(w.segments), 1, d_hits, 0, gY=gY)
        assert e.value.code == G.ERR_ARG
        w.atmosphere.disp_B = 20000.0
        ctx.setup(w)
        with pytest.raises(G.ClightError) as e:
            ctx.trace_adjoint(d_segs, len(w.segments), 1, d_hits, 0, gY=gY)
        assert e.value.code == G.ERR_ARG
        w.atmosphere.disp_B = 0.0
        ctx.setup(w)
        g = ctx.trace_adjoint(d_segs, len(w.segments), 1, d_hits, 0, gY=gY)
        assert np.all(np.isfinite(g))
    finally:
        ctx.close()
