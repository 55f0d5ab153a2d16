"""The adjoint against central finite differences of the FP64 oracle.

theta = (c_1..c_5, K, L0).  Loss: sum over the hits of gx x_rel + gy y_rel +
gt t plus sum over telescopes of gY Y, with seeded upstream gradients; Y is
the soft-edged (sigma = 0.5 m, cut 20 m) absorption-weighted yield.  Bunch
counts and random numbers are held at their nominal values on both sides.
The oracle's loss is evaluated at theta (1 +- 1e-4) per component.
Agreement: 1e-4 relative, component by component (a component that is
exactly zero in the oracle, a layer no ray reaches, must be zero on the GPU
too).  The GPU carries the tangents in binary32 and sums them over every hit,
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


def _check(n_segs, seed, rel=1e-4):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_15861_gb300.autograd import atmosphere_at
    w = I.workload_shower_1tev(n=n_segs, seed=seed)
    ctx = G.Context(0)
    try:
        ctx.setup(w)
        hits, counts, sums, st = G.run_workload(ctx, w)
        rng = np.random.default_rng(seed)
        gx = rng.normal(size=len(hits)).astype(np.float32)
        gy = rng.normal(size=len(hits)).astype(np.float32)
        gt = rng.normal(size=len(hits)).astype(np.float32)
        gY = rng.normal(size=len(w.telescopes))
        dev = "cuda"
        d_segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).to(dev)
        d_hits = torch.from_numpy(hits.view(np.uint8).reshape(-1).copy()).to(dev)
        tg = lambda a: torch.from_numpy(a).to(dev)
        grad = ctx.trace_adjoint(d_segs, len(w.segments), 1, d_hits, len(hits), tg(gx), tg(gy), tg(gt), tg(gY))[:7]
        # finite differences of the FP64 oracle
        nbc, nbf = O.bunch_counts(w.segments, w.atmosphere, w.params)
        theta = np.array(list(w.atmosphere.c) + [w.atmosphere.K, w.atmosphere.L0])
        fd = np.zeros(7)
        for p in range(7):
            hp = 1e-4 * theta[p]
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
                          w.params, gx, gy, gt)
              + O.grad_soft(w.segments, nbc, nbf, w.atmosphere, w.telescopes, w.params, gY, s=0.5, W=20.0))
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
