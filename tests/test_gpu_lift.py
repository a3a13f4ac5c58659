"""Lifting of orders two and three (Def. 1 with the Chapman-Enskog terms
h2, h3 of Sec. 2.1) on the GPU: mm_lift against the oracle's lifting, and
parareal with relifting of order L through parareal_run and the batch
engine against the oracle's Algorithm 1 with the same order."""
import numpy as np
import pytest

import oracle as O
from paper_2511_13386_gb300 import mm, workloads as W
from tests.gpu_helpers import FP32_TOL, FP64_TOL, device, gdtype, oparams, params, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


U = 2.0 ** -53


def lift_tol(L, eps, nx):
    """FP64 tolerance of the lifting of order L, relative to max |g|.  The
    CUDA path applies Table 1 with integer weights, the oracle with the
    printed fractions: both are correct and round differently.  The order-l
    term carries l - 1 more x-derivatives of J than the first-order term
    (each stencil amplifies rounding by sum |c_k| / dx <= 2 nx) and a factor
    eps^(l-1) relative to it, so the difference is bounded by
    sum_l eps^(l-1) (2 nx)^(l-1) u, with a margin of 8."""
    return FP64_TOL + 8 * U * sum((eps * 2 * nx) ** (l - 1) for l in range(2, L + 1))


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32G])
@pytest.mark.parametrize("L", [1, 2, 3])
@pytest.mark.parametrize("nx,nv", [(256, 32), (777, 20), (4096, 64)])
def test_lift_order_parity(prec, L, nx, nv):
    dev = device()
    w = W.batched(nx=nx, nv=nv, eps=0.05)
    rho, _ = w.with_batch(2)
    p = params(nx, nv, 0.05, prec, rho_bar=1.0, lift_order=L)
    ctx = mm.mm_create(p)
    r = torch.tensor(rho, device=dev)
    g = torch.empty((2, nx, nv), device=dev, dtype=gdtype(prec))
    mm.mm_lift(ctx, 2, r, g)
    ctx.close()
    _, wts, _, _ = O.velocity_grid(oparams(p))
    for b in range(2):
        ref = O.lift(oparams(p), rho[b], L)
        got = g[b].double().cpu().numpy()
        tol = lift_tol(L, 0.05, nx) if prec == mm.MM_FP64 else 1e-6
        assert rel(got, ref) <= tol, (rel(got, ref), tol)
        if prec == mm.MM_FP64:
            assert np.abs(got @ wts).max() <= 1e-15 * np.abs(got).max() * nv


def test_lift_order_rejects_out_of_range():
    device()
    for L in (0, 4):
        with pytest.raises(mm.MMError):
            mm.mm_create(params(64, 32, 1.0, mm.MM_FP64, lift_order=L))


def _parareal_case():
    w = W.batched(nx=256, nv=32, eps=0.01, n_slices=5)
    p = params(w.nx, w.nv, w.eps, mm.MM_FP64, rho_bar=1.0)
    ctx = mm.mm_create(p)
    w.t_end = 5 * 30 * mm.mm_query(ctx, 1.0)["dt_limit"]
    ctx.close()
    return w


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32G])
@pytest.mark.parametrize("L", [2, 3])
def test_parareal_with_higher_order_relifting(prec, L):
    dev = device()
    w = _parareal_case()
    p = params(w.nx, w.nv, w.eps, prec, rho_bar=1.0, lift_order=L)
    ctx = mm.mm_create(p)
    out = torch.empty((w.n_slices + 1, w.nx), dtype=torch.float64, device=dev)
    info = mm.parareal_run(ctx, w.t_end, w.n_slices, 3, 0.0, torch.tensor(w.rho0, device=dev),
                           torch.tensor(w.g0, device=dev, dtype=gdtype(prec)), out)
    ctx.close()
    op = oparams(p)
    ref, err, it = O.parareal(op, w.rho0, w.g0, w.t_end, w.n_slices, 3, lift_order=L)
    assert info["iterations"] == it == 3
    # the oracle's own sensitivity to one-ulp changes of rho0 bounds what two
    # correct implementations that round differently can disagree by
    rng = np.random.default_rng(7)
    sens = 0.0
    for _ in range(2):
        r0 = w.rho0 * (1.0 + U * 2 * rng.choice([-1.0, 1.0], size=w.nx))
        o2, _, _ = O.parareal(op, r0, w.g0, w.t_end, w.n_slices, 3, lift_order=L)
        sens = max(sens, rel(o2, ref))
    tol = max(FP64_TOL, 20 * sens) if prec == mm.MM_FP64 else FP32_TOL
    got = out.cpu().numpy()
    assert rel(got, ref) <= tol, (rel(got, ref), tol)
    # the relifting order matters: order one gives a different iterate
    ref1, _, _ = O.parareal(oparams(p), w.rho0, w.g0, w.t_end, w.n_slices, 3, lift_order=1)
    assert rel(ref1, ref) > 100 * tol


@pytest.mark.parametrize("L", [2, 3])
def test_batch_engine_relifts_with_the_same_order(L):
    """The work-list kernel lifts inside the fine kernel: results equal
    parareal_run's with the same lifting order (to rounding)."""
    dev = device()
    w = _parareal_case()
    p = params(w.nx, w.nv, w.eps, mm.MM_FP32G, rho_bar=1.0, lift_order=L)
    cfg = (w.t_end, w.n_slices, 3, 0.0)
    outs = [np.empty((w.n_slices + 1, w.nx))]
    mm.parareal_run_many([p], [cfg], [np.ascontiguousarray(w.rho0)],
                         [np.ascontiguousarray(w.g0.astype(np.float32))], outs)
    ref, _, _ = O.parareal(oparams(p), w.rho0, w.g0, w.t_end, w.n_slices, 3, lift_order=L)
    assert rel(outs[0], ref) <= FP32_TOL, rel(outs[0], ref)
