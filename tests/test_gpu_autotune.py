"""The launch-shape autotuner of F: every candidate it times runs the same
scheme (results agree with the oracle to the FP32 tolerances), the choice
is one of the candidates and the fastest of them, mm_query and later calls
use it, params.fine_kernel restricts the candidates, and batch 0 restores
the default."""
import numpy as np
import pytest

import oracle as O
from paper_2511_13386_gb300 import mm, workloads as W
from tests.gpu_helpers import FP32_TOL, device, oparams, params, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _arrays(w, batch, dev, gdt=None):
    rho, g = w.with_batch(batch)
    gdt = gdt or torch.float32
    r = torch.tensor(rho, device=dev)
    gg = torch.tensor(g, device=dev, dtype=gdt)
    return rho, g, r, gg, torch.empty_like(r), torch.empty_like(gg)


def test_autotune_batched_grid_picks_fastest_and_stays_correct():
    dev = device()
    w = W.batched()
    rho, g, r, gg, ro, go = _arrays(w, 8, dev)
    p = params(w.nx, w.nv, w.eps, mm.MM_FP32G, rho_bar=1.0)
    ctx = mm.mm_create(p)
    default = mm.mm_query(ctx, 1.0)
    res = mm.mm_autotune(ctx, 8, 24, r, gg, ro, go)
    cands = res["candidates"]
    # resident with clusters of 4 and 8 CTAs (256 and 128 cells per CTA)
    # and the streaming layouts of 8, 4, 2 nodes per lane (nv = 64)
    kinds = {(c["fine_kernel"], c["cluster"], c["vpt"]) for c in cands}
    assert (1, 1, 8) in kinds and (1, 1, 4) in kinds and (1, 1, 2) in kinds
    assert {c["cluster"] for c in cands if c["fine_kernel"] == 2} == {4, 8}
    assert res["n_candidates"] == 5
    assert all(c["ms"] > 0 for c in cands)
    assert res["best_ms"] == min(c["ms"] for c in cands)
    q = mm.mm_query(ctx, 1.0)
    assert (q["fine_kernel"], q["cluster"]) == (res["fine_kernel"], res["cluster"])
    if res["fine_kernel"] == 1:
        assert q["vpt"] == res["vpt"]
    # the tuned shape computes the same F
    span = 30 * q["dt_limit"] * (1 - 1e-9)
    st = mm.mm_fine_propagate(ctx, 8, span, r, gg, ro, go, stats=True)
    assert st["device_status"] == 0
    op = oparams(p)
    ro_h = ro.cpu().numpy()
    for b in (0, 5):
        r_ref, _, _, _ = O.fine(op, 30, mm.mm_query(ctx, span)["dt"], rho[b], g[b])
        assert rel(ro_h[b], r_ref) <= FP32_TOL
    # batch 0 restores the default choice
    mm.mm_autotune(ctx, 0, 1, None, None, None, None)
    d2 = mm.mm_query(ctx, 1.0)
    assert (d2["fine_kernel"], d2["cluster"], d2["vpt"]) == (default["fine_kernel"], default["cluster"],
                                                              default["vpt"])
    ctx.close()


@pytest.mark.parametrize("prec,vpt", [(mm.MM_FP32G, 8), (mm.MM_FP32G, 4), (mm.MM_FP32G, 2), (mm.MM_FP32G, 1),
                                      (mm.MM_FP64, 4), (mm.MM_FP64, 2), (mm.MM_FP64, 1)])
def test_every_streaming_layout_matches_oracle(prec, vpt):
    """Each lane layout the tuner may pick for the streaming kernel, forced
    with params.fine_vpt, on a hybrid state (adaptation, both criteria)
    against the oracle: identical masks in FP64."""
    dev = device()
    nx, nv = 520, 32
    w = W.hybrid(nx=nx, nv=nv, eps=1e-2, v_max=8.0)
    rho, g = w.with_batch(2)
    rho = rho + 0.01 * np.cos(2 * np.pi * (np.arange(nx) + 0.5) / nx)[None, :]
    p = params(nx, nv, 1e-2, prec, rho_bar=1.0, adapt=1, thr_g=1e-3, thr_R=1e-2, r_scale=1,
               fine_kernel=1, fine_vpt=vpt)
    ctx = mm.mm_create(p)
    q = mm.mm_query(ctx, 1.0)
    assert q["vpt"] == vpt and q["fine_kernel"] == 1
    span = 40 * q["dt_limit"] * (1 - 1e-9)
    dt = mm.mm_query(ctx, span)["dt"]
    gdt = torch.float32 if prec == mm.MM_FP32G else torch.float64
    r = torch.tensor(rho, device=dev)
    gg = torch.tensor(g, device=dev, dtype=gdt)
    ro, go = torch.empty_like(r), torch.empty_like(gg)
    mo = torch.empty(r.shape, dtype=torch.uint8, device=dev)
    st = mm.mm_fine_propagate(ctx, 2, span, r, gg, ro, go, mo, stats=True)
    assert st["device_status"] == 0
    res = mm.mm_autotune(ctx, 2, 4, r, gg, torch.empty_like(r), torch.empty_like(gg))
    assert res["n_candidates"] == 1 and res["vpt"] == vpt   # fine_vpt restricts the tuner
    ctx.close()
    op = oparams(p)
    for b in range(2):
        r_ref, g_ref, m_ref, _ = O.fine(op, 40, dt, rho[b], g[b])
        if prec == mm.MM_FP64:
            assert rel(ro[b].cpu().numpy(), r_ref) <= 1e-12
            assert np.array_equal(mo[b].cpu().numpy(), m_ref)
        else:
            assert rel(ro[b].cpu().numpy(), r_ref) <= FP32_TOL
            assert (mo[b].cpu().numpy() != m_ref).sum() <= 2
        assert 0 < m_ref.sum() < nx


def test_fine_vpt_rejects_impossible_layouts():
    device()
    with pytest.raises(mm.MMError):
        mm.mm_create(params(64, 32, 1.0, mm.MM_FP64, fine_vpt=8))    # FP64: 8 per lane only where 4 cannot
    mm.mm_create(params(64, 256, 1.0, mm.MM_FP64, fine_vpt=8)).close()  # nv = 256: 4 per lane needs 64 lanes
    with pytest.raises(mm.MMError):
        mm.mm_create(params(64, 12, 1.0, mm.MM_FP32G, fine_vpt=4))   # nv/2 = 6 is not a multiple of 4
    with pytest.raises(mm.MMError):
        mm.mm_create(params(64, 32, 1.0, mm.MM_FP32G, fine_vpt=3))


def test_autotune_rejects_aliased_outputs():
    dev = device()
    w = W.small()
    rho, g, r, gg, ro, go = _arrays(w, 2, dev, torch.float64)
    ctx = mm.mm_create(params(w.nx, w.nv, w.eps, mm.MM_FP64, rho_bar=1.0))
    with pytest.raises(mm.MMError) as e:
        mm.mm_autotune(ctx, 2, 4, r, gg, ro, gg)
    assert e.value.status == mm.MM_ERR_INVALID
    res = mm.mm_autotune(ctx, 2, 4, r, gg, ro, go)
    assert res["fine_kernel"] == 1 and res["n_candidates"] == 3   # FP64: 4, 2, 1 nodes per lane
    ctx.close()


def test_autotune_measures_the_step_chunk_entry_cost():
    """When the resident kernel wins, the tuner times one full wave for
    `steps` and 2 `steps` steps and keeps the entry cost of a step chunk (in
    steps) that sets the steps per launch of larger batches; a batch of 160
    states (more than the GPU holds at once) then runs in rounds of chunks
    and still matches the oracle."""
    dev = device()
    w = W.batched()
    B = 160
    rho, g, r, gg, ro, go = _arrays(w, B, dev)
    p = params(w.nx, w.nv, w.eps, mm.MM_FP32G, rho_bar=1.0)
    p.fine_kernel = 2
    ctx = mm.mm_create(p)
    res = mm.mm_autotune(ctx, B, 32, r, gg, ro, go)
    assert res["fine_kernel"] == 2
    assert 0.0 < res["res_entry_steps"] < 1000.0
    q = mm.mm_query(ctx, 1.0)
    span = 200 * q["dt_limit"] * (1 - 1e-9)
    st = mm.mm_fine_propagate(ctx, B, span, r, gg, ro, go, stats=True)
    assert st["device_status"] == 0 and st["launches"] > 1
    op = oparams(p)
    dt = mm.mm_query(ctx, span)["dt"]
    ro_h = ro.cpu().numpy()
    for b in (0, B - 1):
        r_ref, _, _, _ = O.fine(op, 200, dt, rho[b], g[b])
        assert rel(ro_h[b], r_ref) <= FP32_TOL
    mm.mm_autotune(ctx, 0, 1, None, None, None, None)
    ctx.close()


def test_set_chunk_entry_fixes_the_launch_plan():
    """mm_set_chunk_entry replaces the measured entry cost in the launch
    planner: a very high cost runs a batch larger than the GPU holds as one
    launch of whole states (two waves), a low one in rounds of chunks; both results match the
    oracle, and out-of-range costs are refused."""
    dev = device()
    w = W.batched()
    B = 160
    rho, g, r, gg, ro, go = _arrays(w, B, dev)
    p = params(w.nx, w.nv, w.eps, mm.MM_FP32G, rho_bar=1.0)
    p.fine_kernel = 2
    ctx = mm.mm_create(p)
    mm.mm_autotune(ctx, B, 32, r, gg, ro, go)
    q = mm.mm_query(ctx, 1.0)
    span = 200 * q["dt_limit"] * (1 - 1e-9)
    dt = mm.mm_query(ctx, span)["dt"]
    op = oparams(p)
    launches = {}
    for e in (1.0, 1000.0):
        mm.mm_set_chunk_entry(ctx, e)
        st = mm.mm_fine_propagate(ctx, B, span, r, gg, ro, go, stats=True)
        assert st["device_status"] == 0
        launches[e] = st["launches"]
        ro_h = ro.cpu().numpy()
        for b in (0, B - 1):
            r_ref, _, _, _ = O.fine(op, 200, dt, rho[b], g[b])
            assert rel(ro_h[b], r_ref) <= FP32_TOL
    assert launches[1.0] > launches[1000.0] == 1, launches  # rounds of chunks vs one launch of whole states
    for bad in (-1.0, 1001.0, float("nan")):
        with pytest.raises(mm.MMError):
            mm.mm_set_chunk_entry(ctx, bad)
    ctx.close()
