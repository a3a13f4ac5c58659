"""Parity of the resident fine kernel (g held in the shared memory of a
thread-block cluster for the whole call) with the oracle, for every cluster
size and lane-group width it supports, and its agreement with the streaming
kernel on the same inputs.

FP32-g tolerances: <= 1e-5 relative (max-norm) on rho, <= 1e-3 on g; mass
drift <= 1e-12 relative.  The resident kernel advances the field by the
discrete Ampere identity instead of re-solving the Poisson law each step
(the two agree in exact arithmetic); the long-window test bounds the drift
this could add."""
import numpy as np
import pytest

import oracle as O
from paper_2511_13386_gb300 import mm, workloads as W
from tests.gpu_helpers import FP32_TOL, oparams, params, rel, run_fine

pytestmark = pytest.mark.gpu

# (nx, nv): cluster sizes 1, 2, 4, 8; lane groups of 4..32 lanes; runs of 4
# and 8 columns per group
SHAPES = [(1024, 64), (512, 64), (256, 64), (2048, 64), (2048, 128), (256, 256), (512, 32),
          (1024, 32), (1024, 128)]


def _state(nx, nv, batch, seed=11):
    w = W.batched(nx, nv, 1e-2, seed=W.SEED_BASE + seed)
    return w, *w.with_batch(batch)


@pytest.mark.parametrize("nx,nv", SHAPES)
def test_resident_matches_oracle(nx, nv):
    w, rho, g = _state(nx, nv, 2)
    p = params(nx, nv, w.eps, mm.MM_FP32G, rho_bar=1.0, fine_kernel=2)
    ctx = mm.mm_create(p)
    dt = mm.mm_query(ctx, 1.0)["dt_limit"]
    ctx.close()
    ro, go, mo, st, q = run_fine(p, rho, g, 37 * dt * (1 - 1e-9))
    assert q["n_steps"] == 37 and st["device_status"] == 0
    assert st["kinetic_updates"] == 2 * 37 * nx * nv
    assert (mo == 1).all()
    op = oparams(p)
    for b in range(2):
        r_ref, g_ref, _, _ = O.fine(op, q["n_steps"], q["dt"], rho[b], g[b])
        assert rel(ro[b], r_ref) <= FP32_TOL, (b, rel(ro[b], r_ref))
        assert rel(go[b], g_ref) <= 1e-3, (b, rel(go[b], g_ref))
        assert abs(ro[b].sum() - rho[b].sum()) / rho[b].sum() <= 1e-12


@pytest.mark.parametrize("steps", [1, 2, 5])
def test_resident_few_steps_and_equilibrium(steps):
    """1, 2 and 5 steps; a global equilibrium (rho = 1, g = 0) stays fixed."""
    nx, nv = 1024, 64
    w, rho, g = _state(nx, nv, 2)
    rho[1] = 1.0
    g[1] = 0.0
    p = params(nx, nv, w.eps, mm.MM_FP32G, rho_bar=1.0, fine_kernel=2)
    ctx = mm.mm_create(p)
    dt = mm.mm_query(ctx, 1.0)["dt_limit"]
    ctx.close()
    ro, go, _, st, q = run_fine(p, rho, g, steps * dt * (1 - 1e-9))
    assert q["n_steps"] == steps
    r_ref, g_ref, _, _ = O.fine(oparams(p), steps, q["dt"], rho[0], g[0])
    assert rel(ro[0], r_ref) <= FP32_TOL
    assert rel(go[0], g_ref) <= 1e-3
    assert np.array_equal(ro[1], np.ones(nx)) and not go[1].any()


def test_resident_long_window_and_field_drift():
    """2000 steps on the batched grid: the Ampere update of the field must
    not drift from the Poisson law the oracle solves every step."""
    nx, nv = 1024, 64
    w, rho, g = _state(nx, nv, 2, seed=5)
    p = params(nx, nv, w.eps, mm.MM_FP32G, rho_bar=1.0, fine_kernel=2)
    ctx = mm.mm_create(p)
    dt = mm.mm_query(ctx, 1.0)["dt_limit"]
    ctx.close()
    ro, go, _, st, q = run_fine(p, rho, g, 2000 * dt * (1 - 1e-12), mask=False)
    for b in range(2):
        r_ref, g_ref, _, _ = O.fine(oparams(p), q["n_steps"], q["dt"], rho[b], g[b])
        assert rel(ro[b], r_ref) <= FP32_TOL, rel(ro[b], r_ref)
        assert rel(go[b], g_ref) <= 1e-3
        assert abs(ro[b].sum() - rho[b].sum()) / rho[b].sum() <= 1e-12


def test_resident_rho_bar_from_input_mean():
    nx, nv = 1024, 64
    w, rho, g = _state(nx, nv, 2)
    rho[1] *= 1.3
    p = params(nx, nv, w.eps, mm.MM_FP32G, rho_bar=float("nan"), fine_kernel=2)
    ctx = mm.mm_create(p)
    dt = mm.mm_query(ctx, 1.0)["dt_limit"]
    ctx.close()
    ro, _, _, _, q = run_fine(p, rho, g, 20 * dt * (1 - 1e-9), mask=False)
    for b in range(2):
        op = oparams(p)
        op.rho_bar = float(rho[b].mean())
        r_ref, _, _, _ = O.fine(op, q["n_steps"], q["dt"], rho[b], g[b])
        assert rel(ro[b], r_ref) <= FP32_TOL


@pytest.mark.parametrize("nx,nv", [(1024, 64), (1024, 32)])
def test_resident_agrees_with_streaming(nx, nv):
    w, rho, g = _state(nx, nv, 3)
    outs = []
    for kernel in (1, 2):
        p = params(nx, nv, w.eps, mm.MM_FP32G, rho_bar=1.0, fine_kernel=kernel)
        outs.append(run_fine(p, rho, g, 1e-4, mask=False))
    (r1, g1, _, _, _), (r2, g2, _, _, _) = outs
    assert rel(r2, r1) <= 2 * FP32_TOL
    assert rel(g2, g1) <= 2e-3


def test_resident_rejects_unsupported_options():
    for kw in (dict(adapt=1), dict(flux_rule=1), dict(precision=mm.MM_FP64), dict(nv=48),
               dict(nx=8192, nv=32), dict(nx=64, nv=64), dict(nx=2048, nv=16)):
        base = dict(nx=1024, nv=64, eps=1e-2, prec=mm.MM_FP32G)
        if "precision" in kw:
            base["prec"] = kw.pop("precision")
        base.update({k: v for k, v in kw.items() if k in ("nx", "nv")})
        extra = {k: v for k, v in kw.items() if k not in ("nx", "nv")}
        p = params(base["nx"], base["nv"], base["eps"], base["prec"], fine_kernel=2, **extra)
        with pytest.raises(mm.MMError) as e:
            mm.mm_create(p)
        assert e.value.status == mm.MM_ERR_INVALID


def _rounds_case(rho_bar):
    """640 states of Nx=256, Nv=32 (one CTA each, two per SM): more states
    than the GPU holds at once, over enough steps that the launch runs in
    rounds of step chunks."""
    nx, nv, B, steps = 256, 32, 640, 380
    w, rho, g = _state(nx, nv, 8, seed=23)
    rho = np.tile(rho, (B // 8, 1)) * (1.0 + 0.01 * np.arange(B))[:, None]
    g = np.tile(g, (B // 8, 1, 1))
    p = params(nx, nv, w.eps, mm.MM_FP32G, rho_bar=rho_bar, fine_kernel=2)
    ctx = mm.mm_create(p)
    dt = mm.mm_query(ctx, 1.0)["dt_limit"]
    ctx.close()
    return p, rho, g, steps * dt * (1 - 1e-9), steps


@pytest.mark.parametrize("rho_bar", [1.0, float("nan")], ids=["fixed", "input-mean"])
def test_resident_rounds_of_step_chunks(rho_bar):
    """States in every round and chunk position match the oracle; every
    state conserves mass; the kinetic-update count covers every chunk."""
    p, rho, g, span, steps = _rounds_case(rho_bar)
    ro, go, mo, st, q = run_fine(p, rho, g, span)
    B, nx, nv = rho.shape[0], p.nx, p.nv
    assert q["n_steps"] == steps and st["device_status"] == 0
    assert st["launches"] > 1, st
    assert st["kinetic_updates"] == B * steps * nx * nv
    assert (mo == 1).all()
    assert np.abs(ro.sum(axis=1) - rho.sum(axis=1)).max() / rho.sum(axis=1).max() <= 1e-12
    for b in (0, 151, 303, 304, 455, 607, 639):
        op = oparams(p)
        if np.isnan(rho_bar):
            op.rho_bar = float(rho[b].mean())
        r_ref, g_ref, _, _ = O.fine(op, q["n_steps"], q["dt"], rho[b], g[b])
        assert rel(ro[b], r_ref) <= FP32_TOL, (b, rel(ro[b], r_ref))
        assert rel(go[b], g_ref) <= 1e-3, (b, rel(go[b], g_ref))


def test_resident_rounds_in_place():
    """Rounds with the outputs aliasing the inputs give the same bits as
    with separate outputs."""
    torch = pytest.importorskip("torch")
    from tests.gpu_helpers import device
    dev = device()
    p, rho, g, span, _ = _rounds_case(1.0)
    ctx = mm.mm_create(p)
    r = torch.tensor(rho, device=dev)
    gg = torch.tensor(g, device=dev, dtype=torch.float32)
    ro, go = torch.empty_like(r), torch.empty_like(gg)
    st = mm.mm_fine_propagate(ctx, rho.shape[0], span, r, gg, ro, go, stats=True)
    assert st["launches"] > 1
    mm.mm_fine_propagate(ctx, rho.shape[0], span, r, gg, r, gg)
    ctx.close()
    assert torch.equal(r, ro) and torch.equal(gg, go)
