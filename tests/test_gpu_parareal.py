"""Parity of the coarse propagator, the lifting and the device parareal loop
(Algorithm 1) with the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2511_13386_gb300 import mm, workloads as W
from tests.gpu_helpers import (FP32_TOL, FP64_TOL, device, gdtype, oparams, params,
                               parareal_with_sensitivity, rel)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,steps", [(0, 1), (0, 3), (1, 1)])
@pytest.mark.parametrize("nx", [64, 1024, 4096])
def test_coarse_parity(kind, steps, nx):
    dev = device()
    w = W.batched(nx=nx, nv=16, eps=1e-2)
    rho, _ = w.with_batch(3)
    p = params(nx, 16, 1e-2, mm.MM_FP64, rho_bar=1.0, coarse_kind=kind, coarse_steps=steps)
    ctx = mm.mm_create(p)
    span = 1.0 / 128
    r = torch.tensor(rho, device=dev)
    out = torch.empty_like(r)
    mm.mm_coarse(ctx, 3, span, r, out)
    out = out.cpu().numpy()
    ctx.close()
    op = oparams(p)
    n_sub = steps
    if kind == 1:
        _, _, _, m2 = O.velocity_grid(op)
        lim = 0.9 * (1.0 / nx) ** 2 / (2 * m2)
        n_sub = max(steps, int(np.ceil(span / lim)))
    for b in range(3):
        ref = O.coarse(op, span, rho[b], kind=kind, n_sub=n_sub)
        assert rel(out[b], ref) <= FP64_TOL, rel(out[b], ref)


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32G])
def test_lift_parity(prec):
    dev = device()
    w = W.batched(nx=512, nv=64, eps=1e-2)
    rho, _ = w.with_batch(2)
    p = params(512, 64, 1e-2, prec, rho_bar=1.0)
    ctx = mm.mm_create(p)
    r = torch.tensor(rho, device=dev)
    g = torch.empty((2, 512, 64), device=dev, dtype=gdtype(prec))
    mm.mm_lift(ctx, 2, r, g)
    ctx.close()
    for b in range(2):
        ref = O.lift(oparams(p), rho[b])
        tol = FP64_TOL if prec == mm.MM_FP64 else 1e-6
        assert rel(g[b].double().cpu().numpy(), ref) <= tol


def _parareal(prec, w, K, tol=0.0, **kw):
    dev = device()
    p = params(w.nx, w.nv, w.eps, prec, v_max=w.v_max, rho_bar=1.0, **kw)
    ctx = mm.mm_create(p)
    out = torch.empty((w.n_slices + 1, w.nx), dtype=torch.float64, device=dev)
    info = mm.parareal_run(ctx, w.t_end, w.n_slices, K, tol, torch.tensor(w.rho0, device=dev),
                           torch.tensor(w.g0, device=dev, dtype=gdtype(prec)), out)
    ctx.close()
    return p, out.cpu().numpy(), info


def test_parareal_small_workload():
    """The small workload (FP64): Nx=64, Nv=32, eps=1, T=0.05, N=4, K=4.
    Slices 0 and 1 (one fine propagation from the given data) at 1e-12;
    the later slices within the oracle's own rounding sensitivity."""
    w = W.small()
    p, out, info = _parareal(mm.MM_FP64, w, w.max_iter)
    ref, err, it, sens = parareal_with_sensitivity(oparams(p), w, w.max_iter)
    assert info["iterations"] == it
    assert rel(out[:2], ref[:2]) <= FP64_TOL
    assert rel(out, ref) <= max(FP64_TOL, 20 * sens), (rel(out, ref), sens)
    assert np.allclose(info["err"], err, rtol=1e-6, atol=1e-14)
    assert info["mass_drift"] <= 1e-12


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32G])
def test_parareal_batched_grid_reduced_span(prec):
    """The batched workload's grid (Nx=1024, Nv=64, eps=1e-2) with N=6
    slices over a short span, K=3, and stopping on a tolerance."""
    w = W.batched(n_slices=6)
    w.t_end = 6 * 25 * 1.0986e-6
    p, out, info = _parareal(prec, w, 3)
    ref, err, it = O.parareal(oparams(p), w.rho0, w.g0, w.t_end, w.n_slices, 3)
    assert info["iterations"] == it
    tol = FP64_TOL if prec == mm.MM_FP64 else FP32_TOL
    assert rel(out, ref) <= tol, rel(out, ref)
    # tolerance stop: same iteration count as the oracle
    p2, out2, info2 = _parareal(prec, w, 6, tol=err[1] * 1.0001)
    ref2, err2, it2 = O.parareal(oparams(p2), w.rho0, w.g0, w.t_end, w.n_slices, 6, tol=err[1] * 1.0001)
    assert info2["iterations"] == it2 == 2


def test_parareal_reproduces_sequential_at_K_equals_N():
    w = W.small(nx=64, nv=32)
    p, out, info = _parareal(mm.MM_FP64, w, w.n_slices)
    seq = O.sequential(oparams(p), w.rho0, w.g0, w.t_end, w.n_slices)
    _, _, _, sens = parareal_with_sensitivity(oparams(p), w, w.n_slices)
    assert rel(out, seq) <= max(FP64_TOL, 20 * sens), (rel(out, seq), sens)


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32G])
def test_parareal_hybrid(prec):
    """Parareal with domain adaptation on (hybrid bump, small grid)."""
    w = W.hybrid(nx=256, nv=32, eps=1e-2, n_slices=4, v_max=8.0)
    w.t_end = 4 * 30 * 4.0e-6
    p, out, info = _parareal(prec, w, 2, adapt=1, thr_g=1e-3, thr_R=1e-2, r_scale=1)
    ref, err, it = O.parareal(oparams(p), w.rho0, w.g0, w.t_end, w.n_slices, 2)
    tol = FP64_TOL if prec == mm.MM_FP64 else FP32_TOL
    assert rel(out, ref) <= tol, rel(out, ref)


@pytest.mark.parametrize("eps,L", [(1.0, 1), (1e-1, 3), (1e-3, 3)])
def test_parareal_paper_setup(eps, L):
    """The paper's own setup (Sec. 5) in its 1D-1V reduction: torus length
    2 pi, f = M v^4 (1 + 0.9 cos x), thresholds 1e-5 on both criteria,
    lifting of order 3 (order 1 at eps = 1, where the truncated
    Chapman-Enskog series of order 3 makes the relifted iteration diverge
    on this data, eps k = 1); here N = 8 slices over T = 0.2 and K = 3,
    FP64, against the oracle's Algorithm 1 with the same options."""
    dev = device()
    w = W.paper(eps, n_slices=8)
    w.t_end = 0.2
    p = params(w.nx, w.nv, eps, mm.MM_FP64, v_max=w.v_max, x_len=w.x_len, rho_bar=w.rho_bar,
               adapt=1, thr_g=w.thr_g, thr_R=w.thr_R, r_scale=w.r_scale, lift_order=L)
    ctx = mm.mm_create(p)
    out = torch.empty((w.n_slices + 1, w.nx), dtype=torch.float64, device=dev)
    info = mm.parareal_run(ctx, w.t_end, w.n_slices, 3, 0.0, torch.tensor(w.rho0, device=dev),
                           torch.tensor(w.g0, device=dev), out)
    ctx.close()
    op = oparams(p)
    ref, err, it = O.parareal(op, w.rho0, w.g0, w.t_end, w.n_slices, 3, lift_order=L)
    assert info["iterations"] == it == 3
    got = out.cpu().numpy()
    # slice 1 is one fine propagation of the given data: 1e-12; later slices
    # within the oracle's own sensitivity to one-ulp changes of rho0
    assert rel(got[:2], ref[:2]) <= FP64_TOL, rel(got[:2], ref[:2])
    rng = np.random.default_rng(3)
    sens = 0.0
    for _ in range(2):
        r0 = w.rho0 * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=w.nx))
        o2, _, _ = O.parareal(op, r0, w.g0, w.t_end, w.n_slices, 3, lift_order=L)
        sens = max(sens, rel(o2, ref))
    assert rel(got, ref) <= max(FP64_TOL, 20 * sens), (rel(got, ref), sens)
    assert info["mass_drift"] <= 1e-12


@pytest.mark.parametrize("prec,L", [(mm.MM_FP64, 1), (mm.MM_FP64, 3), (mm.MM_FP32G, 1)])
def test_full_state_parareal(prec, L):
    """MM_PARAREAL_FULL_STATE: the slices carry (rho, g); against the
    oracle's full-state Algorithm 1 after 2 iterations, and at K = N the
    plain sequential F (no relifting) within the parity tolerance."""
    dev = device()
    w = W.batched(nx=128, nv=32, eps=1e-2, n_slices=4)
    p = params(w.nx, w.nv, w.eps, prec, rho_bar=1.0, lift_order=L)
    ctx = mm.mm_create(p)
    w.t_end = 4 * 30 * mm.mm_query(ctx, 1.0)["dt_limit"]
    gdt = gdtype(prec)
    outs = {}
    for K in (2, 4):
        out = torch.empty((w.n_slices + 1, w.nx), dtype=torch.float64, device=dev)
        info = mm.parareal_run(ctx, w.t_end, w.n_slices, K, 0.0, torch.tensor(w.rho0, device=dev),
                               torch.tensor(w.g0, device=dev, dtype=gdt), out, mode=mm.MM_PARAREAL_FULL_STATE)
        assert info["iterations"] == K
        outs[K] = out.cpu().numpy()
    ctx.close()
    op = oparams(p)
    tol = FP64_TOL if prec == mm.MM_FP64 else FP32_TOL
    ref, err, it = O.parareal(op, w.rho0, w.g0, w.t_end, w.n_slices, 2, lift_order=L, mode=1)
    assert rel(outs[2], ref) <= tol, rel(outs[2], ref)
    plain = O.sequential(op, w.rho0, w.g0, w.t_end, w.n_slices, mode=1)
    assert rel(outs[4], plain) <= tol, rel(outs[4], plain)
    # the density mode reaches the relifted sequence, a different one
    seq = O.sequential(op, w.rho0, w.g0, w.t_end, w.n_slices, lift_order=L)
    assert rel(seq, plain) > 100 * tol


def test_batch_rejects_full_state():
    device()
    w = W.small()
    p = params(w.nx, w.nv, w.eps, mm.MM_FP32G, rho_bar=1.0)
    b = mm.mm_batch_create()
    with pytest.raises(mm.MMError) as e:
        mm.mm_batch_add(b, p, w.t_end, w.n_slices, 2, 0.0, np.ascontiguousarray(w.rho0),
                        np.ascontiguousarray(w.g0.astype(np.float32)), mode=mm.MM_PARAREAL_FULL_STATE)
    assert e.value.status == mm.MM_ERR_INVALID
    b.close()


def test_parareal_overlapped_with_fine_rounds():
    """More slice states than the GPU holds at once (320 states of Nx=256,
    Nv=32, one CTA each, two per SM), 400 fine steps per slice: the resident
    kernel runs in rounds of step chunks, the rest of the coarse guess and
    its lifting run on a second stream during the first round, and the
    correction of the slices whose last chunk has run during the last
    round.  Two iterations against the oracle's Algorithm 1."""
    N = 320
    w = W.batched(256, 32, 1e-2, n_slices=N)
    p = params(256, 32, 1e-2, mm.MM_FP32G, v_max=w.v_max, rho_bar=1.0, fine_kernel=2)
    ctx = mm.mm_create(p)
    w.t_end = N * 400 * mm.mm_query(ctx, 1.0)["dt_limit"] * (1 - 1e-9)
    ctx.close()
    p, out, info = _parareal(mm.MM_FP32G, w, 2, fine_kernel=2)
    assert info["fine_launches"] > 2, info  # rounds in both iterations
    ref, err, it = O.parareal(oparams(p), w.rho0, w.g0, w.t_end, N, 2)
    assert info["iterations"] == it == 2
    assert rel(out, ref) <= FP32_TOL, rel(out, ref)
    # successive errors: the FP32 path's density carries ~1e-7 rounding
    assert np.allclose(info["err"], err, rtol=1e-3, atol=1e-6), (info["err"], err)
    assert info["mass_drift"] <= 1e-12


def _lapack_step(op, rho, dt):
    """The linearly implicit S^0 step solved another way: E from the
    oracle's Poisson law, the cyclic tridiagonal system (I - m2 dt L_E) x =
    rho written out and solved by LAPACK's banded LU with the two corner
    entries handled by the Sherman-Morrison formula."""
    from scipy.linalg import solve_banded
    nx = op.nx
    dx = op.x_len / nx
    E = O.poisson(op, rho)
    _, _, _, m2 = O.velocity_grid(op)
    k, idx = m2 * dt / dx, 1.0 / dx
    El = np.roll(E, 1)
    lo, up = -k * (idx + 0.5 * El), -k * (idx - 0.5 * E)
    di = 1.0 - k * (-2.0 * idx - 0.5 * E + 0.5 * El)
    gamma = -di[0]
    d2 = di.copy()
    d2[0] -= gamma
    d2[-1] -= up[-1] * lo[0] / gamma
    ab = np.zeros((3, nx))
    ab[0, 1:], ab[1], ab[2, :-1] = up[:-1], d2, lo[1:]
    u = np.zeros(nx)
    u[0], u[-1] = gamma, up[-1]
    y, z = solve_banded((1, 1), ab, rho), solve_banded((1, 1), ab, u)
    return y - z * (y[0] + lo[0] * y[-1] / gamma) / (1.0 + z[0] + lo[0] * z[-1] / gamma)


def _chain_rounding_spread(op, rho0, span, N, ref, fr=None, want=None):
    """How far correct double-precision evaluations of the same chain of
    implicit steps drift apart, for the coarse guess and, given the fine
    results `fr` and the oracle's corrected states `want`, for one
    correction sweep: the larger of (a) the oracle's chain against the same
    chain solved by LAPACK on the oracle's own coefficients, and (b) the
    oracle's chain against itself from a density perturbed by one ulp per
    cell, which stands for a different rounding of the coefficients (an
    implementation that computes the field in another summation order).
    At Nx = 4096 the system's conditioning makes (a) 3.9e-12 after 12
    steps, above the 1e-12 parity target; below Nx = 1024 both are ~1e-13."""
    def guess(step, r0):
        r = [r0]
        for n in range(N):
            r.append(step(op, r[-1], span))
        return np.array(r)

    def sweep(step, g0):
        c, gprev = g0.copy(), g0.copy()
        for n in range(N):
            gn = step(op, c[n], span)
            c[n + 1] = fr[n + 1] + (gn - gprev[n + 1])
        return c

    rng = np.random.default_rng(11)
    cands = [(_lapack_step, rho0)]
    for _ in range(3):
        cands.append((lambda o, r, dt: O.coarse(o, dt, r),
                      rho0 * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=rho0.size))))
    spread = 0.0
    for step, r0 in cands:
        r = guess(step, r0)
        spread = max(spread, rel(r, ref))
        if fr is not None:
            spread = max(spread, rel(sweep(step, r), want))
    return spread


@pytest.mark.parametrize("nx", [64, 256, 1024, 2048, 4096, 8192, 32768])
def test_coarse_guess_and_correction_entry_points(nx):
    """Algorithm 1's sequential parts through their own entry points (from
    Nx = 256 one solve's implicit step runs over a thread-block cluster,
    one row per thread up to Nx = 1024 and chunks of 2, 4, 8 and 32 rows
    per thread beyond; Nx = 64 on one CTA): the coarse guess rho^{n+1,0} = G(rho^{n,0}) over 12 slices and
    one correction sweep rho^{n+1,1} = F + (G(rho^{n,1}) - G(rho^{n,0})),
    against the oracle's G composed slice by slice: at 1e-12, or where the
    chain's conditioning makes correct double-precision evaluations drift
    further apart than that (Nx >= 4096), within twice their drift."""
    dev = device()
    N = 12
    w = W.batched(nx=nx, nv=16, eps=1e-2)
    p = params(nx, 16, 1e-2, mm.MM_FP64, rho_bar=1.0)
    ctx = mm.mm_create(p)
    # one coarse step per slice of 1/128, shortened above Nx = 4096 so that
    # m2 dt / dx^2 stays at its Nx = 4096 value (1.3e5), as in a solve whose
    # slices hold a fixed number of fine steps
    span = 1.0 / 128 * min(1.0, (4096 / nx) ** 2)
    rho = torch.zeros((N + 1, nx), dtype=torch.float64, device=dev)
    rho[0] = torch.tensor(w.rho0, device=dev)
    gp = torch.zeros_like(rho)
    mm.mm_coarse_guess(ctx, N, span, rho, gp)
    got = rho.cpu().numpy()
    op = oparams(p)
    ref = np.empty((N + 1, nx))
    ref[0] = w.rho0
    for n in range(N):
        ref[n + 1] = O.coarse(op, span, ref[n])
    tol = max(FP64_TOL, 2.0 * _chain_rounding_spread(op, w.rho0, span, N, ref))
    assert rel(got, ref) <= tol, (rel(got, ref), tol)
    assert np.array_equal(gp.cpu().numpy()[1:], got[1:])
    # one correction sweep with fine results F = G + a smooth offset
    rng = np.random.default_rng(5)
    fr = ref + 1e-3 * np.sin(2 * np.pi * (np.arange(nx) + 0.5) / nx)[None, :] * rng.uniform(0.5, 1.5, (N + 1, 1))
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    mm.mm_parareal_correct(ctx, N, 0, span, rho, torch.tensor(fr, device=dev), gp, err)
    want = ref.copy()
    gprev = ref.copy()
    for n in range(N):
        gn = O.coarse(op, span, want[n])
        want[n + 1] = fr[n + 1] + (gn - gprev[n + 1])
        gprev[n + 1] = gn
    tol = max(FP64_TOL, 2.0 * _chain_rounding_spread(op, w.rho0, span, N, ref, fr, want))
    assert rel(rho.cpu().numpy(), want) <= tol, (rel(rho.cpu().numpy(), want), tol)
    # the successive error, a difference of two states each held to tol
    e_ref = np.abs(want - ref).max()
    assert abs(err.item() - e_ref) <= max(1e-9 * e_ref, 2.0 * tol * np.abs(want).max()), (err.item(), e_ref)
    ctx.close()
