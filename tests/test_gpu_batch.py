"""Many parareal solves of uneven shapes advanced together (mm_batch /
parareal_run_many): one persistent work-list launch per iteration for all
fine propagations of all solves.

Each solve's result must agree with the single-solve path (parareal_run) and
with the oracle at the FP64 / FP32 tolerances, and must not depend on which
other solves share the batch (bitwise: every (solve, slice) item is computed
by one CTA independently of the rest of the list)."""
import numpy as np
import pytest

import oracle as O
from paper_2511_13386_gb300 import mm, workloads as W
from tests.gpu_helpers import FP32_TOL, FP64_TOL, device, gdtype, oparams, params, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _mixed_set():
    """Solves of different grids, Knudsen numbers, slice counts, iteration
    caps, precisions and adaptation; short spans so the oracle is fast."""
    out = []
    specs = [  # nx, nv, eps, N, K, prec, adapt
        (64, 32, 1.0, 4, 4, mm.MM_FP64, 0),
        (128, 32, 1e-2, 5, 3, mm.MM_FP64, 0),
        (256, 64, 1e-2, 3, 2, mm.MM_FP64, 1),
        (128, 64, 1e-1, 4, 2, mm.MM_FP32G, 0),
        (256, 32, 1e-2, 6, 3, mm.MM_FP32G, 1),
        (512, 64, 1e-3, 3, 2, mm.MM_FP32G, 0),
    ]
    for q, (nx, nv, eps, N, K, prec, adapt) in enumerate(specs):
        w = W.batched(nx, nv, eps, seed=W.SEED_BASE + 31 * q, n_slices=N)
        p = params(nx, nv, eps, prec, rho_bar=1.0, adapt=adapt, thr_g=1e-3, thr_R=1e-2, r_scale=1)
        ctx = mm.mm_create(p)
        dt = mm.mm_query(ctx, 1.0)["dt_limit"]
        ctx.close()
        t_end = N * (6 + 3 * q) * dt * (1 - 1e-9)
        out.append((p, w, t_end, N, K))
    return out


def _sensitivity(p, w, t_end, N, K, ref):
    """The oracle's own change under one-ulp perturbations of rho0."""
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(2):
        r = w.rho0 * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=w.nx))
        out, _, _ = O.parareal(oparams(p), r, w.g0, t_end, N, K)
        worst = max(worst, rel(out, ref))
    return worst


def _single(p, w, t_end, N, K, tol=0.0):
    dev = device()
    ctx = mm.mm_create(p)
    out = torch.empty((N + 1, w.nx), dtype=torch.float64, device=dev)
    info = mm.parareal_run(ctx, t_end, N, K, tol, torch.tensor(w.rho0, device=dev),
                           torch.tensor(w.g0, device=dev, dtype=gdtype(p.precision)), out)
    ctx.close()
    return out.cpu().numpy(), info


def _host_g0(p, w):
    return np.ascontiguousarray(w.g0.astype(np.float32 if p.precision == mm.MM_FP32G else np.float64))


def _run_batch(solves, tol=0.0):
    b = mm.mm_batch_create()
    ids = [mm.mm_batch_add(b, p, t_end, N, K, tol, np.ascontiguousarray(w.rho0), _host_g0(p, w))
           for (p, w, t_end, N, K) in solves]
    steps = 0
    while mm.mm_batch_step(b) > 0:
        steps += 1
    outs, infos = [], []
    for (p, w, t_end, N, K), i in zip(solves, ids):
        assert mm.mm_batch_query(b, i)
        o = np.empty((N + 1, w.nx))
        infos.append(mm.mm_batch_take(b, i, o))
        outs.append(o)
    assert mm.mm_batch_bytes(b) == 0
    b.close()
    return outs, infos, steps


def test_batch_matches_single_solves_and_oracle():
    solves = _mixed_set()
    outs, infos, steps = _run_batch(solves)
    assert steps == max(K for *_, K in solves)
    for (p, w, t_end, N, K), o, info in zip(solves, outs, infos):
        tol = FP64_TOL if p.precision == mm.MM_FP64 else FP32_TOL
        single, sinfo = _single(p, w, t_end, N, K)
        assert info["iterations"] == sinfo["iterations"] == K
        assert rel(o, single) <= tol, (p.nx, p.nv, rel(o, single))
        ref, err, it = O.parareal(oparams(p), w.rho0, w.g0, t_end, N, K)
        assert it == K
        # slices 0 and 1 (one fine propagation of the given data) at the
        # parity tolerance; later slices too below eps = 1, while at eps = 1
        # relifting amplifies rounding from slice to slice (see gpu_helpers),
        # so they are held to 20 times the oracle's own one-ulp sensitivity
        assert rel(o[:2], ref[:2]) <= tol, (p.nx, p.nv, rel(o[:2], ref[:2]))
        bound = tol if p.eps < 1.0 else max(tol, 20 * _sensitivity(p, w, t_end, N, K, ref))
        assert rel(o, ref) <= bound, (p.nx, p.nv, rel(o, ref), bound)
        assert info["mass_drift"] <= 1e-12


def test_batch_result_independent_of_the_mix():
    """Each solve alone in a batch equals the same solve in the full mix,
    bitwise (continuous batching must not perturb results)."""
    solves = _mixed_set()
    mixed, _, _ = _run_batch(solves)
    for q, s in enumerate(solves):
        alone, _, _ = _run_batch([s])
        assert np.array_equal(alone[0], mixed[q]), q


def test_batch_admits_between_steps():
    """Solves added while others are in flight (continuous batching) give the
    results they give alone."""
    solves = _mixed_set()
    ref, _, _ = _run_batch(solves)
    b = mm.mm_batch_create()
    ids = {}
    pending = list(enumerate(solves))
    done = {}
    rounds = 0
    while pending or ids:
        if pending:  # one new solve per round
            q, (p, w, t_end, N, K) = pending.pop(0)
            ids[q] = mm.mm_batch_add(b, p, t_end, N, K, 0.0, np.ascontiguousarray(w.rho0), _host_g0(p, w))
        mm.mm_batch_step(b)
        rounds += 1
        for q in list(ids):
            if mm.mm_batch_query(b, ids[q]):
                p, w, t_end, N, K = solves[q]
                o = np.empty((N + 1, w.nx))
                mm.mm_batch_take(b, ids.pop(q), o)
                done[q] = o
        assert rounds < 100
    b.close()
    for q in range(len(solves)):
        assert np.array_equal(done[q], ref[q]), q


def test_batch_tolerance_stop_and_zero_iterations():
    (p, w, t_end, N, _), = [_mixed_set()[1]]
    _, err, _ = O.parareal(oparams(p), w.rho0, w.g0, t_end, N, 4)
    outs, infos, _ = _run_batch([(p, w, t_end, N, 4)], tol=err[1] * 1.0001)
    assert infos[0]["iterations"] == 2
    outs0, infos0, _ = _run_batch([(p, w, t_end, N, 0)])
    single, _ = _single(p, w, t_end, N, 0)
    assert infos0[0]["iterations"] == 0
    assert rel(outs0[0], single) <= FP64_TOL


def test_parareal_run_many_device_arrays():
    dev = device()
    solves = _mixed_set()[:3]
    ps = [s[0] for s in solves]
    cfgs = [(t_end, N, K, 0.0) for (_, _, t_end, N, K) in solves]
    r0 = [torch.tensor(w.rho0, device=dev) for (_, w, *_r) in solves]
    g0 = [torch.tensor(w.g0, device=dev, dtype=gdtype(p.precision)) for (p, w, *_r) in solves]
    outs = [torch.empty((N + 1, w.nx), dtype=torch.float64, device=dev) for (_, w, _, N, _) in solves]
    infos = mm.parareal_run_many(ps, cfgs, r0, g0, outs)
    ref, _, _ = _run_batch(solves)
    for q in range(3):
        assert np.array_equal(outs[q].cpu().numpy(), ref[q])
        assert infos[q]["iterations"] == solves[q][4]


def test_batch_rejects_bad_input():
    b = mm.mm_batch_create()
    p = params(64, 20, 1.0, mm.MM_FP32G)  # 10 nodes per half: no 8-node lanes
    with pytest.raises(mm.MMError) as e:
        mm.mm_batch_add(b, p, 0.01, 2, 1, 0.0, np.ones(64), np.zeros((64, 20), np.float32))
    assert e.value.status == mm.MM_ERR_INVALID
    with pytest.raises(mm.MMError):
        mm.mm_batch_add(b, params(64, 32, 1.0, mm.MM_FP64), 0.01, 0, 1, 0.0, np.ones(64), np.zeros((64, 32)))
    with pytest.raises(mm.MMError) as e:
        mm.mm_batch_take(b, 12345, None)
    assert e.value.status == mm.MM_ERR_UNKNOWN_TICKET
    b.close()


@pytest.mark.parametrize("eps,shapes", [
    (1e-2, [(8192, 256), (8192, 32), (128, 256)]),
    (5e-4, [(2048, 256), (2048, 32), (128, 256)]),
])
def test_batch_extreme_many_solve_shapes_match_oracle(eps, shapes):
    """The work-list kernel at the corners of the many-solve family (FP32 g,
    adaptation on with the hybrid thresholds on eps^2 |R|), three shapes in
    one batch, two slices of a few fine steps, one parareal iteration,
    against the oracle's Algorithm 1 (density within 1e-5, mass drift
    1e-12).  At eps = 1e-2 nearly every cell is kinetic, up to Nx = 8192
    and Nv = 256; at 5e-4 the masks are mixed (67-85% kinetic).  Mixed
    masks at Nx = 8192 are left to the FP64 path: there the remainder
    criterion amplifies float-g rounding past its threshold (see
    test_gpu_fine.py::test_fp64_nx8192_mixed_masks)."""
    solves = []
    for q, (nx, nv) in enumerate(shapes):
        w = W.batched(nx, nv, eps, seed=W.SEED_BASE + 101 * q, n_slices=2)
        p = params(nx, nv, eps, mm.MM_FP32G, rho_bar=1.0, adapt=1, thr_g=1e-3, thr_R=1e-2, r_scale=1)
        ctx = mm.mm_create(p)
        dt = mm.mm_query(ctx, 1.0)["dt_limit"]
        ctx.close()
        solves.append((p, w, 2 * 6 * dt * (1 - 1e-9), 2, 1))
    outs, infos, _ = _run_batch(solves)
    for (p, w, t_end, N, K), o, info in zip(solves, outs, infos):
        ref, _, it = O.parareal(oparams(p), w.rho0, w.g0, t_end, N, K)
        assert info["iterations"] == it == 1
        assert rel(o, ref) <= FP32_TOL, (p.nx, p.nv, rel(o, ref))
        assert info["mass_drift"] <= 1e-12


def test_batch_large_grid_sequential_parts_on_a_cluster():
    """A solve of Nx = 16384 in the batch engine: its coarse guess and
    corrections run over a thread-block cluster (chunks of 16 rows per
    thread), as in parareal_run; the result matches the single-solve run,
    and the oracle at 1e-12 or, where the implicit step's conditioning
    (about 2.5e4 here) makes a correct double-precision evaluation drift
    further, within twice the oracle's own change under one-ulp
    perturbations of rho0."""
    nx, nv, N, K = 16384, 16, 5, 2
    w = W.batched(nx, nv, 1e-2, seed=W.SEED_BASE + 77, n_slices=N)
    p = params(nx, nv, 1e-2, mm.MM_FP64, rho_bar=1.0)
    ctx = mm.mm_create(p)
    dt = mm.mm_query(ctx, 1.0)["dt_limit"]
    ctx.close()
    t_end = N * 3 * dt * (1 - 1e-9)
    outs, infos, _ = _run_batch([(p, w, t_end, N, K)])
    single, sinfo = _single(p, w, t_end, N, K)
    assert infos[0]["iterations"] == sinfo["iterations"] == K
    assert rel(outs[0], single) <= FP64_TOL, rel(outs[0], single)
    ref, _, it = O.parareal(oparams(p), w.rho0, w.g0, t_end, N, K)
    assert it == K
    bound = max(FP64_TOL, 2 * _sensitivity(p, w, t_end, N, K, ref))
    assert rel(outs[0], ref) <= bound, (rel(outs[0], ref), bound)
    assert infos[0]["mass_drift"] <= 1e-12


def test_batch_mid_size_grids_sequential_parts_on_a_cluster():
    """A batch that has the GPU to itself runs the coarse guess and the
    corrections of its solves of Nx >= 4096 over a thread-block cluster, one
    launch per grid size after the one-CTA launch of the smaller solves:
    every result matches its single-solve run (which takes the cluster
    layout at every supported grid), each mid-size solve is bitwise the same
    alone and in the mix, and the Nx = 4096 solve matches the oracle within
    the rounding spread of its implicit steps."""
    specs = [(4096, 16, 1e-2, 4, 2), (1024, 16, 1e-2, 5, 2), (8192, 16, 1e-1, 3, 2)]
    solves = []
    for q, (nx, nv, eps, N, K) in enumerate(specs):
        w = W.batched(nx, nv, eps, seed=W.SEED_BASE + 131 + q, n_slices=N)
        p = params(nx, nv, eps, mm.MM_FP64, rho_bar=1.0)
        ctx = mm.mm_create(p)
        dt = mm.mm_query(ctx, 1.0)["dt_limit"]
        ctx.close()
        solves.append((p, w, N * 2 * dt * (1 - 1e-9), N, K))
    outs, infos, _ = _run_batch(solves)
    for (p, w, t_end, N, K), o, info in zip(solves, outs, infos):
        single, sinfo = _single(p, w, t_end, N, K)
        assert info["iterations"] == sinfo["iterations"] == K
        assert rel(o, single) <= FP64_TOL, (p.nx, rel(o, single))
        assert info["mass_drift"] <= 1e-12
    for q in (0, 2):
        alone, _, _ = _run_batch([solves[q]])
        assert np.array_equal(alone[0], outs[q]), q
    p, w, t_end, N, K = solves[0]
    ref, _, it = O.parareal(oparams(p), w.rho0, w.g0, t_end, N, K)
    assert it == K
    bound = max(FP64_TOL, 2 * _sensitivity(p, w, t_end, N, K, ref))
    assert rel(outs[0], ref) <= bound, (rel(outs[0], ref), bound)


def test_batch_groups_large_solves_by_grid():
    """Large solves of two grid sizes beside a small one in one batch: the
    sequential parts run as one cluster launch per grid size (Nx = 16384,
    two solves; Nx = 32768, one) and one work-list launch for the small
    solve; every result matches its single-solve run, and each large solve
    is bitwise the same alone in a batch and in the mix."""
    specs = [(16384, 16, 1e-2, 4, 2), (256, 32, 1e-2, 5, 3), (32768, 16, 1e-1, 3, 2), (16384, 16, 1e-3, 3, 2)]
    solves = []
    for q, (nx, nv, eps, N, K) in enumerate(specs):
        w = W.batched(nx, nv, eps, seed=W.SEED_BASE + 91 + q, n_slices=N)
        p = params(nx, nv, eps, mm.MM_FP64, rho_bar=1.0)
        ctx = mm.mm_create(p)
        dt = mm.mm_query(ctx, 1.0)["dt_limit"]
        ctx.close()
        solves.append((p, w, N * 2 * dt * (1 - 1e-9), N, K))
    outs, infos, _ = _run_batch(solves)
    for (p, w, t_end, N, K), o, info in zip(solves, outs, infos):
        single, sinfo = _single(p, w, t_end, N, K)
        assert info["iterations"] == sinfo["iterations"] == K
        assert rel(o, single) <= FP64_TOL, (p.nx, rel(o, single))
    for q in (0, 2):
        alone, _, _ = _run_batch([solves[q]])
        assert np.array_equal(alone[0], outs[q]), q
