"""Serving with continuous batching (mm_server_create / serve_submit /
serve_poll): every result equals the same solve run alone, whatever it was
batched with; admission respects the HBM budget; failures are reported per
request."""
import time

import numpy as np
import pytest

from paper_2511_13386_gb300 import mm, workloads as W
from tests.gpu_helpers import device
from tests.test_gpu_batch import _host_g0, _mixed_set, _run_batch

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _footprint(p, t_end, N, K):
    gsz = 4 if p.precision == mm.MM_FP32G else 8
    n_sm = torch.cuda.get_device_properties(device()).multi_processor_count
    return mm.mm_batch_footprint(p, t_end, N, K, 0.0) + 2 * p.nx * p.nv * gsz * n_sm + (1 << 20)


def _serve(solves, budget, slots, stagger_s=0.0):
    srv = mm.mm_server_create(budget, slots, wait_limit_ms=60000)
    tickets = []
    for (p, w, t_end, N, K) in solves:
        tickets.append(mm.serve_submit(srv, p, t_end, N, K, 0.0, np.ascontiguousarray(w.rho0), _host_g0(p, w)))
        if stagger_s:
            time.sleep(stagger_s)
    res = []
    for t, (p, w, *_r) in zip(tickets, solves):
        r = mm.serve_poll(srv, t, w.nx, timeout_ms=60000)
        assert r is not None
        res.append(r)
    srv.close()
    return res


def test_serving_results_equal_solo_runs():
    solves = _mixed_set()
    solo = [_run_batch([s])[0][0][-1] for s in solves]
    for stagger in (0.0, 0.002):
        res = _serve(solves, budget=1 << 40, slots=64, stagger_s=stagger)
        for q, r in enumerate(res):
            assert r["status"] == mm.MM_OK
            assert r["iterations"] == solves[q][4]
            assert r["latency_ns"] > 0
            assert np.array_equal(r["rho_T"], solo[q]), q


def test_serving_budget_serialises_admission():
    solves = _mixed_set()[:4]
    biggest = max(_footprint(p, t, N, K) for (p, w, t, N, K) in solves)
    res = _serve(solves, budget=biggest, slots=64)  # one resident solve at a time
    solo = [_run_batch([s])[0][0][-1] for s in solves]
    for q, r in enumerate(res):
        assert r["status"] == mm.MM_OK
        assert np.array_equal(r["rho_T"], solo[q])
    res1 = _serve(solves, budget=1 << 40, slots=1)  # one slot
    for q, r in enumerate(res1):
        assert np.array_equal(r["rho_T"], solo[q])


def test_serving_rejections_and_per_request_failures():
    (p, w, t_end, N, K) = _mixed_set()[0]
    srv = mm.mm_server_create(_footprint(p, t_end, N, K) - 1, 4)
    with pytest.raises(mm.MMError) as e:  # above the whole budget
        mm.serve_submit(srv, p, t_end, N, K, 0.0, np.ascontiguousarray(w.rho0), _host_g0(p, w))
    assert e.value.status == mm.MM_ERR_INVALID
    with pytest.raises(mm.MMError) as e:
        mm.serve_poll(srv, 999, w.nx)
    assert e.value.status == mm.MM_ERR_UNKNOWN_TICKET
    srv.close()
    # a request the batch refuses (no 8-node lanes) fails alone; the other completes
    srv = mm.mm_server_create(1 << 40, 4)
    bad = mm.mm_params_default(nx=64, nv=20, eps=1.0, precision=mm.MM_FP32G, rho_bar=1.0)
    tb = mm.serve_submit(srv, bad, 0.01, 2, 1, 0.0, np.ones(64), np.zeros((64, 20), np.float32))
    tg = mm.serve_submit(srv, p, t_end, N, K, 0.0, np.ascontiguousarray(w.rho0), _host_g0(p, w))
    rb = mm.serve_poll(srv, tb, 64, timeout_ms=60000)
    rg = mm.serve_poll(srv, tg, w.nx, timeout_ms=60000)
    srv.close()
    assert rb["status"] == mm.MM_ERR_INVALID
    assert rg["status"] == mm.MM_OK
    assert np.array_equal(rg["rho_T"], _run_batch([(p, w, t_end, N, K)])[0][0][-1])


def _long_request():
    """A solve whose parareal iteration costs ~2.7e10 fine cell-updates
    (above the server's long-lane threshold of 2e10): Nx=2048, Nv=64,
    N=32 slices of 6,400 steps, FP32, one iteration."""
    nx, nv, N = 2048, 64, 32
    w = W.batched(nx, nv, 1e-2, seed=W.SEED_BASE + 977, n_slices=N)
    p = mm.mm_params_default(nx=nx, nv=nv, eps=1e-2, precision=mm.MM_FP32G, rho_bar=1.0)
    ctx = mm.mm_create(p)
    dt = mm.mm_query(ctx, 1.0)["dt_limit"]
    ctx.close()
    return (p, w, N * 6400 * dt * (1 - 1e-9), N, 1)


def test_short_requests_do_not_wait_behind_a_long_one():
    """Two lanes: the long request (submitted first) runs on most of the
    SMs while the short ones run beside it on the SMs kept for them, so all
    short requests complete before the long one; every result equals its
    solo run."""
    device()
    long_req = _long_request()
    shorts = _mixed_set()
    solves = [long_req] + shorts
    res = _serve(solves, budget=1 << 40, slots=64)
    assert all(r["status"] == mm.MM_OK for r in res)
    lat = [r["latency_ns"] for r in res]
    assert max(lat[1:]) < lat[0], lat
    solo = [_run_batch([s])[0][0][-1] for s in solves]
    for q, r in enumerate(res):
        assert np.array_equal(r["rho_T"], solo[q]), q


def test_serving_refused_allocation_fails_alone():
    """Device memory comes from the caller's allocator (here torch's caching
    allocator behind a wrapper that refuses every request of one size, the
    slice arrays of one marked solve: Nx=64, N=13, (N+1) x 64 doubles =
    7,168 bytes).  The marked request fails alone with MM_ERR_OOM; every
    other request of the mix completes with its solo result, bit for bit."""
    device()
    base = mm.torch_allocator()
    refused = []

    def alloc(n, stream):
        if n == 14 * 64 * 8:
            refused.append(n)
            return 0
        return base._alloc(n, stream)

    picky = mm.Allocator(alloc, base._free)
    nx, nv, N = 64, 32, 13
    wm = W.batched(nx, nv, 1e-1, seed=W.SEED_BASE + 4242, n_slices=N)
    pm = mm.mm_params_default(nx=nx, nv=nv, eps=1e-1, precision=mm.MM_FP32G, rho_bar=1.0)
    ctx = mm.mm_create(pm)
    t_m = N * 5 * mm.mm_query(ctx, 1.0)["dt_limit"] * (1 - 1e-9)
    ctx.close()
    solves = _mixed_set()
    solves.insert(2, (pm, wm, t_m, N, 2))
    srv = mm.mm_server_create(1 << 40, 64, wait_limit_ms=60000, alloc=picky)
    tickets = [mm.serve_submit(srv, p, t, n, k, 0.0, np.ascontiguousarray(w.rho0), _host_g0(p, w))
               for (p, w, t, n, k) in solves]
    res = [mm.serve_poll(srv, tk, w.nx, timeout_ms=60000) for tk, (p, w, *_r) in zip(tickets, solves)]
    srv.close()
    assert refused
    for q, r in enumerate(res):
        if q == 2:
            assert r["status"] == mm.MM_ERR_OOM
            continue
        assert r["status"] == mm.MM_OK, q
        assert np.array_equal(r["rho_T"], _run_batch([solves[q]])[0][0][-1]), q
