"""mm_fine_propagate_noalloc, the fine propagator for callers that cannot
allocate device memory when they run it (an application that has given all
of the GPU's memory to its own pool, a real-time loop that must not reach
the allocator).  It takes its scratch from a fixed device array inside the
library; its results must equal those of mm_fine_propagate, call after call,
since every call reuses (and must re-initialise) the same array, and it
runs the same kernel as mm_fine_propagate for the context.  Its calls must
leave the device's free memory unchanged.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2511_13386_gb300 import mm, workloads as W
from tests.gpu_helpers import FP32_TOL, FP64_TOL, device, gdtype, params, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pair(p, rho, g, span, in_place=False, tune_steps=0):
    """Reference call through mm_fine_propagate, then two no-alloc calls in
    a row through the C ABI; returns the three (rho, g, mask) results and
    the kernel launches each made."""
    dev = device()
    ctx = mm.mm_create(p)
    if tune_steps:
        r0 = torch.tensor(rho, device=dev)
        g0 = torch.tensor(g, device=dev, dtype=gdtype(p.precision))
        mm.mm_autotune(ctx, rho.shape[0], tune_steps, r0, g0, torch.empty_like(r0), torch.empty_like(g0))
    B = rho.shape[0]
    r = torch.tensor(rho, device=dev)
    gg = torch.tensor(g, device=dev, dtype=gdtype(p.precision))
    outs = []
    for k in range(3):
        ro = torch.empty_like(r)
        mo = torch.empty(r.shape, dtype=torch.uint8, device=dev)
        gi = gg.clone()
        go = gi if in_place else torch.empty_like(gg)
        if k == 0:
            st = mm.mm_fine_propagate(ctx, B, span, r, gi, ro, go, mo, stats=True)
        else:
            st = mm.mm_fine_propagate_noalloc(ctx, B, span, r, gi, ro, go, mo, stats=True)
        assert st["device_status"] == 0
        outs.append((ro.cpu().numpy(), go.double().cpu().numpy(), mo.cpu().numpy(),
                     st["kinetic_updates"], st["launches"]))
    ctx.close()
    return outs


def _agree(p, outs):
    tol = FP64_TOL if p.precision == mm.MM_FP64 else FP32_TOL
    r0, g0, m0, k0, n0 = outs[0]
    for r, g, m, k, n in outs[1:]:
        assert rel(r, r0) <= tol
        assert rel(g, g0) <= (10 * tol if p.precision == mm.MM_FP64 else 1e-3)
        assert np.array_equal(m, m0)
        assert k == k0 and n == n0


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32G])
def test_noalloc_matches_allocating_call_small(prec):
    """Nx=64, Nv=32, eps=1, 3 slice states (column arrays in shared memory)."""
    w = W.small()
    rho, g = w.with_batch(3)
    p = params(w.nx, w.nv, w.eps, prec, rho_bar=1.0)
    _agree(p, _pair(p, rho, g, w.t_end / w.n_slices))


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32G])
def test_noalloc_matches_allocating_call_hybrid_columns_in_scratch(prec):
    """Nx=4096 hybrid grid, Nv=16: the column arrays do not fit shared
    memory, so they too come from the fixed array; adaptation on."""
    w = W.hybrid(nx=4096, nv=16)
    rho, g = w.with_batch(2)
    p = params(w.nx, w.nv, w.eps, prec, v_max=w.v_max, adapt=1, thr_g=w.thr_g, thr_R=w.thr_R,
               r_scale=w.r_scale, rho_bar=1.0)
    ctx = mm.mm_create(p)
    dt = mm.mm_query(ctx, 1.0)["dt_limit"]
    ctx.close()
    _agree(p, _pair(p, rho, g, 9 * dt * (1 - 1e-9)))


@pytest.mark.parametrize("odd", [True, False])
def test_noalloc_in_place_g(odd):
    """g_out aliasing g_in, with an odd and an even step count."""
    w = W.small()
    rho, g = w.with_batch(2)
    p = params(w.nx, w.nv, w.eps, mm.MM_FP64, rho_bar=1.0)
    ctx = mm.mm_create(p)
    dt = mm.mm_query(ctx, 1.0)["dt_limit"]
    ctx.close()
    _agree(p, _pair(p, rho, g, (7 if odd else 6) * dt * (1 - 1e-9), in_place=True))


def test_noalloc_rejects_oversized_and_host_arrays():
    dev = device()
    # 160 states of Nx=1024, Nv=64 in FP64: 80 MiB of step buffer > 64 MiB
    p = params(1024, 64, 1e-2, mm.MM_FP64, rho_bar=1.0)
    ctx = mm.mm_create(p)
    B = 160
    r = torch.ones((B, 1024), dtype=torch.float64, device=dev)
    g = torch.zeros((B, 1024, 64), dtype=torch.float64, device=dev)
    assert g.numel() * 8 > mm.NOALLOC_SCRATCH_BYTES
    with pytest.raises(mm.MMError) as e:
        mm.mm_fine_propagate_noalloc(ctx, B, 1e-6, r, g, r.clone(), g.clone())
    assert e.value.status == mm.MM_ERR_INVALID
    assert "scratch" in str(e.value)
    # host arrays are refused (they would need staging buffers)
    rh = np.ones((1, 1024))
    gh = np.zeros((1, 1024, 64))
    with pytest.raises(mm.MMError) as e:
        mm.mm_fine_propagate_noalloc(ctx, 1, 1e-6, rh, gh, rh.copy(), gh.copy())
    assert e.value.status == mm.MM_ERR_INVALID
    ctx.close()


def test_noalloc_runs_the_resident_kernel_where_it_applies():
    """The batched workload's grid in FP32 (Nx=1024, Nv=64, eps=1e-2,
    adaptation off), a batch larger than the GPU holds at once: the context
    chooses the resident kernel, in rounds of step chunks, and the no-alloc
    call runs that same kernel, so its results are bitwise those of
    mm_fine_propagate."""
    w = W.batched()
    B = 160
    rho, g = w.with_batch(B)
    p = params(w.nx, w.nv, w.eps, mm.MM_FP32G, rho_bar=1.0)
    ctx = mm.mm_create(p)
    q = mm.mm_query(ctx, 1.0)
    ctx.close()
    assert q["fine_kernel"] == 2
    outs = _pair(p, rho, g, 40 * q["dt_limit"] * (1 - 1e-9))
    assert outs[0][4] > 1                     # rounds of step chunks
    r0, g0, m0, k0, n0 = outs[0]
    for r, gg, m, k, n in outs[1:]:
        assert np.array_equal(r, r0) and np.array_equal(gg, g0) and np.array_equal(m, m0)
        assert k == k0 and n == n0


def test_noalloc_follows_the_autotuned_choice():
    """After mm_autotune restricted to the streaming kernel with 4 nodes per
    lane (the context's default layout has 8), both entry points run the
    tuned layout: bitwise equal results."""
    w = W.small()
    rho, g = w.with_batch(3)
    p = params(w.nx, w.nv, w.eps, mm.MM_FP32G, rho_bar=1.0)
    p.fine_kernel = 1
    p.fine_vpt = 4
    outs = _pair(p, rho, g, w.t_end / w.n_slices, tune_steps=4)
    r0, g0, m0, _, _ = outs[0]
    for r, gg, m, _, _ in outs[1:]:
        assert np.array_equal(r, r0) and np.array_equal(gg, g0) and np.array_equal(m, m0)


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32G])
def test_noalloc_calls_leave_device_memory_unchanged(prec):
    """A fresh context: once mm_create has returned (it reserves the fixed
    array and loads the kernels), the first and the later no-alloc calls
    allocate nothing on the device, whether the context runs the streaming
    kernel (FP64) or the resident kernel (FP32)."""
    dev = device()
    w = W.batched(nx=1024, nv=64)
    rho, g = w.with_batch(4)
    p = params(w.nx, w.nv, w.eps, prec, rho_bar=1.0)
    r = torch.tensor(rho, device=dev)
    gi = torch.tensor(g, device=dev, dtype=gdtype(prec))
    ro, go = torch.empty_like(r), torch.empty_like(gi)
    mo = torch.empty(r.shape, dtype=torch.uint8, device=dev)
    ctx = mm.mm_create(p)
    span = 5 * mm.mm_query(ctx, 1.0)["dt_limit"] * (1 - 1e-9)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        st = mm.mm_fine_propagate_noalloc(ctx, 4, span, r, gi, ro, go, mo, stats=True)
        assert st["device_status"] == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ctx.close()
