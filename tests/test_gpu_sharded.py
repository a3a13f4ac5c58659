"""Algorithm 1 with the fine propagations spread over ranks
(paper_2511_13386_gb300.sharded) on the GPU through the C ABI
(mm_coarse_guess, mm_lift, mm_fine_propagate, mm_parareal_correct).  One
GPU: one rank, and two ranks emulated as two threads with their own
contexts that exchange the F results on the host (no kernel of one waits on
the other's).  Against parareal_run, which runs the same kernels in one
call."""
import threading

import numpy as np
import pytest

from paper_2511_13386_gb300 import mm, sharded as S, workloads as W
from tests.gpu_helpers import FP32_TOL, FP64_TOL, device, gdtype, params, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(prec, nx=256, nv=32, eps=1e-2, N=6, steps=20):
    w = W.batched(nx, nv, eps, n_slices=N)
    p = params(nx, nv, eps, prec, rho_bar=1.0)
    ctx = mm.mm_create(p)
    t_end = N * steps * mm.mm_query(ctx, 1.0)["dt_limit"] * (1 - 1e-9)
    ctx.close()
    return w, p, t_end


def _reference(p, w, t_end, K):
    dev = device()
    ctx = mm.mm_create(p)
    out = torch.empty((w.n_slices + 1, w.nx), dtype=torch.float64, device=dev)
    info = mm.parareal_run(ctx, t_end, w.n_slices, K, 0.0, torch.tensor(w.rho0, device=dev),
                           torch.tensor(w.g0, device=dev, dtype=gdtype(p.precision)), out)
    ctx.close()
    return out.cpu().numpy(), info


def _sharded(p, w, t_end, K, comm=None):
    dev = device()
    ctx = mm.mm_create(p)
    ops = S.LibOps(ctx, t_end, w.n_slices, dev)
    rho, errs = S.parareal_sharded(ops, torch.tensor(w.rho0, device=dev), w.g0, w.n_slices, K, 0.0, comm=comm)
    out = rho.cpu().numpy()
    ctx.close()
    return out, errs


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32G])
def test_one_rank_matches_parareal_run(prec):
    w, p, t_end = _setup(prec)
    ref, info = _reference(p, w, t_end, 3)
    got, errs = _sharded(p, w, t_end, 3)
    tol = FP64_TOL if prec == mm.MM_FP64 else FP32_TOL
    assert rel(got, ref) <= tol, rel(got, ref)
    assert np.allclose(errs, info["err"], rtol=1e-9, atol=1e-15)


def test_two_thread_ranks_equal_one_rank_bitwise():
    """FP64 (streaming kernel, one CTA per slice state): a slice's F does
    not depend on which slices share its launch, so two ranks give the
    one-rank result bit for bit, and both ranks hold the same iterate."""
    w, p, t_end = _setup(mm.MM_FP64, N=5)
    one, errs1 = _sharded(p, w, t_end, 4)
    tc = S.ThreadComm(2)
    res = [None, None]

    def run(r):
        res[r] = _sharded(p, w, t_end, 4, comm=tc.for_rank(r))

    th = [threading.Thread(target=run, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for r in range(2):
        assert np.array_equal(res[r][0], one), r
        assert res[r][1] == errs1


def test_parareal_correct_rejects_bad_arguments():
    dev = device()
    p = params(64, 16, 1e-2, mm.MM_FP64, rho_bar=1.0)
    ctx = mm.mm_create(p)
    a = torch.zeros((5, 64), dtype=torch.float64, device=dev)
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(mm.MMError) as e:
        mm.mm_parareal_correct(ctx, 4, 4, 0.01, a, a.clone(), a.clone(), err)   # k == N
    assert e.value.status == mm.MM_ERR_INVALID
    with pytest.raises(mm.MMError) as e:
        mm.mm_coarse_guess(ctx, 4, 0.01, np.zeros((5, 64)), a)                    # host array
    assert e.value.status == mm.MM_ERR_INVALID
    ctx.close()
