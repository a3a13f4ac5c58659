"""Shared helpers of the GPU parity tests: run the CUDA path through the C
ABI and the oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle as O
from paper_2511_13386_gb300 import mm

torch = pytest.importorskip("torch")

FP64_TOL = 1e-12   # relative, FP64 path vs oracle (max-norm)
FP32_TOL = 1e-5    # relative, FP32-g path vs oracle on the density


def device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def gdtype(prec):
    return torch.float64 if prec == mm.MM_FP64 else torch.float32


def params(nx, nv, eps, prec, **kw):
    return mm.mm_params_default(nx=nx, nv=nv, eps=eps, precision=prec, **kw)


def oparams(p: "mm.mm_params") -> O.Params:
    return O.Params(nx=p.nx, nv=p.nv, eps=p.eps, v_max=p.v_max, x_len=p.x_len,
                    rho_bar=p.rho_bar, adapt=bool(p.adapt), thr_g=p.thr_g, thr_R=p.thr_R,
                    r_scale=p.r_scale, flux_rule=p.flux_rule)


def run_fine(p, rho, g, t_span, mask=True):
    """CUDA F on a batch (numpy in, numpy out)."""
    dev = device()
    ctx = mm.mm_create(p)
    r = torch.tensor(rho, device=dev)
    gg = torch.tensor(g, device=dev, dtype=gdtype(p.precision))
    ro, go = torch.empty_like(r), torch.empty_like(gg)
    mo = torch.empty(r.shape, dtype=torch.uint8, device=dev) if mask else None
    st = mm.mm_fine_propagate(ctx, r.shape[0], t_span, r, gg, ro, go, mo, stats=True)
    q = mm.mm_query(ctx, t_span)
    ctx.close()
    return (ro.cpu().numpy(), go.double().cpu().numpy(),
            mo.cpu().numpy() if mask else None, st, q)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def parareal_with_sensitivity(op, w, K, tol=0.0, trials=2):
    """The oracle's parareal result and its own rounding sensitivity: the
    largest relative change of the result when rho0 is perturbed by one
    unit in the last place (random signs).  With the rho-only relifting of
    Algorithm 1, the lifted g carries the discrete gradient of rho, so at
    eps ~ 1 rounding-level differences grow from slice to slice; two
    correct implementations that round in a different order can differ by
    this much."""
    ref, err, it = O.parareal(op, w.rho0, w.g0, w.t_end, w.n_slices, K, tol=tol)
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(trials):
        r = w.rho0 * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=w.nx))
        out, _, _ = O.parareal(op, r, w.g0, w.t_end, w.n_slices, K, tol=tol)
        worst = max(worst, rel(out, ref))
    return ref, err, it, worst
