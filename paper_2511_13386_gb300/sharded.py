"""Algorithm 1 (Sec. 3.3) with the fine propagations of each iteration
spread over several ranks: the parallel loop over slices run on distributed
memory, which the paper's conclusion (Sec. 6) leaves for future work.

At iteration k, rank r of W runs F on a contiguous block of the slices
n = k..N-1 (`block`); one all-gather gives every rank F(rho^{n,k}) for every
n; every rank then runs the same sequential correction and takes the same
stopping decision, so all ranks hold the same iterate.  The only data-path
collective is that all-gather of N x nx doubles per iteration.

This module only orders the calls.  The arithmetic runs in an `ops` object:
`LibOps` calls libmm's kernels through the C ABI (mm_coarse_guess, mm_lift,
mm_fine_propagate, mm_parareal_correct) on the rank's GPU; the CPU tests
pass an object built on the oracle.  A fine propagation of one slice does
not depend on which other slices share its launch (one CTA, or one cluster,
per slice state), so with the streaming kernel the result is bitwise the
same for every number of ranks.
"""
from __future__ import annotations

import threading


def block(n0: int, n1: int, rank: int, world: int) -> tuple[int, int]:
    """Rank `rank`'s contiguous share of the slices n0..n1-1: the first
    (n1 - n0) mod world ranks take one slice more."""
    n = max(n1 - n0, 0)
    q, r = divmod(n, world)
    lo = n0 + rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


class LocalComm:
    """One rank, no exchange."""
    rank, world = 0, 1

    def allgather(self, t):
        return [t]


class TorchComm:
    """torch.distributed (NCCL between GPUs, gloo on CPU)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def allgather(self, t):
        out = [t.new_empty(t.shape) for _ in range(self.world)]
        self.dist.all_gather(out, t.contiguous(), group=self.group)
        return out


class ThreadComm:
    """Ranks as threads of one process (one per context), exchanging through
    shared slots at a barrier; lets one device run several ranks' calls
    without any of their kernels waiting on another."""

    def __init__(self, world: int):
        self.world = world
        self._slots = [None] * world
        self._bar = threading.Barrier(world)

    def for_rank(self, rank: int):
        parent = self

        class _R:
            def __init__(self):
                self.rank, self.world = rank, parent.world

            def allgather(self, t):
                parent._slots[rank] = t.clone()
                parent._bar.wait()
                out = list(parent._slots)
                parent._bar.wait()
                return out
        return _R()


def parareal_sharded(ops, rho0, g0, n_slices: int, max_iter: int, tol: float, comm=None):
    """Algorithm 1 in density mode (the lifting of each slice density, slice
    0 from g0) with F spread over the ranks of `comm`.  Returns
    (rho_slices [N+1][nx], successive errors).  `ops` provides slices()
    (a zeroed [N+1][nx] array), coarse_guess(rho, gprev), fine(rho_block,
    g0_or_None) -> F of the block, correct(rho, frho, gprev, k) -> error."""
    comm = comm or LocalComm()
    N = n_slices
    rho, gprev, frho = ops.slices(), ops.slices(), ops.slices()
    rho[0] = rho0
    ops.coarse_guess(rho, gprev)
    errs = []
    for k in range(min(max_iter, N)):
        lo, hi = block(k, N, comm.rank, comm.world)
        width = -(-(N - k) // comm.world)        # padded block of the exchange
        mine = ops.slices()[:width]
        if hi > lo:
            mine[:hi - lo] = ops.fine(rho[lo:hi], g0 if lo == 0 else None)
        for r, part in enumerate(comm.allgather(mine)):
            a, b = block(k, N, r, comm.world)
            frho[a + 1:b + 1] = part[:b - a]
        err = ops.correct(rho, frho, gprev, k)
        errs.append(err)
        if err < tol:
            break
    return rho, errs


class LibOps:
    """The building blocks of Algorithm 1 on one GPU through libmm.  The
    context's params.rho_bar must be set (not NaN) so that every rank uses
    the same neutralising density."""

    def __init__(self, ctx, t_end: float, n_slices: int, device, stream=None):
        import math

        import torch

        from . import mm
        if math.isnan(ctx.params.rho_bar):
            raise ValueError("LibOps needs params.rho_bar set")
        self.mm, self.torch, self.ctx, self.dev = mm, torch, ctx, device
        self.N, self.span = n_slices, t_end / n_slices
        self.nx, self.nv = ctx.params.nx, ctx.params.nv
        self.gdt = torch.float32 if ctx.params.precision == mm.MM_FP32G else torch.float64
        self.stream = stream
        self._err = torch.zeros(1, dtype=torch.float64, device=device)

    def slices(self):
        return self.torch.zeros((self.N + 1, self.nx), dtype=self.torch.float64, device=self.dev)

    def coarse_guess(self, rho, gprev):
        self.mm.mm_coarse_guess(self.ctx, self.N, self.span, rho, gprev, stream=self.stream)

    def fine(self, rho_block, g0):
        torch = self.torch
        b = rho_block.shape[0]
        g = torch.empty((b, self.nx, self.nv), dtype=self.gdt, device=self.dev)
        if g0 is not None:
            g[0] = torch.as_tensor(g0, device=self.dev, dtype=self.gdt)
            if b > 1:
                self.mm.mm_lift(self.ctx, b - 1, rho_block[1:].contiguous(), g[1:], stream=self.stream)
        else:
            self.mm.mm_lift(self.ctx, b, rho_block.contiguous(), g, stream=self.stream)
        out = torch.empty((b, self.nx), dtype=torch.float64, device=self.dev)
        self.mm.mm_fine_propagate(self.ctx, b, self.span, rho_block.contiguous(), g, out, g,
                                  stream=self.stream)
        return out

    def correct(self, rho, frho, gprev, k):
        self.mm.mm_parareal_correct(self.ctx, self.N, k, self.span, rho, frho, gprev, self._err,
                                    stream=self.stream)
        return float(self._err.item())
