"""Algorithm 1 with the fine propagations spread over ranks
(paper_2511_13386_gb300.sharded), on CPU: two gloo ranks, with the building
blocks of Algorithm 1 taken from the oracle (F, G and the lifting) and the
correction written out from Algorithm 1.  The driver only splits the slices,
gathers the F results and repeats the correction on every rank, so the
two-rank result must be bitwise the one-rank result, and bitwise the
oracle's own Algorithm 1."""
import math
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2511_13386_gb300 import sharded as S  # noqa: E402


class OracleOps:
    """Algorithm 1's building blocks from the oracle, on CPU tensors."""

    def __init__(self, p, t_end, n_slices):
        import oracle as O
        self.O, self.p, self.N = O, p, n_slices
        self.span = t_end / n_slices
        lim = O.dt_limit(p)
        self.n = max(1, math.ceil(self.span / lim))
        self.dt = self.span / self.n

    def slices(self):
        return torch.zeros((self.N + 1, self.p.nx), dtype=torch.float64)

    def coarse_guess(self, rho, gprev):
        for n in range(self.N):
            g = torch.from_numpy(self.O.coarse(self.p, self.span, rho[n].numpy()))
            rho[n + 1] = g
            gprev[n + 1] = g

    def fine(self, rho_block, g0):
        out = []
        for q in range(rho_block.shape[0]):
            r = rho_block[q].numpy()
            g = np.asarray(g0, dtype=np.float64) if (q == 0 and g0 is not None) else self.O.lift(self.p, r)
            out.append(self.O.fine(self.p, self.n, self.dt, r, g)[0])
        return torch.from_numpy(np.stack(out))

    def correct(self, rho, frho, gprev, k):
        # rho^{n+1,k+1} = F(rho^{n,k}) + (G(rho^{n,k+1}) - G(rho^{n,k})), n = k..N-1 in order
        old = rho.clone()
        for n in range(k, self.N):
            gn = torch.from_numpy(self.O.coarse(self.p, self.span, rho[n].numpy()))
            rho[n + 1] = frho[n + 1] + (gn - gprev[n + 1])
            gprev[n + 1] = gn
        return float((rho - old).abs().max())


def _problem():
    import oracle as O
    from paper_2511_13386_gb300 import workloads as W
    w = W.batched(64, 16, 1e-2, n_slices=5)
    p = O.Params(nx=64, nv=16, eps=1e-2, rho_bar=1.0)
    t_end = 5 * 7 * O.dt_limit(p) * (1 - 1e-9)
    return w, p, t_end


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, K, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2511_13386_gb300 import sharded
    w, p, t_end = _problem()
    rho, errs = sharded.parareal_sharded(OracleOps(p, t_end, w.n_slices), torch.from_numpy(w.rho0), w.g0,
                                         w.n_slices, K, 0.0, comm=sharded.TorchComm())
    out[rank] = (rho.numpy().copy(), list(errs))
    td.destroy_process_group()


def test_block_split_covers_every_slice_once():
    for n0, n1 in [(0, 5), (2, 5), (4, 5), (0, 128), (7, 200), (3, 3)]:
        for world in (1, 2, 3, 4, 8):
            got = []
            for r in range(world):
                a, b = S.block(n0, n1, r, world)
                assert a <= b
                got += list(range(a, b))
            assert got == list(range(n0, n1))


@pytest.mark.parametrize("K", [2, 5])
def test_two_gloo_ranks_equal_one_rank_and_the_oracle(K):
    import oracle as O
    w, p, t_end = _problem()
    one, errs1 = S.parareal_sharded(OracleOps(p, t_end, w.n_slices), torch.from_numpy(w.rho0), w.g0,
                                    w.n_slices, K, 0.0)
    ref, err_ref, it = O.parareal(p, w.rho0, w.g0, t_end, w.n_slices, K)
    assert it == K == len(errs1)
    assert np.array_equal(one.numpy(), ref)
    assert errs1 == list(err_ref)
    world = 2
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.start_processes(_worker, args=(world, _free_port(), K, out), nprocs=world, join=True,
                        start_method="spawn")
    for r in range(world):
        assert np.array_equal(out[r][0], one.numpy()), r
        assert out[r][1] == errs1


def test_stops_on_tolerance_like_the_oracle():
    import oracle as O
    w, p, t_end = _problem()
    _, err, _ = O.parareal(p, w.rho0, w.g0, t_end, w.n_slices, 5)
    tol = err[1] * 1.0001
    rho, errs = S.parareal_sharded(OracleOps(p, t_end, w.n_slices), torch.from_numpy(w.rho0), w.g0,
                                   w.n_slices, 5, tol)
    ref, _, it = O.parareal(p, w.rho0, w.g0, t_end, w.n_slices, 5, tol=tol)
    assert len(errs) == it == 2
    assert np.array_equal(rho.numpy(), ref)
