"""The seeded synthetic inputs against their stated recipe: the generator's
published reference outputs, the initial data of each workload family, and
the size distributions of the many-solve and serving families."""
import math

import numpy as np

from paper_2511_13386_gb300 import workloads as W


def test_splitmix64_reference_outputs():
    """SplitMix64 (Steele, Lea, Flood 2014) reference outputs for seeds 0 and
    1234567, and the 53-bit uniform mapping (x >> 11) 2^-53."""
    r = W.SplitMix64(0)
    assert [r.next_u64() for _ in range(4)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    r = W.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973,
                                                 9817491932198370423]
    r, q = W.SplitMix64(99), W.SplitMix64(99)
    for _ in range(100):
        u = r.uniform()
        assert 0.0 <= u < 1.0
        assert u == (q.next_u64() >> 11) * 2.0 ** -53


def test_small_workload():
    w = W.small()
    x = (np.arange(64) + 0.5) / 64
    assert np.array_equal(w.rho0, 1.0 + 0.5 * np.cos(2 * np.pi * x))
    assert not w.g0.any()
    assert (w.nx, w.nv, w.eps, w.t_end, w.n_slices, w.max_iter) == (64, 32, 1.0, 0.05, 4, 4)


def test_batched_workload_recipe():
    w = W.batched()
    assert (w.nx, w.nv, w.eps, w.n_slices) == (1024, 64, 1e-2, 128)
    # rho0 = 1 + 0.2 cos 2 pi x + sum_{k=2..8} 0.02 u_k cos(2 pi k x + phase): mean 1
    # over the period, the first harmonic of amplitude 0.2
    x = (np.arange(1024) + 0.5) / 1024
    assert abs(w.rho0.mean() - 1.0) < 1e-14
    c1 = 2 * np.mean((w.rho0 - 1.0) * np.cos(2 * np.pi * x))
    s1 = 2 * np.mean((w.rho0 - 1.0) * np.sin(2 * np.pi * x))
    assert abs(c1 - 0.2) < 1e-12 and abs(s1) < 1e-12
    assert np.abs(w.rho0 - 1.0).max() <= 0.2 + 7 * 0.02
    # g0 = eps a(x) (v^2 - 1) M(v) with max |a| = 0.1: rank one, that v-profile
    v = W.velocity_nodes(64, 8.0)
    prof = (v * v - 1.0) * W.gaussian(v)
    a = w.g0 @ prof / (prof @ prof) / w.eps
    assert np.allclose(w.g0, w.eps * np.outer(a, prof), rtol=0, atol=1e-15)
    assert abs(np.abs(a).max() - 0.1) < 1e-12
    # deterministic per seed; a batch holds distinct states
    assert np.array_equal(W.batched().rho0, w.rho0)
    assert not np.array_equal(W.batched(seed=W.SEED_BASE + 1).rho0, w.rho0)
    rb, gb = w.with_batch(3)
    assert rb.shape == (3, 1024) and gb.shape == (3, 1024, 64)
    assert not np.array_equal(rb[0], rb[1]) and not np.array_equal(rb[1], rb[2])


def test_hybrid_workload_recipe():
    w = W.hybrid()
    assert (w.nx, w.nv, w.eps, w.v_max, w.n_slices) == (4096, 128, 1e-3, 10.0, 256)
    assert w.adapt and (w.thr_g, w.thr_R, w.r_scale) == (1e-3, 1e-2, 1)
    assert np.array_equal(w.rho0, np.ones(4096))
    xf = (np.arange(4096) + 1.0) / 4096
    inside = (xf >= 0.45 - 1e-12) & (xf <= 0.55 + 1e-12)
    v = W.velocity_nodes(128, 10.0)
    bump = 0.5 * (W.gaussian(v - 2.0) - W.gaussian(v))
    assert np.array_equal(w.g0[inside], np.broadcast_to(bump, (int(inside.sum()), 128)))
    assert not w.g0[~inside].any()
    assert 0.09 < inside.mean() < 0.11


def test_many_solve_size_distribution():
    ws = W.many(2048, lazy=True)
    assert len(ws) == 2048
    nx = np.array([w.nx for w in ws])
    nv = np.array([w.nv for w in ws])
    eps = np.array([w.eps for w in ws])
    n = np.array([w.n_slices for w in ws])
    assert set(nx) == {128, 256, 512, 1024, 2048, 4096, 8192}
    assert set(nv) == {32, 64, 128, 256}
    assert eps.min() >= 1e-4 and eps.max() <= 1.0
    # log-uniform eps: the decades are about equally filled
    dec = np.histogram(np.log10(eps), bins=4, range=(-4, 0))[0]
    assert dec.min() > 0.8 * 2048 / 4
    assert n.min() >= 16 and n.max() <= 256
    assert all(w.adapt and w.r_scale == 1 for w in ws)
    assert len({w.seed for w in ws}) == 2048


def test_serving_arrivals():
    arr = W.serving(rate=200.0, duration=60.0)
    n = len(arr)
    # Poisson arrivals at 200/s for 60 s: 12,000 +- a few sigma (sqrt(12000) ~ 110)
    assert abs(n - 12000) < 5 * math.sqrt(12000)
    t = np.array([a.t for a in arr])
    assert np.all(np.diff(t) > 0) and t[-1] < 60.0
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200) < 5 * (1 / 200) / math.sqrt(n)
    large = np.array([a.workload.nx == 32768 for a in arr])
    assert abs(large.mean() - 0.05) < 5 * math.sqrt(0.05 * 0.95 / n)
    big = [a.workload for a in arr if a.workload.nx == 32768]
    assert all(w.nv == 256 and w.n_slices == 512 for w in big)
