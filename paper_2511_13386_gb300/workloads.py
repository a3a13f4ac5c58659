"""Seeded synthetic workloads (initial data and problem sizes).

This module only generates inputs: grid sizes, Knudsen numbers, slice counts
and the initial density / perturbation sampled from closed-form initial
conditions.  It holds none of the scheme's arithmetic (no quadrature, no
discrete Maxwellian, no projection); the initial perturbations are sampled
with the continuous Gaussian exp(-v^2/2)/sqrt(2 pi), whose trapezoid moments
on these grids equal the continuous ones to ~1e-15, so <g0> vanishes to that
level.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) with the uniform mapping
u = (x >> 11) * 2^-53, so the draws are the same on every platform.

The initial conditions stand in for the paper's single far-from-equilibrium
initial condition (Sec. 5) and follow the five workload descriptions:
  small     Nx=64,   Nv=32,  eps=1,    rho0 = 1 + 0.5 cos(2 pi x), g0 = 0
  batched   Nx=1024, Nv=64,  eps=1e-2, random Fourier density + smooth
            random (v^2-1) M perturbation of amplitude 0.1 eps
  hybrid    Nx=4096, Nv=128 on [-10,10], eps=1e-3, localized bump
            0.5 (M(v-2) - M(v)) on x in [0.45, 0.55]
  many      2048 solves of random sizes, data as "batched"
  serving   Poisson arrivals of "many" solves plus 5% large solves
  paper     the paper's own setup (Sec. 5) reduced to 1D-1V: Nx=32, Nv=32 on
            [-8,8], torus length 2 pi, f = M(v) v^4 (1 + 0.9 cos x), which
            factorises in the passive velocities v_y, v_z
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

SEED_BASE = 2511133860
_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (64-bit state, golden-gamma increment)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, n: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(n)])

    def exponential(self, rate: float) -> float:
        return -math.log(1.0 - self.uniform()) / rate


def gaussian(v):
    """Continuous unit Gaussian exp(-v^2/2)/sqrt(2 pi) (initial data only)."""
    v = np.asarray(v, dtype=np.float64)
    return np.exp(-0.5 * v * v) / math.sqrt(2.0 * math.pi)


def velocity_nodes(nv: int, v_max: float) -> np.ndarray:
    """Velocity nodes on [-v_max, v_max] (both ends included)."""
    dv = 2.0 * v_max / (nv - 1)
    return (2.0 * np.arange(nv) - nv + 1) * (0.5 * dv)


def centres(nx: int, x_len: float = 1.0) -> np.ndarray:
    return (np.arange(nx) + 0.5) * (x_len / nx)


def interfaces(nx: int, x_len: float = 1.0) -> np.ndarray:
    """x_{i+1/2}, stored at index i."""
    return (np.arange(nx) + 1.0) * (x_len / nx)


@dataclass
class Workload:
    """One solve: problem parameters plus its initial data."""
    name: str
    nx: int
    nv: int
    eps: float
    v_max: float = 8.0
    x_len: float = 1.0
    t_end: float = 1.0
    n_slices: int = 1
    max_iter: int = 1
    adapt: bool = False
    thr_g: float = 1e-3
    thr_R: float = 1e-2
    r_scale: int = 0
    rho_bar: float = 1.0
    seed: int = SEED_BASE
    rho0: np.ndarray = field(default=None, repr=False)
    g0: np.ndarray = field(default=None, repr=False)

    @property
    def cells(self) -> int:
        return self.nx * self.nv

    def with_batch(self, batch: int):
        """Initial data replicated into a batch of slice states (each slice
        gets a different random Fourier content when the workload is random)."""
        rhos, gs = [], []
        for b in range(batch):
            w = random_state(self, self.seed + 7919 * (b + 1))
            rhos.append(w.rho0)
            gs.append(w.g0)
        return np.stack(rhos), np.stack(gs)


def _fourier_density(rng: SplitMix64, x, base_amp=0.2, kmax=8, amp=0.02):
    rho = 1.0 + base_amp * np.cos(2.0 * np.pi * x)
    for k in range(2, kmax + 1):
        u, up = rng.uniform(), rng.uniform()
        rho = rho + amp * u * np.cos(2.0 * np.pi * k * x + 2.0 * np.pi * up)
    return rho


def _smooth_field(rng: SplitMix64, x, amp=0.1, kmax=4):
    a = np.zeros_like(x)
    for k in range(1, kmax + 1):
        u, up = rng.uniform(), rng.uniform()
        a = a + (2.0 * u - 1.0) * k ** -2.0 * np.cos(2.0 * np.pi * k * x + 2.0 * np.pi * up)
    return amp * a / np.max(np.abs(a))


def small(nx: int = 64, nv: int = 32) -> Workload:
    """Plain method, full kinetic: rho0 = 1 + 0.5 cos(2 pi x), g0 = 0."""
    x = centres(nx)
    rho0 = 1.0 + 0.5 * np.cos(2.0 * np.pi * x)
    g0 = np.zeros((nx, nv))
    return Workload("small", nx, nv, eps=1.0, v_max=8.0, t_end=0.05, n_slices=4,
                    max_iter=4, rho0=rho0, g0=g0)


def batched(nx: int = 1024, nv: int = 64, eps: float = 1e-2, seed: int = SEED_BASE,
            n_slices: int = 128, v_max: float = 8.0) -> Workload:
    """Batched parareal, full kinetic: random Fourier density and a smooth
    random (v^2 - 1) M perturbation of amplitude 0.1 eps."""
    rng = SplitMix64(seed)
    rho0 = _fourier_density(rng, centres(nx))
    a = _smooth_field(rng, interfaces(nx))
    v = velocity_nodes(nv, v_max)
    g0 = eps * a[:, None] * ((v * v - 1.0) * gaussian(v))[None, :]
    return Workload("batched", nx, nv, eps=eps, v_max=v_max, t_end=1.0,
                    n_slices=n_slices, max_iter=8, seed=seed, rho0=rho0, g0=g0)


def hybrid(nx: int = 4096, nv: int = 128, eps: float = 1e-3, n_slices: int = 256,
           v_max: float = 10.0, lo: float = 0.45, hi: float = 0.55) -> Workload:
    """Hybrid domain adaptation: equilibrium background with rho = 1 and a
    localized non-equilibrium bump 0.5 (M(v-2) - M(v)) on x in [lo, hi]."""
    xf = interfaces(nx)
    v = velocity_nodes(nv, v_max)
    bump = (xf >= lo - 1e-12) & (xf <= hi + 1e-12)
    g0 = np.zeros((nx, nv))
    g0[bump, :] = 0.5 * (gaussian(v - 2.0) - gaussian(v))[None, :]
    rho0 = np.ones(nx)
    return Workload("hybrid", nx, nv, eps=eps, v_max=v_max, t_end=1.0,
                    n_slices=n_slices, max_iter=8, adapt=True, thr_g=1e-3,
                    thr_R=1e-2, r_scale=1, rho0=rho0, g0=g0)


def paper(eps: float, nx: int = 32, nv: int = 32, v_max: float = 8.0, n_slices: int = 200) -> Workload:
    """The far-from-equilibrium initial condition of Sec. 5,
    f(0, x, v) = M(v) v_x^4 (1 + 0.9 cos(2 pi x / x_len)) on a torus of
    length 2 pi, in its 1D-1V reduction (the factor M(v_y) M(v_z) is carried
    unchanged by the scheme).  With the continuous Gaussian's moment
    int v^4 M = 3: rho0 = 3 (1 + 0.9 cos x) at the centres and
    g0 = (v^4 - 3) M(v) (1 + 0.9 cos x) at the interfaces.  Thresholds
    1e-5 on both criteria (on eps^2 |R|, the scaling under which the
    paper's adaptation speedups at small eps are reachable), N = 200
    slices, T = 1.  On this
    coarse velocity grid (dv ~ 0.52) the trapezoid rule gives
    <v^4 M> = 3 to ~1e-11, so <g0> vanishes to that level, not 1e-15."""
    x_len = 2.0 * math.pi
    xc, xf = centres(nx, x_len), interfaces(nx, x_len)
    v = velocity_nodes(nv, v_max)
    rho0 = 3.0 * (1.0 + 0.9 * np.cos(2.0 * np.pi * xc / x_len))
    g0 = ((v ** 4 - 3.0) * gaussian(v))[None, :] * (1.0 + 0.9 * np.cos(2.0 * np.pi * xf / x_len))[:, None]
    return Workload("paper", nx, nv, eps=eps, v_max=v_max, x_len=x_len, t_end=1.0, n_slices=n_slices,
                    max_iter=n_slices, adapt=True, thr_g=1e-5, thr_R=1e-5, r_scale=1, rho_bar=3.0,
                    rho0=rho0, g0=g0)


def random_state(w: Workload, seed: int) -> Workload:
    """Another initial state of the same family (used to fill batches)."""
    if w.name == "batched":
        return batched(w.nx, w.nv, w.eps, seed=seed, n_slices=w.n_slices, v_max=w.v_max)
    if w.name == "small":
        rng = SplitMix64(seed)
        x = centres(w.nx)
        rho0 = _fourier_density(rng, x, base_amp=0.5, kmax=4, amp=0.05)
        a = _smooth_field(rng, interfaces(w.nx), amp=0.05)
        v = velocity_nodes(w.nv, w.v_max)
        g0 = a[:, None] * ((v * v - 1.0) * gaussian(v))[None, :]
        return replace(w, seed=seed, rho0=rho0, g0=g0)
    if w.name == "hybrid":
        rng = SplitMix64(seed)
        c = 0.3 + 0.4 * rng.uniform()
        half = 0.05
        out = hybrid(w.nx, w.nv, w.eps, w.n_slices, w.v_max, c - half, c + half)
        return replace(out, seed=seed)
    return replace(w, seed=seed)


POW2_NX = (128, 256, 512, 1024, 2048, 4096, 8192)
NV_CHOICES = (32, 64, 128, 256)


def many(n_solves: int = 2048, seed: int = SEED_BASE, lazy: bool = False) -> list[Workload]:
    """Many-solve batching: independent solves of random sizes (Nx a power of
    two in 128..8192, Nv in {32,64,128,256}, eps log-uniform in [1e-4, 1],
    N uniform in 16..256), data as 'batched', adaptation on.  With
    lazy=True the initial data is left empty (sizes only); materialise()
    fills it in."""
    rng = SplitMix64(seed)
    out = []
    for s in range(n_solves):
        nx = POW2_NX[int(rng.uniform() * len(POW2_NX))]
        nv = NV_CHOICES[int(rng.uniform() * len(NV_CHOICES))]
        eps = 10.0 ** (-4.0 * rng.uniform())
        n = 16 + int(rng.uniform() * 241)
        w = Workload("many", nx, nv, eps=eps, n_slices=n, max_iter=8, adapt=True, thr_g=1e-3,
                     thr_R=1e-2, r_scale=1, seed=seed + s)
        out.append(w if lazy else materialise(w))
    return out


@dataclass
class Arrival:
    t: float
    workload: Workload


def serving(rate: float = 200.0, duration: float = 60.0, large_frac: float = 0.05,
            seed: int = SEED_BASE, max_requests: int | None = None,
            lazy: bool = True) -> list[Arrival]:
    """Open-loop Poisson arrivals: 'many' solves plus a fraction of large
    solves (Nx=32768, Nv=256, N=512).  With lazy=True the initial data is
    left empty (sizes only); call materialise() on the arrivals needed."""
    rng = SplitMix64(seed ^ 0x5EED)
    t, out, s = 0.0, [], 0
    while True:
        t += rng.exponential(rate)
        if t >= duration or (max_requests is not None and len(out) >= max_requests):
            break
        if rng.uniform() < large_frac:
            nx, nv, n, eps = 32768, 256, 512, 10.0 ** (-4.0 * rng.uniform())
        else:
            nx = POW2_NX[int(rng.uniform() * len(POW2_NX))]
            nv = NV_CHOICES[int(rng.uniform() * len(NV_CHOICES))]
            eps = 10.0 ** (-4.0 * rng.uniform())
            n = 16 + int(rng.uniform() * 241)
        w = Workload("serving", nx, nv, eps=eps, n_slices=n, max_iter=8, adapt=True,
                     thr_g=1e-3, thr_R=1e-2, r_scale=1, seed=seed + s)
        if not lazy:
            w = materialise(w)
        out.append(Arrival(t, w))
        s += 1
    return out


def materialise(w: Workload) -> Workload:
    """Fill in the initial data of a size-only workload."""
    b = batched(w.nx, w.nv, w.eps, seed=w.seed, n_slices=w.n_slices, v_max=w.v_max)
    return replace(w, rho0=b.rho0, g0=b.g0)
