"""Pins of the oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: printed
values (Table 1), closed forms, invariants, special cases that reduce to a
textbook result, exact-rational brute force on tiny grids, and the paper's
own statements (Lemma 1, the AP limit of Sec. 1 / 2.3, parareal exactness).
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest
import sympy as sp

import oracle as O
from paper_2511_13386_gb300 import workloads as W
from tests import rational_scheme as RS


def P(**kw):
    base = dict(nx=32, nv=16, eps=1.0)
    base.update(kw)
    return O.Params(**base)


# ------------------------------------------------------------- Table 1 ---

def test_table1_matches_printed_values():
    T = RS.table1()
    for d in range(1, 5):
        got = O.fd_coefficients(d)
        want = np.array([float(c) for c in T[d]])
        assert np.array_equal(got, want), d


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_table1_polynomial_moments(d):
    """Row d differentiates x^p exactly for p <= 6: sum_k c_k k^p = d! [p==d]."""
    c = RS.table1()[d]
    for p in range(0, 7):
        s = sum(ck * Fr(k) ** p for ck, k in zip(c, range(-3, 4)))
        assert s == (math.factorial(d) if p == d else 0), (d, p, s)


@pytest.mark.parametrize("d,order", [(1, 6), (2, 6), (3, 4), (4, 4)])
def test_fd_derivative_convergence_order(d, order):
    """Periodic derivative of sin(2 pi x): error falls like dx^order."""
    errs = []
    for nx in (32, 64):
        x = (np.arange(nx) + 0.5) / nx
        f = np.sin(2 * np.pi * x)
        exact = (2 * np.pi) ** d * np.sin(2 * np.pi * x + d * np.pi / 2)
        errs.append(np.abs(O.fd_derivative(f, 1.0 / nx, d) - exact).max())
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.3, (errs, rate)


# --------------------------------------------------------- velocity grid -

def test_velocity_grid_symmetric_and_normalised():
    p = P(nv=32, v_max=8.0)
    v, w, M, m2 = O.velocity_grid(p)
    assert np.array_equal(v, -v[::-1])
    assert v[0] == -8.0 and v[-1] == 8.0
    assert abs(np.sum(w * M) - 1.0) < 1e-15
    assert np.sum(w) == pytest.approx(16.0, rel=1e-15)
    # Gaussian shape: M_j / M_k = exp(-(v_j^2 - v_k^2) / 2)
    mid = len(v) // 2
    assert np.allclose(M / M[mid], np.exp(-0.5 * (v * v - v[mid] ** 2)), rtol=1e-14)
    # trapezoid moment of the Gaussian on [-8, 8]: m2 = 1 up to truncation
    assert abs(m2 - 1.0) < 1e-12
    assert abs(np.sum(w * v * M)) < 1e-16


# -------------------------------------------------------------- Poisson --

@pytest.mark.parametrize("nx,m", [(64, 1), (64, 3), (100, 2)])
def test_poisson_closed_form(nx, m):
    """rho = rho_bar + A cos(2 pi m x_i): E_{i+1/2} = A dx sin(2 pi m (i+1) dx)
    / (2 sin(pi m dx)) (telescoping sine identity), mean zero."""
    A, dx = 0.3, 1.0 / nx
    x = (np.arange(nx) + 0.5) * dx
    p = P(nx=nx, rho_bar=1.0)
    E = O.poisson(p, 1.0 + A * np.cos(2 * np.pi * m * x))
    th = 2 * np.pi * m * dx
    want = A * dx * np.sin(th * (np.arange(nx) + 1)) / (2 * np.sin(th / 2))
    assert np.abs(E - want).max() < 1e-15


def test_poisson_constant_density_gives_zero_field():
    p = P(nx=48, rho_bar=1.25)
    assert np.array_equal(O.poisson(p, np.full(48, 1.25)), np.zeros(48))


def test_flux_J_closed_form():
    """J_{i+1/2} for a cosine density, from the sum/difference formulas."""
    nx, A, m = 64, 0.2, 2
    dx = 1.0 / nx
    x = (np.arange(nx) + 0.5) * dx
    p = P(nx=nx)
    rho = 1.0 + A * np.cos(2 * np.pi * m * x)
    J = O.flux_J(p, rho, O.poisson(p, rho))
    th, k = 2 * np.pi * m * dx, np.arange(nx) + 1
    E = A * dx * np.sin(th * k) / (2 * np.sin(th / 2))
    want = -2 * A * np.sin(th * k) * np.sin(th / 2) / dx - E * (1.0 + A * np.cos(th * k) * np.cos(th / 2))
    assert np.abs(J - want).max() < 1e-12


# ------------------------------------------------------------ remainder --

def test_remainder_constant_density_is_zero():
    p = P(nx=40)
    rho = np.ones(40)
    # the stencil rows sum to zero; only their rounding residue remains
    assert np.abs(O.remainder(p, rho, O.poisson(p, rho))).max() < 1e-9


def test_remainder_converges_to_continuous_formula():
    """eq. Remainder evaluated analytically (sympy) on a two-mode density,
    with d_t E = J - mean(J): the discrete R converges (second order, set by
    the centred E) and a wrong sign or coefficient would not."""
    xs = sp.symbols("x")
    A, B, rb = sp.Rational(1, 5), sp.Rational(1, 10), 1
    rho = rb + A * sp.cos(2 * sp.pi * xs) + B * sp.sin(4 * sp.pi * xs)
    E = A * sp.sin(2 * sp.pi * xs) / (2 * sp.pi) - B * sp.cos(4 * sp.pi * xs) / (4 * sp.pi)
    J = sp.diff(rho, xs) - E * rho
    meanJ = sp.integrate(J, (xs, 0, 1))
    R = (-sp.diff(J, xs, 3) + E * sp.diff(J, xs, 2) + (2 * rho - 3 * rb) * sp.diff(J, xs)
         + 2 * J * sp.diff(rho, xs) - sp.diff(rho, xs) * (J - meanJ))
    Rf = sp.lambdify(xs, R, "numpy")
    rf = sp.lambdify(xs, rho, "numpy")
    errs = []
    for nx in (64, 128, 256):
        x = (np.arange(nx) + 0.5) / nx
        p = P(nx=nx, rho_bar=1.0)
        r = rf(x)
        Rd = O.remainder(p, r, O.poisson(p, r))
        errs.append(np.abs(Rd - Rf(x)).max() / np.abs(Rf(x)).max())
    assert errs[-1] < 2e-3
    assert math.log2(errs[0] / errs[1]) > 1.8 and math.log2(errs[1] / errs[2]) > 1.8


# ------------------------------------------------------------- status ----

def test_status_rule_transitions():
    """Sec. 2.3 rule: K->F only when both interface norms and |R| are small;
    the mixed norm case stays kinetic; F->K when |R| is large."""
    nx, nv = 8, 4
    p = P(nx=nx, nv=nv, adapt=True, thr_g=1e-3, thr_R=1e-2)
    rho = np.ones(nx)
    g = np.zeros((nx, nv))
    g[2, :] = [1e-2, -1e-2, 1e-2, -1e-2]      # interface 2+1/2 far from equilibrium
    mask = np.array([1, 1, 1, 1, 0, 0, 1, 0], dtype=np.uint8)
    out = O.update_status(p, rho, g, mask)
    # cells 2 and 3 touch interface 2+1/2 (mixed or both large) -> stay kinetic
    # cells 0,1,6 have both norms zero and R = 0 -> become fluid
    assert out.tolist() == [0, 0, 1, 1, 0, 0, 0, 0]
    # a non-constant density with a tiny threshold turns fluid cells kinetic
    x = (np.arange(nx) + 0.5) / nx
    p2 = P(nx=nx, nv=nv, adapt=True, thr_g=1e-3, thr_R=1e-12)
    out2 = O.update_status(p2, 1.0 + 0.1 * np.cos(2 * np.pi * x), g, np.zeros(nx, np.uint8))
    assert out2.tolist() == [1] * nx


def test_initial_status_adapt_off_is_all_kinetic():
    p = P(nx=16, nv=8, adapt=False)
    assert O.initial_status(p, np.ones(16), np.zeros((16, 8))).tolist() == [1] * 16


# --------------------------------------------------------- fine scheme ---

def test_global_equilibrium_fixed_bitwise():
    for adapt in (False, True):
        p = P(nx=32, nv=16, eps=0.1, adapt=adapt, rho_bar=1.0)
        rho, g = np.ones(32), np.zeros((32, 16))
        r2, g2, _, _ = O.fine(p, 25, 1e-4, rho, g)
        assert np.array_equal(r2, rho) and np.array_equal(g2, g)
        # the linear solve of the implicit G reproduces it to rounding only
        assert np.abs(O.coarse(p, 0.01, rho) - rho).max() <= 4 * np.finfo(float).eps
        assert np.array_equal(O.coarse(p, 0.01, rho, kind=1, n_sub=4), rho)
        assert np.array_equal(O.lift(p, rho), g)


def test_homogeneous_relaxation_is_exponential():
    """x-independent g with rho = rho_bar: the transport, field and
    projection terms vanish, so g^n = a^n g^0 (a = exp(-dt/eps^2)) and rho
    stays put, bitwise."""
    nx, nv, eps, dt = 16, 12, 0.5, 1e-3
    p = P(nx=nx, nv=nv, eps=eps)
    v, w, M, _ = O.velocity_grid(p)
    h = np.sin(v) * M + 0.3 * v * v * M
    g = np.tile(h, (nx, 1))
    rho = np.ones(nx)
    a = math.exp(-dt / (eps * eps))
    want = g.copy()
    for _ in range(7):
        want = a * want
    r2, g2, _, _ = O.fine(p, 7, dt, rho, g)
    assert np.array_equal(g2, want)
    assert np.array_equal(r2, rho)


def _projected_state(p, seed):
    rng = W.SplitMix64(seed)
    v, w, M, _ = O.velocity_grid(p)
    x = (np.arange(p.nx) + 0.5) / p.nx
    rho = 1.0 + 0.2 * np.cos(2 * np.pi * x + rng.uniform()) + 0.05 * np.sin(6 * np.pi * x)
    amp = 0.05 * np.cos(2 * np.pi * (x + 0.5 / p.nx) + rng.uniform())
    h = amp[:, None] * ((v * v - 1.0) * M + 0.3 * v * M)[None, :]
    g = h - (h @ w)[:, None] * M[None, :]
    return rho, g


@pytest.mark.parametrize("eps", [1.0, 1e-2])
def test_mean_of_g_stays_zero(eps):
    """<g^{n+1}> = a <g^n> since <M> = 1 and <xi M> = 0 (Sec. 3.2: the
    perturbation carries no mass)."""
    p = P(nx=32, nv=24, eps=eps)
    v, w, M, _ = O.velocity_grid(p)
    rho, g = _projected_state(p, 11)
    dt = O.dt_limit(p)
    mask = np.ones(p.nx, np.uint8)
    for _ in range(10):
        rho, g, mask, _ = O.fine_step(p, dt, rho, g, mask)
        assert np.abs(g @ w).max() <= 1e-15 * max(np.abs(g).max(), 1e-300) * 10


def _hybrid_small(flux_rule):
    w = W.hybrid(nx=128, nv=32, eps=1e-2, v_max=8.0)
    p = O.Params(nx=w.nx, nv=w.nv, eps=w.eps, v_max=w.v_max, adapt=True,
                 thr_g=w.thr_g, thr_R=1e-2, r_scale=1, flux_rule=flux_rule)
    return w, p


def test_mass_conservation_flux_matching_and_remark2_defect():
    """One flux per interface conserves mass to rounding (the premise of
    Lemma 1); the cell-based rule printed in S^HMM does not (Remark after
    Lemma 1)."""
    w, p = _hybrid_small(0)
    rho0 = 1.0 + 0.01 * np.cos(2 * np.pi * (np.arange(w.nx) + 0.5) / w.nx)
    dt = O.dt_limit(p)
    rho, g, mask, st = O.fine(p, 60, dt, rho0, w.g0)
    assert 0 < mask.sum() < w.nx            # a genuinely hybrid state
    assert abs(rho.sum() - rho0.sum()) / rho0.sum() < 1e-14
    _, p1 = _hybrid_small(1)
    rho1, _, _, _ = O.fine(p1, 60, dt, rho0, w.g0)
    assert abs(rho1.sum() - rho0.sum()) / rho0.sum() > 1e-12


def test_all_fluid_hybrid_equals_explicit_limit_scheme():
    """With every cell fluid, S^HMM is S^0 with the same step (Sec. 2.3)."""
    nx, nv = 32, 16
    p = P(nx=nx, nv=nv, eps=1e-3, adapt=True, thr_g=np.inf, thr_R=np.inf)
    rho, g = _projected_state(p, 5)
    dt = O.dt_limit(p)
    r2, g2, mask, st = O.fine(p, 9, dt, rho, g)
    ref = rho.copy()
    for _ in range(9):
        ref = O.limit_step(p, dt, ref)
    assert mask.sum() == 0 and st["kinetic_updates"] == 0
    assert np.abs(g2).max() == 0.0
    assert np.abs(r2 - ref).max() <= 1e-15 * np.abs(ref).max()


def test_asymptotic_preserving_limit_is_first_order_in_eps():
    """AP property (Sec. 1, Fig. 1 and Sec. 2.3): F_rho - S^0_rho = O(eps)
    over a fixed window with well-prepared (lifted) data."""
    nx, nv = 32, 32
    errs = []
    eps_list = [1e-3, 1e-4, 1e-5, 1e-6]   # one step size stable for all of them
    for eps in eps_list:
        p = P(nx=nx, nv=nv, eps=eps)
        _, _, _, m2 = O.velocity_grid(p)
        dt = 0.9 * (1.0 / nx) ** 2 / (2 * m2)
        x = (np.arange(nx) + 0.5) / nx
        rho = 1.0 + 0.3 * np.cos(2 * np.pi * x)
        rf, _, _, _ = O.fine(p, 40, dt, rho, O.lift(p, rho))
        rs = rho.copy()
        for _ in range(40):
            rs = O.limit_step(p, dt, rs)
        errs.append(np.abs(rf - rs).max())
    slopes = [math.log10(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(0.85 < s < 1.15 for s in slopes), (errs, slopes)


# ---------------------------------------------------------- limit / G ----

@pytest.mark.parametrize("implicit", [False, True])
def test_limit_scheme_fourier_decay(implicit):
    """Linearised S^0 on a cosine mode: factor 1 - m2 dt (4 sin^2(th/2)/dx^2 +
    rho_bar) (explicit); with E frozen from the old density the field term
    stays explicit, so the linearly implicit factor is
    (1 - m2 dt rho_bar) / (1 + m2 dt 4 sin^2(th/2)/dx^2)."""
    nx, m, delta = 64, 3, 1e-7
    dx = 1.0 / nx
    p = P(nx=nx, nv=32, rho_bar=1.0)
    _, _, _, m2 = O.velocity_grid(p)
    x = (np.arange(nx) + 0.5) * dx
    mode = np.cos(2 * np.pi * m * x)
    rho = 1.0 + delta * mode
    th = 2 * np.pi * m * dx
    lap = m2 * 4 * math.sin(th / 2) ** 2 / dx ** 2
    dt = 0.4 * dx * dx / (2 * m2) if not implicit else 5e-3
    out = O.limit_step_implicit(p, dt, rho) if implicit else O.limit_step(p, dt, rho)
    amp = np.dot(out - 1.0, mode) / np.dot(mode, mode)
    if implicit:
        lam = (1.0 - dt * m2 * 1.0) / (1.0 + dt * lap)
    else:
        lam = 1.0 - dt * (lap + m2 * 1.0)
    assert abs(amp / delta - lam) < 1e-6


def test_implicit_coarse_conserves_mass():
    """(I - m2 dt L) has unit column sums, so the implicit S^0 step conserves
    mass up to the linear solve's backward error, which grows with the
    condition number ~ 4 m2 dt / dx^2 of the system."""
    w = W.batched(nx=128, nv=16, eps=1e-2)
    p = O.Params(nx=128, nv=16, eps=1e-2)
    dt = 1.0 / 16
    out = O.coarse(p, dt, w.rho0)
    cond = 4 * dt * 128 ** 2
    rel = abs(out.sum() - w.rho0.sum()) / w.rho0.sum()
    assert rel < 1e-16 * cond / math.sqrt(128) * 10
    assert np.abs(out - w.rho0).max() > 1e-3      # the step did something


# ------------------------------------------------------------------ lift -

def test_lift_carries_no_mass_and_gives_the_fluid_flux():
    """<L rho> = 0 (Sec. 3.2) and <xi L rho>/eps = -m2 J + <xi M>^2 J: the
    lifted perturbation reproduces the drift-diffusion flux of S^0."""
    p = P(nx=64, nv=32, eps=1e-2)
    v, w, M, m2 = O.velocity_grid(p)
    x = (np.arange(64) + 0.5) / 64
    rho = 1.0 + 0.3 * np.cos(2 * np.pi * x)
    g = O.lift(p, rho)
    J = O.flux_J(p, rho, O.poisson(p, rho))
    assert np.abs(g @ w).max() < 1e-17
    assert np.abs((g @ (w * v)) / p.eps + m2 * J).max() < 1e-14 * np.abs(J).max() * 10


@pytest.mark.parametrize("L", [2, 3])
def test_higher_order_lift_carries_no_mass(L):
    """Def. 1: the lifted perturbation has zero mass for every order."""
    p = P(nx=64, nv=32, eps=0.05)
    v, w, M, m2 = O.velocity_grid(p)
    x = (np.arange(64) + 0.5) / 64
    g = O.lift(p, 1.0 + 0.3 * np.cos(2 * np.pi * x), L)
    assert np.abs(g @ w).max() < 1e-16


def _ce_terms_continuous(A, xs):
    """Chapman-Enskog terms of Sec. 2.1 (eq. Identification) for
    rho = 1 + A cos(2 pi x) on the unit torus, in closed form: the Poisson
    law E' = rho - 1 with mean-zero E gives E = A sin(2 pi x) / (2 pi);
    J = rho' - E rho; K = J' - E J; dJ/dt = J'' - rho (J - mean J) - E J'."""
    x = sp.symbols("x")
    rho = 1 + A * sp.cos(2 * sp.pi * x)
    E = A * sp.sin(2 * sp.pi * x) / (2 * sp.pi)
    J = sp.diff(rho, x) - E * rho
    Jbar = sp.integrate(J, (x, 0, 1))
    K = sp.diff(J, x) - E * J
    dtJ = sp.diff(J, x, 2) - rho * (J - Jbar) - E * sp.diff(J, x)
    f = {k: sp.lambdify(x, e, "numpy") for k, e in
         dict(E=E, J=J, K=K, K1=sp.diff(K, x), dtJ=dtJ).items()}
    return {k: np.broadcast_to(np.asarray(fn(xs), dtype=float), xs.shape) for k, fn in f.items()}


def test_higher_order_lift_converges_to_chapman_enskog_terms():
    """The discrete lifting of order 3 at the interfaces converges, at second
    order in dx (the interface flux J of S^0 is centred), to
    (I - Pi)[eps h1 + eps^2 h2 + eps^3 h3] built from the closed-form
    fields; a dropped term, a wrong sign or coefficient in h2 or h3, or a
    shifted stencil would leave an O(1) error."""
    A, eps, nv = 0.3, 0.1, 32
    errs = []
    for nx in (64, 128, 256):
        p = P(nx=nx, nv=nv, eps=eps, rho_bar=1.0)
        v, w, M, m2 = O.velocity_grid(p)
        xi = (np.arange(nx) + 1.0) / nx           # interfaces x_{i+1/2}
        c = _ce_terms_continuous(A, xi)
        V, Mj = v[None, :], M[None, :]
        h1 = -V * Mj * c["J"][:, None]
        h2 = (V * V - 1) * Mj * c["K"][:, None]
        rho_i = 1 + A * np.cos(2 * np.pi * xi)
        h3 = V * Mj * (c["dtJ"][:, None] - (V * V - 1) * c["K1"][:, None]
                       - c["E"][:, None] * (3 - V * V) * c["K"][:, None])
        h = eps * h1 + eps ** 2 * h2 + eps ** 3 * h3
        g_cont = h - (h @ w)[:, None] * Mj
        x = (np.arange(nx) + 0.5) / nx
        g = O.lift(p, 1 + A * np.cos(2 * np.pi * x), 3)
        errs.append(np.abs(g - g_cont).max() / np.abs(g_cont).max())
        del rho_i
    assert errs[-1] < 2e-4
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5, errs


def _relaxed_gap(eps, L, nx=512, nv=64):
    """Distance between the perturbation F itself relaxes to and the lifting
    of order L of F's density: F runs for 20 eps^2 (twenty relaxation times,
    a^n ~ e^-20, short against the macroscopic time) from (rho, L rho)."""
    p = P(nx=nx, nv=nv, eps=eps, rho_bar=1.0)
    x = (np.arange(nx) + 0.5) / nx
    rho = 1 + 0.3 * np.cos(2 * np.pi * x)
    dt = O.dt_limit(p)
    n = int(math.ceil(20 * eps * eps / dt))
    r, g, _, _ = O.fine(p, n, dt, rho, O.lift(p, rho, L))
    return np.abs(g - O.lift(p, r, L)).max() / np.abs(g).max()


def test_lift_order_matches_the_schemes_relaxed_perturbation():
    """Chapman-Enskog consistency (Sec. 2.1, Def. 1): the scheme's own
    relaxed perturbation differs from the lifting of order L by O(eps^L)
    (relative), so each order gains a factor ~eps, down to the
    discretisation floor of the upwind transport.  Slopes in eps: 1 for
    L = 1, 2 for L = 2, more than 2 for L = 3."""
    gaps = {L: [_relaxed_gap(e, L) for e in (0.02, 0.01)] for L in (1, 2, 3)}
    slope = {L: math.log2(gaps[L][0] / gaps[L][1]) for L in (1, 2, 3)}
    assert 0.9 < slope[1] < 1.1, gaps
    assert 1.8 < slope[2] < 2.2, gaps
    assert slope[3] > 2.3, gaps
    assert gaps[1][1] > 10 * gaps[2][1] > 40 * gaps[3][1], gaps


# --------------------------------------------------------------- dt rule -

def _jacobian(p, dt, n_eq=1.0, h=1e-7):
    nx, nv = p.nx, p.nv
    rho0, g0 = np.full(nx, n_eq), np.zeros((nx, nv))
    mask = np.ones(nx, np.uint8)
    base_r, base_g, _, _ = O.fine_step(p, dt, rho0, g0, mask)
    base = np.concatenate([base_r, base_g.ravel()])
    n = nx + nx * nv
    Jm = np.empty((n, n))
    for k in range(n):
        r, g = rho0.copy(), g0.copy().ravel()
        if k < nx:
            r[k] += h
        else:
            g[k - nx] += h
        rr, gg, _, _ = O.fine_step(p, dt, r, g.reshape(nx, nv), mask)
        Jm[:, k] = (np.concatenate([rr, gg.ravel()]) - base) / h
    return Jm


@pytest.mark.parametrize("eps", [1.0, 1e-2, 0.466 / (8.0 * 16), 0.25 / (8.0 * 16)])
def test_dt_rule_is_linearly_stable(eps):
    """The step-size rule (the paper gives none) keeps the linearised step
    around equilibrium stable at theta = 0.9 and not at 1.3.  The last two
    cases are diffusive (dt >> eps^2) with eps v_max / dx = 0.466 and 0.25,
    where the upwind transport of g and the diffusion of rho through g
    couple: a rule that bounds each alone (phi_t <= 1, phi_d <= 1) gives a
    spectral radius of about 1.16 there at theta = 0.9."""
    p = P(nx=16, nv=8, eps=eps, rho_bar=1.0)
    lim = O.dt_limit(p, 1.0)
    r09 = np.abs(np.linalg.eigvals(_jacobian(p, 0.9 * lim))).max()
    r13 = np.abs(np.linalg.eigvals(_jacobian(p, 1.3 * lim))).max()
    assert r09 <= 1.0 + 1e-6
    assert r13 > 1.0 + 1e-3


# -------------------------------------------------------------- parareal -

def _parareal_case():
    w = W.small(nx=32, nv=16)
    p = O.Params(nx=32, nv=16, eps=0.5)
    return w, p


@pytest.mark.parametrize("k,L", [(1, 1), (2, 1), (3, 1), (2, 2), (2, 3)])
def test_parareal_first_k_slices_equal_sequential(k, L):
    """After k iterations the first k+1 slice values are the sequential fine
    solution (parareal property, Sec. 3.1), bitwise with the F + (G - G)
    form of the correction, for liftings of order L = 1, 2, 3."""
    w, p = _parareal_case()
    seq = O.sequential(p, w.rho0, w.g0, w.t_end, w.n_slices, lift_order=L)
    out, err, it = O.parareal(p, w.rho0, w.g0, w.t_end, w.n_slices, k, lift_order=L)
    assert it == k
    assert np.array_equal(out[: k + 1], seq[: k + 1])
    if k < w.n_slices:
        assert np.abs(out[k + 1:] - seq[k + 1:]).max() > 0.0


@pytest.mark.parametrize("k", [1, 2, 3])
def test_full_state_parareal_first_k_slices_equal_plain_F(k):
    """Full-state mode (U = (rho, g), G(U) = (G rho, L G rho)): after k
    iterations the first k+1 slices are the plain sequential F carried
    through the slices without relifting (the parareal property of
    Sec. 3.1 for the state of the fine scheme), bitwise; at K = N, all of
    them.  The plain reference is F composed slice by slice, written out
    here, not the oracle's sequential routine."""
    w, p = _parareal_case()
    dt = O.dt_limit(p)
    span = w.t_end / w.n_slices
    nf = int(math.ceil(span / dt))
    plain = [w.rho0.copy()]
    r, g = w.rho0.copy(), w.g0.copy()
    for n in range(w.n_slices):
        r, g, _, _ = O.fine(p, nf, span / nf, r, g)
        plain.append(r.copy())
    plain = np.array(plain)
    out, err, it = O.parareal(p, w.rho0, w.g0, w.t_end, w.n_slices, k, mode=1)
    assert it == k
    assert np.array_equal(out[: k + 1], plain[: k + 1])
    full, _, _ = O.parareal(p, w.rho0, w.g0, w.t_end, w.n_slices, w.n_slices, mode=1)
    assert np.array_equal(full, plain)
    # the density-only mode converges to the relifted sequence instead
    rho_only, _, _ = O.parareal(p, w.rho0, w.g0, w.t_end, w.n_slices, w.n_slices)
    assert np.abs(rho_only[2:] - plain[2:]).max() > 0.0


def test_parareal_converges_everywhere_at_K_equals_N():
    w, p = _parareal_case()
    seq = O.sequential(p, w.rho0, w.g0, w.t_end, w.n_slices)
    out, err, it = O.parareal(p, w.rho0, w.g0, w.t_end, w.n_slices, w.n_slices)
    assert np.array_equal(out, seq)


def test_parareal_mass_lemma1():
    """Lemma 1: every slice of every iterate keeps the initial mass."""
    w = W.batched(nx=64, nv=16, eps=1e-2, n_slices=6)
    p = O.Params(nx=64, nv=16, eps=1e-2)
    m0 = w.rho0.sum()
    for K in (1, 3):
        out, err, it = O.parareal(p, w.rho0, w.g0, 0.02, 6, K)
        assert np.abs(out.sum(axis=1) - m0).max() / m0 < 1e-14


def test_parareal_stops_at_tolerance():
    w, p = _parareal_case()
    out, err, it = O.parareal(p, w.rho0, w.g0, w.t_end, w.n_slices, 4, tol=0.02)
    assert err[-1] < 0.02 and all(e >= 0.02 for e in err[:-1])


# ---------------------------------------------------- rational brute force

def _exact_constants(p, dt):
    v, w, M, m2 = O.velocity_grid(p)
    a = math.exp(-dt / (p.eps * p.eps))
    b = p.eps * (1.0 - a)
    dv = 2.0 * p.v_max / (p.nv - 1)
    return dict(v=[Fr(x) for x in v], w=[Fr(x) for x in w], M=[Fr(x) for x in M],
                m2=Fr(m2), a=Fr(a), b=Fr(b), dx=Fr(p.x_len / p.nx), dv=Fr(dv),
                eps=Fr(p.eps), dt=Fr(dt), rho_bar=Fr(p.rho_bar), adapt=p.adapt,
                thr_g=Fr(p.thr_g), thr_R=Fr(p.thr_R),
                r=Fr(p.eps * p.eps) if p.r_scale else Fr(1))


# (adapt, flux_rule, r_scale, thr_R): the thresholds put eps^2 |R| and |R|
# on different sides of thr_R for some cells (eps = 0.5, so the two scalings
# differ by 4x and a plain eps would differ from both), and leave a mixed
# kinetic/fluid mask, so the cell-based density update differs from the
# one-flux rule.
_BRUTE_CASES = [
    (False, 0, 0, 100.0),
    (True, 0, 0, 100.0),
    (True, 1, 0, 500.0),
    (True, 0, 1, 150.0),
    (True, 1, 1, 150.0),
]


@pytest.mark.parametrize("adapt,flux_rule,r_scale,thr_R", _BRUTE_CASES)
def test_bruteforce_rational_tiny_grid(adapt, flux_rule, r_scale, thr_R):
    """Nx=8, Nv=4, three steps in exact rationals (eq. S^HMM with the status
    rules of Sec. 2.3; the cell-based density update as printed when
    flux_rule = 1; the remainder criterion scaled by eps^2 when r_scale = 1):
    the oracle agrees to 1e-14 and the masks are identical."""
    nx, nv = 8, 4
    p = O.Params(nx=nx, nv=nv, eps=0.5, v_max=4.0, adapt=adapt, thr_g=2e-3,
                 thr_R=thr_R, rho_bar=1.0, r_scale=r_scale, flux_rule=flux_rule)
    rng = W.SplitMix64(99)
    rho = 1.0 + 0.2 * (rng.uniforms(nx) - 0.5)
    g = 0.01 * (rng.uniforms(nx * nv).reshape(nx, nv) - 0.5)
    g[2:7] *= 1e-3      # cells 3..6: both interface norms below thr_g
    dt = 0.5 * O.dt_limit(p)
    c = _exact_constants(p, dt)
    c["flux_rule"] = flux_rule
    mask = O.initial_status(p, rho, g)
    rr = [Fr(x) for x in rho]
    gg = [[Fr(x) for x in row] for row in g]
    mm = [int(x) for x in mask]
    r_o, g_o, m_o = rho.copy(), g.copy(), mask.copy()
    saw_mixed = False
    for _ in range(3):
        saw_mixed |= 0 < sum(mm) < nx
        rr, gg, mm = RS.step(c, rr, gg, mm)
        r_o, g_o, m_o, _ = O.fine_step(p, dt, r_o, g_o, m_o)
        assert m_o.tolist() == mm
    rr = np.array([float(x) for x in rr])
    gg = np.array([[float(x) for x in row] for row in gg])
    assert np.abs(r_o - rr).max() <= 1e-14
    assert np.abs(g_o - gg).max() <= 1e-14 * np.abs(gg).max()
    if adapt:
        assert saw_mixed


def test_bruteforce_cases_separate_the_two_remainder_scalings():
    """The r_scale cases above are only a pin of the eps^2 factor if the
    literal and the scaled criterion give different masks on their data."""
    nx, nv = 8, 4
    rng = W.SplitMix64(99)
    rho = 1.0 + 0.2 * (rng.uniforms(nx) - 0.5)
    g = 0.01 * (rng.uniforms(nx * nv).reshape(nx, nv) - 0.5)
    g[2:7] *= 1e-3
    masks = []
    for r_scale in (0, 1):
        p = O.Params(nx=nx, nv=nv, eps=0.5, v_max=4.0, adapt=True, thr_g=2e-3,
                     thr_R=150.0, rho_bar=1.0, r_scale=r_scale)
        m = O.initial_status(p, rho, g)
        masks.append(O.update_status(p, rho, g, m).tolist())
    assert masks[0] != masks[1]


def test_cell_based_mass_defect_is_the_flux_mismatch_at_mixed_interfaces():
    """Remark after Lemma 1: the cell-based update of eq. S^HMM is not
    conservative.  Summing its per-cell flux differences, every interface
    between two cells of the same status cancels, and an interface between a
    kinetic cell i and a fluid cell i+1 leaves -(<xi g^{n+1}>/eps + m2 J);
    the reverse order leaves the opposite.  So one step changes the mass
    sum(rho) dx by exactly dt times the signed sum of that mismatch over the
    mixed interfaces."""
    w, p = _hybrid_small(1)
    v, wq, M, m2 = O.velocity_grid(p)
    dx = p.x_len / p.nx
    x = (np.arange(w.nx) + 0.5) / w.nx
    rho = 1.0 + 0.01 * np.cos(2 * np.pi * x)
    g = w.g0.copy()
    mask = O.initial_status(p, rho, g)
    dt = O.dt_limit(p)
    checked = 0
    for _ in range(25):
        E = O.poisson(p, rho)
        J = O.flux_J(p, rho, E)
        r1, g1, m1, _ = O.fine_step(p, dt, rho, g, mask)
        mom = (g1 * (wq * v)[None, :]).sum(axis=1) / p.eps
        left, right = mask.astype(int), np.roll(mask, -1).astype(int)
        sign = right - left            # -1: kinetic|fluid, +1: fluid|kinetic
        mismatch = sign * (mom + m2 * J)
        want = dt * mismatch.sum()
        got = (r1 - rho).sum() * dx
        scale = dt * np.abs(mismatch).sum()
        if 0 < mask.sum() < w.nx:
            assert abs(got - want) <= 1e-12 * scale + 1e-16 * rho.sum() * dx
            checked += abs(want) > 1e-6 * scale
        else:
            assert abs(got) <= 1e-15 * rho.sum() * dx
        rho, g, mask = r1, g1, m1
    assert checked > 0


@pytest.mark.parametrize("eps", [0.1, 0.03])
def test_remainder_threshold_flips_exactly_at_eps2_scaled_R(eps):
    """Sec. 2.3 compares |R_i| with thr_R; r_scale = 1 compares eps^2 |R_i|
    (the O(eps^2) factor in front of R in eq. HigherOrderModel).  With g = 0
    (both interface norms below thr_g) the status of a cell then depends on
    the remainder alone, and it must flip exactly where thr_R crosses
    eps^2 |R_i| (resp. |R_i|).  R_i is evaluated independently, in exact
    rationals from the printed Table 1."""
    nx, nv = 16, 8
    x = (np.arange(nx) + 0.5) / nx
    rho = 1.0 + 0.1 * np.cos(2 * np.pi * x) + 0.03 * np.sin(6 * np.pi * x)
    dx = Fr(1, nx)
    rr = [Fr(r) for r in rho]
    R = [float(r) for r in RS.remainder(rr, RS.poisson(rr, Fr(1), dx), Fr(1), dx, RS.table1())]
    g = np.zeros((nx, nv))
    big = [i for i in range(nx) if abs(R[i]) > 1e-3 * max(map(abs, R))]
    assert len(big) >= nx // 2
    for r_scale, fac in ((1, eps * eps), (0, 1.0)):
        for i in big:
            for side, want in ((1 + 1e-6, 0), (1 - 1e-6, 1)):
                p = O.Params(nx=nx, nv=nv, eps=eps, adapt=True, thr_g=1e-3,
                             thr_R=fac * abs(R[i]) * side, rho_bar=1.0, r_scale=r_scale)
                for start in (0, 1):    # fluid -> kinetic and kinetic -> fluid rules
                    m = O.update_status(p, rho, g, np.full(nx, start, np.uint8))
                    assert m[i] == want, (r_scale, i, side, start)


# ------------------------------------------- linear symbol of one step ---

def _fine_symbol(p, dt, theta):
    """The (Nv+1) x (Nv+1) matrix of one step of the scheme (every
    interface kinetic, one flux per interface) on the Fourier mode e^{i theta
    i} of a small perturbation of rho = rho_bar, g = 0, written out from the
    step's definition: the Poisson prefix sum with its mean removed, the
    flux J, the upwind x-fluxes of g, the projection P = <X> M, the
    exponential relaxation g* = a g - b (X - P M + v M J) and the flux-form
    density update with Phi = <v g*> / eps.  The field term E d_v g is
    quadratic in the perturbation and drops out.  State (rho^, g^_0..)."""
    v, w, M, _ = O.velocity_grid(p)
    nv, dx, eps = p.nv, p.x_len / p.nx, p.eps
    a = math.exp(-dt / eps ** 2)
    b = eps * (1.0 - a)
    z = np.exp(1j * theta)
    vp, vm = np.maximum(v, 0.0), np.maximum(-v, 0.0)
    sym_E = dx / (1.0 - 1.0 / z)                         # E^ per rho^
    sym_J = (z - 1.0) / dx - p.rho_bar * sym_E           # J^ per rho^
    sym_A = (vp * (1.0 - 1.0 / z) - vm * (z - 1.0)) / dx  # A^_j per g^_j
    A = np.zeros((nv + 1, nv + 1), dtype=complex)
    for col in range(nv + 1):
        u = np.zeros(nv + 1, dtype=complex)
        u[col] = 1.0
        rho_h, g_h = u[0], u[1:]
        X = sym_A * g_h
        Pm = np.dot(w, X)
        gs = a * g_h - b * (X - Pm * M + v * M * (sym_J * rho_h))
        phi = np.dot(w, v * gs) / eps
        A[0, col] = rho_h - (dt / dx) * (1.0 - 1.0 / z) * phi
        A[1:, col] = gs
    return A


@pytest.mark.parametrize("eps", [1.0, 0.1, 0.01])
def test_fine_matches_powers_of_its_linear_symbol(eps):
    """A small cosine mode (amplitude 1e-7) in rho and in g, 12 steps of F:
    the oracle equals A(theta)^12 applied to the mode to first order in the
    amplitude.  A wrong upwind side, sign of the field, index of the
    interface, projection weight or relaxation constant changes A."""
    nx, nv, m, delta, n = 32, 16, 3, 1e-7, 12
    p = P(nx=nx, nv=nv, eps=eps, rho_bar=1.0)
    v, w, M, m2 = O.velocity_grid(p)
    dt = O.dt_limit(p)
    theta = 2 * np.pi * m / nx
    i = np.arange(nx)
    c = (v ** 2 - m2) * M                      # <c> = 0: a valid perturbation of g
    rho0 = 1.0 + delta * np.cos(theta * i)
    g0 = delta * np.outer(np.cos(theta * i), c)
    rho, g, _, _ = O.fine(p, n, dt, rho0, g0)
    u = np.concatenate(([delta], delta * c)).astype(complex)
    un = np.linalg.matrix_power(_fine_symbol(p, dt, theta), n) @ u
    zi = np.exp(1j * theta * i)
    rho_pred = np.real(un[0] * zi)
    g_pred = np.real(np.outer(zi, un[1:]))
    assert np.abs((rho - 1.0) - rho_pred).max() <= 1e-5 * np.abs(rho_pred).max()
    assert np.abs(g - g_pred).max() <= 1e-5 * np.abs(g_pred).max()
    # and the perturbation did evolve: the prediction is not the identity
    assert np.abs(rho_pred - delta * np.cos(theta * i)).max() > 1e-3 * delta
