"""Exact-rational evaluation of the hybrid micro-macro step (Sec. 2.2-2.3).

A brute-force check of the oracle on tiny grids: the scheme's constants are
taken as the binary64 values the oracle uses (v_j, w_j, M_j, m2, a, b, dx,
dv) converted exactly to Fractions, and every operation after that is exact.
Table 1 is read from tests/golden/table1_fd.txt (the printed table), not
from the oracle.  Norm comparisons are done on squares so that no square
root is needed.
"""
from __future__ import annotations

import os
from fractions import Fraction as Fr

_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_fd.txt")


def table1():
    rows = {}
    with open(_GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[int(parts[0])] = [Fr(t) for t in parts[1:]]
    return rows


def _deriv(f, d, dx, T):
    n = len(f)
    c = T[d]
    return [sum(c[k + 3] * f[(i + k) % n] for k in range(-3, 4)) / dx ** d for i in range(n)]


def poisson(rho, rho_bar, dx):
    """E_{i+1/2} - E_{i-1/2} = (rho_i - rho_bar) dx, mean-zero E."""
    S, E = Fr(0), []
    for r in rho:
        S += (r - rho_bar) * dx
        E.append(S)
    mean = sum(E) / len(E)
    return [e - mean for e in E]


def flux_J(rho, E, dx):
    n = len(rho)
    return [(rho[(i + 1) % n] - rho[i]) / dx - E[i] * (rho[i] + rho[(i + 1) % n]) / 2
            for i in range(n)]


def remainder(rho, E, rho_bar, dx, T):
    """eq. Remainder with centred E and d_t E = J - mean(J)."""
    n = len(rho)
    Ec = [(E[(i - 1) % n] + E[i]) / 2 for i in range(n)]
    d1r = _deriv(rho, 1, dx, T)
    Jc = [d1r[i] - Ec[i] * rho[i] for i in range(n)]
    d1J, d2J, d3J = (_deriv(Jc, d, dx, T) for d in (1, 2, 3))
    mJ = sum(Jc) / n
    return [-d3J[i] + Ec[i] * d2J[i] + (2 * rho[i] - 3 * rho_bar) * d1J[i]
            + 2 * Jc[i] * d1r[i] - d1r[i] * (Jc[i] - mJ) for i in range(n)]


def step(c, rho, g, mask):
    """One step of S^HMM.

    c: dict of exact constants: v, w, M (lists), m2, a, b, dx, dv, eps, dt,
    rho_bar, adapt, thr_g, thr_R, r (all Fractions / ints), and optionally
    flux_rule: 0 (default) one flux per interface, 1 the cell-based density
    update as printed in eq. S^HMM (kinetic cell: the difference of the new
    moments <xi g^{n+1}>/eps of its two interfaces, g^{n+1} being 0 on a
    fluid interface; fluid cell: m2 times the difference of the two J).
    Returns (rho, g, mask) at t^{n+1}.
    """
    T = table1()
    nx, nv = len(rho), len(c["v"])
    v, w, M = c["v"], c["w"], c["M"]
    E = poisson(rho, c["rho_bar"], c["dx"])
    J = flux_J(rho, E, c["dx"])
    kin = [mask[i] or mask[(i + 1) % nx] for i in range(nx)]
    new_mask = list(mask)
    if c["adapt"]:
        R = remainder(rho, E, c["rho_bar"], c["dx"], T)
        N2 = [sum(w[j] * g[i][j] ** 2 for j in range(nv)) for i in range(nx)]
        thr_g2 = c["thr_g"] ** 2
        for i in range(nx):
            big_R = c["r"] * abs(R[i]) > c["thr_R"]
            if not mask[i]:
                new_mask[i] = 1 if big_R else 0
            else:
                small = N2[(i - 1) % nx] <= thr_g2 and N2[i] <= thr_g2
                new_mask[i] = 0 if (small and not big_R) else 1
    gn = [[Fr(0)] * nv for _ in range(nx)]
    Phi = [Fr(0)] * nx
    for i in range(nx):
        if not kin[i]:
            Phi[i] = -c["m2"] * J[i]
            continue
        gl, gc, gr = g[(i - 1) % nx], g[i], g[(i + 1) % nx]
        Ei = E[i]
        Ep, Em = (abs(Ei) + Ei) / 2, (abs(Ei) - Ei) / 2
        X = []
        for j in range(nv):
            vp, vm = (abs(v[j]) + v[j]) / 2, (abs(v[j]) - v[j]) / 2
            A = (vp * (gc[j] - gl[j]) - vm * (gr[j] - gc[j])) / c["dx"]
            Gr = Ep * gc[j] - Em * gc[j + 1] if j < nv - 1 else Fr(0)
            Gl = Ep * gc[j - 1] - Em * gc[j] if j > 0 else Fr(0)
            X.append(A + (Gr - Gl) / c["dv"])
        P = sum(w[j] * X[j] for j in range(nv))
        gn[i] = [c["a"] * gc[j] - c["b"] * (X[j] - P * M[j] + v[j] * M[j] * J[i])
                 for j in range(nv)]
        Phi[i] = sum(w[j] * v[j] * gn[i][j] for j in range(nv)) / c["eps"]
    if c.get("flux_rule", 0) == 1:
        # eq. S^HMM as printed: rho_i += dt/dx * Jt_i with a per-cell flux
        # difference chosen by the status of cell i at t^n.
        mom = [sum(w[j] * v[j] * gn[i][j] for j in range(nv)) / c["eps"] for i in range(nx)]
        rn = []
        for i in range(nx):
            if mask[i]:
                Jt = -(mom[i] - mom[(i - 1) % nx])
            else:
                Jt = c["m2"] * (J[i] - J[(i - 1) % nx])
            rn.append(rho[i] + c["dt"] / c["dx"] * Jt)
        return rn, gn, new_mask
    rn = [rho[i] - c["dt"] / c["dx"] * (Phi[i] - Phi[(i - 1) % nx]) for i in range(nx)]
    return rn, gn, new_mask
