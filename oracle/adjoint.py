"""Discrete adjoint of the oracle's 1d1v time step.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): imported by tests/ and
bench.py's CPU legs, never by the product package.  Plain numpy, FP64, all
states kept in memory (small cases only).

Objective (field energy at the final time, the paper's W_E of Eq. 12 with
the factor 1/2 and no 1/cP):

    J = 1/2 sum_i E_i(T)^2 dx,   T = nsteps dt.

Parameters theta: the initial distribution f0 of one species (Sec. 3.3,
Eq. 11 / Eq. 17 form) -- the amplitudes amp_m of its density modes and the
x-drift u_b of each of its beams.  The marker lattice and its jitter do not
depend on theta; theta enters only through the marker values
f_l = f0(x_l, v_l; theta).  Hence

    dJ/dtheta = sum_l (dJ/df_l) df0(x_l, v_l)/dtheta,

with dJ/df_l the total derivative through every later reconstruction (Eq. 4),
moment (Eq. 14), Poisson solve (Eq. 6) and push (Sec. 2) of the forward run,
which is the oracle's own OracleSim step.

Backward recursion (states n = N .. 0; lambda_X, lambda_V per marker, mu_l
accumulates dJ/df_l).  With E^n the field of state n, G the cloud-in-cell
gather, and P the linear Poisson operator (E = P rho):
  e^N      = dx E^N
  e^n      = sum_l (lambda_V^{n+1} + dt lambda_X^{n+1})_l (q/m) dt G(X^n_l)   (n < N)
  psi^n    = q dv P^T e^n,  P^T = -P (the multiplier of Eq. 6 is odd and
             purely imaginary)
  A = psi / D, B = psi F / D on the grid of state n (0 where D = 0), with
             F = N / D the reconstruction of state n
  mu_l    += sum_cells A alpha_l
  g_X, g_V = sum_cells (A f_l - B) d(alpha_l)/dX, d(alpha_l)/dV
  lambda_X^n = lambda_X^{n+1} + lt (q/m) dt dE^n/dx(X^n) + g_X
  lambda_V^n = lt + g_V,   lt = lambda_V^{n+1} + dt lambda_X^{n+1}
(at n = N only the g terms).  The derivatives of the cloud-in-cell weights
are the one-sided ones that go with the floor() of the weight rule.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O


def _cic(y):
    """Lower cell i0 = floor(y - 1/2) and weight w of cell i0 + 1 (cloud in
    cell on a cell-centred grid, Fig. 1); y in cell units."""
    u = y - 0.5
    i0 = np.floor(u)
    return i0.astype(np.int64), u - i0


def _grid_at(G, i, j):
    """G[i, j], 0 where the velocity row j is off the grid."""
    ok = (j >= 0) & (j < G.shape[1])
    out = np.zeros(i.shape)
    out[ok] = G[i[ok], j[ok]]
    return out


def f0_gradient(f0: O.F0, L: float, x, v):
    """df0/d(amp_m) (nmode, n) and df0/d(u_b, x component) (nbeam, n) of the
    1d1v f0 = sum_b n_b M(v; u_b, vth_b) (1 + sum_m amp_m cos(2 pi mode_m x / L
    + phase_m)) at the points (x, v)."""
    x = np.asarray(x, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    pert = np.ones_like(x)
    cosm = []
    for (mode, amp, phase) in f0.modes:
        c = np.cos(2.0 * math.pi * mode * x / L + phase)
        cosm.append(c)
        pert += amp * c
    beams = []
    for (nb, u, vth) in f0.beams:
        s = vth[0]
        beams.append((nb * np.exp(-0.5 * ((v - u[0]) / s) ** 2) / (math.sqrt(2.0 * math.pi) * s), u[0], s))
    B = sum(b[0] for b in beams)
    d_amp = np.array([B * c for c in cosm]) if cosm else np.zeros((0, x.size))
    d_u = np.array([pert * Mb * (v - u) / (s * s) for (Mb, u, s) in beams])
    return d_amp, d_u


def field_energy_gradient(nx, L, dt, species, f0s, lattices, seed, jitter, theta_species, nsteps,
                          cP=1.0, softening=True):
    """Run the oracle forward nsteps from the lattice markers of every species
    (f0s[s], lattices[s]; every species is seeded with `seed`) and return
    (J, dJ/d amp (nmode,), dJ/d u_b (nbeam,), mu) for the f0 of species
    theta_species; mu[s] = dJ/df_l of the markers of species s."""
    ns = len(species)
    dx = L / nx
    sim = O.OracleSim(1, nx, L, dt, species, cP, softening)
    for s in range(ns):
        sim.init_markers(s, lattices[s], f0s[s], seed, jitter)
    x0 = sim.x[theta_species].copy()
    v0 = sim.v[theta_species][0].copy()
    sim.refresh()
    hist = []   # per state n: per species (x, v, F, D), and E

    def snapshot():
        hist.append(([(sim.x[s].copy(), sim.v[s][0].copy(), sim.f[s].copy(), sim.den[s].copy())
                      for s in range(ns)], sim.E.copy()))

    snapshot()
    for _ in range(nsteps):
        sim.step(1)
        snapshot()
    J = 0.5 * float(np.sum(sim.E ** 2)) * dx

    lam_x = [np.zeros(sim.x[s].size) for s in range(ns)]
    lam_v = [np.zeros(sim.x[s].size) for s in range(ns)]
    mu = [np.zeros(sim.x[s].size) for s in range(ns)]
    for n in range(nsteps, -1, -1):
        states, E = hist[n]
        lt = [None] * ns
        if n == nsteps:
            e = dx * E
        else:
            e = np.zeros(nx)
            for s, sp in enumerate(species):
                if not sp.mobile:
                    continue
                xs = states[s][0]
                lt[s] = lam_v[s] + dt * lam_x[s]
                i0, w = _cic(xs / dx)
                ia, ib = np.mod(i0, nx), np.mod(i0 + 1, nx)
                c = lt[s] * (sp.q / sp.m) * dt
                np.add.at(e, ia, c * (1.0 - w))
                np.add.at(e, ib, c * w)
        PTe = -O.poisson(nx, L, cP, softening, e)
        for s, sp in enumerate(species):
            xs, vs, F, D = states[s]
            dv = (sp.vmax[0] - sp.vmin[0]) / sp.nv[0]
            psi = sp.q * dv * PTe
            with np.errstate(divide="ignore", invalid="ignore"):
                A = np.where(D > 0, psi[:, None] / D, 0.0)
                B = np.where(D > 0, psi[:, None] * F / D, 0.0)
            i0, wx = _cic(xs / dx)
            ia, ib = np.mod(i0, nx), np.mod(i0 + 1, nx)
            j0, wv = _cic((vs - sp.vmin[0]) / dv)
            fl = sim.fl[s]
            g_x = np.zeros(xs.size)
            g_v = np.zeros(xs.size)
            for (ii, ax, dax) in ((ia, 1.0 - wx, -1.0 / dx), (ib, wx, 1.0 / dx)):
                for (jj, av, dav) in ((j0, 1.0 - wv, -1.0 / dv), (j0 + 1, wv, 1.0 / dv)):
                    a = _grid_at(A, ii, jj)
                    b = _grid_at(B, ii, jj)
                    mu[s] += a * ax * av
                    cc = a * fl - b
                    g_x += cc * dax * av
                    g_v += cc * ax * dav
            if n == nsteps:
                lam_x[s], lam_v[s] = g_x, g_v
            elif sp.mobile:
                dEdx = (E[ib] - E[ia]) / dx
                lam_x[s] = lam_x[s] + lt[s] * (sp.q / sp.m) * dt * dEdx + g_x
                lam_v[s] = lt[s] + g_v
    d_amp, d_u = f0_gradient(f0s[theta_species], L, x0, v0)
    m = mu[theta_species]
    return J, d_amp @ m, d_u @ m, mu


def field_energy(nx, L, dt, species, f0s, lattices, seed, jitter, nsteps, cP=1.0, softening=True):
    """J of the oracle's forward run (for finite differences)."""
    sim = O.OracleSim(1, nx, L, dt, species, cP, softening)
    for s in range(len(species)):
        sim.init_markers(s, lattices[s], f0s[s], seed, jitter)
    sim.refresh()
    sim.step(nsteps)
    return 0.5 * float(np.sum(sim.E ** 2)) * (L / nx)
