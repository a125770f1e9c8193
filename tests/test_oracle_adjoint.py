"""Pins of the oracle's discrete adjoint (oracle/adjoint.py) against things
that do not share its code: central finite differences of the oracle's own
forward run, finite differences of the C f0, the transpose of the oracle's
Poisson operator, and the quadratic dependence of J on a small amplitude in
the linear regime."""
import math

import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import oracle as O


def two_stream_small(amps=(0.02, 0.01), u=1.5, with_ions=True):
    species = [O.Species(q=-1.0, m=1.0, nv=(24,), vmin=(-5.0,), vmax=(5.0,))]
    f0s = [O.F0(beams=[(0.5, (u,), (0.6,)), (0.5, (-u,), (0.6,))],
                modes=[(1, amps[0], 0.3), (2, amps[1], 1.1)])]
    lattices = [(2, 2, 1, 1)]
    if with_ions:
        species.append(O.Species(q=1.0, m=100.0, nv=(8,), vmin=(-0.5,), vmax=(0.5,), mobile=False))
        f0s.append(O.F0(beams=[(1.0, (0.0,), (0.1,))], modes=[(1, 0.005, 0.0)]))
        lattices.append((1, 1, 1, 1))
    return species, f0s, lattices


NX, L, DT, NSTEPS, SEED = 16, 10.0, 0.1, 25, 11


def with_theta(f0, amps=None, drifts=None):
    modes = [(m, amps[k] if amps is not None else a, ph) for k, (m, a, ph) in enumerate(f0.modes)]
    beams = [(n, ((drifts[b],) if drifts is not None else u), vth) for b, (n, u, vth) in enumerate(f0.beams)]
    return O.F0(beams=beams, modes=modes)


def test_f0_gradient_matches_fd_of_c_f0():
    f0 = O.F0(beams=[(0.4, (1.2,), (0.7,)), (0.6, (-0.4,), (1.3,))], modes=[(1, 0.03, 0.2), (3, 0.02, -1.0)])
    Lx = 7.0
    rng = np.random.default_rng(3)
    x = rng.uniform(0, Lx, 9)
    v = rng.uniform(-3, 3, 9)
    d_amp, d_u = AD.f0_gradient(f0, Lx, x, v)
    h = 1e-6
    for k in range(2):
        for i in range(9):
            ap = [a for (_, a, _) in f0.modes]
            am = list(ap)
            ap[k] += h
            am[k] -= h
            fd = (O.f0_eval(with_theta(f0, amps=ap), 1, Lx, x[i], [v[i]])
                  - O.f0_eval(with_theta(f0, amps=am), 1, Lx, x[i], [v[i]])) / (2 * h)
            assert abs(fd - d_amp[k, i]) < 1e-8 * max(1.0, abs(fd))
    for b in range(2):
        for i in range(9):
            up = [u[0] for (_, u, _) in f0.beams]
            um = list(up)
            up[b] += h
            um[b] -= h
            fd = (O.f0_eval(with_theta(f0, drifts=up), 1, Lx, x[i], [v[i]])
                  - O.f0_eval(with_theta(f0, drifts=um), 1, Lx, x[i], [v[i]])) / (2 * h)
            assert abs(fd - d_u[b, i]) < 1e-8 * max(1.0, abs(fd))


@pytest.mark.parametrize("softening", [True, False])
def test_poisson_operator_is_antisymmetric(softening):
    """<P a, b> = -<a, P b>: the transpose the backward pass uses."""
    rng = np.random.default_rng(5)
    for nx in (16, 15):
        a, b = rng.normal(size=nx), rng.normal(size=nx)
        Pa = O.poisson(nx, 3.3, 1.0, softening, a)
        Pb = O.poisson(nx, 3.3, 1.0, softening, b)
        assert abs(Pa @ b + a @ Pb) < 1e-13 * np.linalg.norm(Pa) * np.linalg.norm(b)


def fd_gradient(species, f0s, lattices, h, jitter=1.0, nsteps=NSTEPS):
    f0 = f0s[0]
    amps = [a for (_, a, _) in f0.modes]
    drifts = [u[0] for (_, u, _) in f0.beams]
    out = []
    for k in range(len(amps)):
        vals = []
        for sgn in (1, -1):
            a = list(amps)
            a[k] += sgn * h
            vals.append(AD.field_energy(NX, L, DT, species, [with_theta(f0, amps=a)] + f0s[1:], lattices,
                                        SEED, jitter, nsteps))
        out.append((vals[0] - vals[1]) / (2 * h))
    for b in range(len(drifts)):
        vals = []
        for sgn in (1, -1):
            d = list(drifts)
            d[b] += sgn * h
            vals.append(AD.field_energy(NX, L, DT, species, [with_theta(f0, drifts=d)] + f0s[1:], lattices,
                                        SEED, jitter, nsteps))
        out.append((vals[0] - vals[1]) / (2 * h))
    return np.array(out)


def test_adjoint_matches_central_differences():
    """Gradient of J with respect to two mode amplitudes and two beam drifts
    of the electrons (an immobile, perturbed ion background present) against
    central differences of the oracle's forward run at h = 1e-6 and h / 2."""
    species, f0s, lattices = two_stream_small()
    J, g_amp, g_u, _ = AD.field_energy_gradient(NX, L, DT, species, f0s, lattices, SEED, 1.0, 0, NSTEPS)
    J0 = AD.field_energy(NX, L, DT, species, f0s, lattices, SEED, 1.0, NSTEPS)
    assert J == pytest.approx(J0, rel=1e-14)
    g = np.concatenate([g_amp, g_u])
    scale = np.max(np.abs(g))
    for h in (1e-6, 5e-7):
        fd = fd_gradient(species, f0s, lattices, h)
        assert np.max(np.abs(fd - g)) < 1e-6 * scale, (h, fd, g)


def test_adjoint_linear_regime_quadratic():
    """Unjittered lattice, one Maxwellian, one small mode: E vanishes at
    amp = 0 and J = c amp^2 + O(amp^3), so amp dJ/damp = 2 J up to O(amp)."""
    species = [O.Species(q=-1.0, m=1.0, nv=(24,), vmin=(-5.0,), vmax=(5.0,))]
    for amp in (1e-3, 5e-4):
        f0s = [O.F0(beams=[(1.0, (0.0,), (1.0,))], modes=[(1, amp, 0.0)])]
        J, g_amp, _, _ = AD.field_energy_gradient(NX, L, DT, species, f0s, [(2, 2, 1, 1)], SEED, 0.0, 0, NSTEPS)
        assert J > 0
        assert amp * g_amp[0] == pytest.approx(2 * J, rel=20 * amp)
