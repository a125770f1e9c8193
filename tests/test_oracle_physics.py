"""Whole-step pins of the oracle: linear plasma theory and conservation.

The oracle strings together push, reconstruction (Eq. 4), moment (Eq. 14)
and Poisson (Eq. 6) in the order of Fig. 2.  A dropped term, a wrong sign or
a transposed index anywhere in that chain changes the Langmuir frequency, the
Landau damping rate or the two-stream growth rate, all of which are fixed by
the roots of the plasma dispersion function computed independently here.
"""
import os

import numpy as np
import pytest
from scipy.optimize import curve_fit

from oracle import oracle as O
import plasma_theory as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _landau_series(nx, nv, L, vmax, lattice, amp, dt, nsteps, seed):
    sp = O.Species(q=-1.0, m=1.0, nv=(nv,), vmin=(-vmax,), vmax=(vmax,))
    sim = O.OracleSim(1, nx, L, dt, [sp])
    sim.init_markers(0, lattice, O.F0(beams=[(1.0, (0.0,), (1.0,))], modes=[(1, amp, 0.0)]),
                     seed=seed, jitter=1.0)
    sim.refresh()
    i = np.arange(nx)
    ph = np.exp(-2j * np.pi * i / nx)
    c = [np.sum(sim.E * ph)]
    d0 = sim.diag()
    for _ in range(nsteps):
        sim.step()
        c.append(np.sum(sim.E * ph))
    return np.arange(nsteps + 1) * dt, np.array(c) * 2 / nx, d0, sim.diag()


def _fit_damped_wave(t, c, t0, t1):
    """Least-squares fit of the standing wave A cos(w t + p) exp(g t) to the
    mode-1 Fourier coefficient projected on its own phase."""
    k0 = np.argmax(np.abs(c))
    r = np.real(c * np.conj(c[k0] / abs(c[k0])))
    sel = (t >= t0) & (t <= t1)

    def model(t, A, w, p, g):
        return A * np.cos(w * t + p) * np.exp(g * t)

    best = None
    for p in np.linspace(0, 2 * np.pi, 8, endpoint=False):
        try:
            popt, _ = curve_fit(model, t[sel], r[sel], p0=[abs(c[k0]), 1.3, p, -0.1], maxfev=20000)
        except RuntimeError:
            continue
        res = np.sum((model(t[sel], *popt) - r[sel]) ** 2)
        if best is None or res < best[0]:
            best = (res, popt)
    return best[1][1], best[1][3]


def test_landau_damping_k05_against_dispersion_root():
    """Landau workload of 64 x 128 cells, 4 markers per cell (32768), L = 4 pi,
    v in [-6, 6], alpha = 0.01, dt = 0.1, 200 steps.  The root of the
    Maxwellian dispersion function at k = 0.5 is omega = 1.4157,
    gamma = -0.1534; fit over t in [1.5, 18] (Sec. 4.2's window, clipped to
    the run).  Tolerances: 1 % on omega, 5 % on gamma (finite dv, dx, dt and
    marker noise; measured 0.2 % and 1.8 %)."""
    t, c, d0, d1 = _landau_series(64, 128, 4 * np.pi, 6.0, (2, 2, 1, 1), 0.01, 0.1, 200, seed=1804039011)
    w, g = _fit_damped_wave(t, c, 1.5, 18.0)
    root = P.landau_root(0.5)
    assert abs(root.real - 1.41566) < 1e-4 and abs(root.imag + 0.15336) < 1e-4
    assert w == pytest.approx(root.real, rel=0.01)
    assert g == pytest.approx(root.imag, rel=0.05)
    # conservation over the run (measured: N 3.5e-5, total energy 2.0e-5)
    assert abs(d1[4] - d0[4]) / d0[4] < 1e-4
    assert abs(d1[2] - d0[2]) / d0[2] < 1e-4


def test_paper_landau_k04_fit():
    """The paper's own Landau run (Sec. 4.2: k = 0.4, L = 5 pi, alpha = 0.05,
    dt = 0.1, v_range = 10 v_th), here at 64 x 256 cells: the fitted damping
    rate over the paper's window t in [1.5, 25] matches the printed fit
    gamma = -0.070 within 5 % (measured -0.0711); the frequency matches the
    exact dispersion root (1.285) within 1 %."""
    gold = {}
    for line in open(os.path.join(GOLDEN, "landau_k04_paper.txt")):
        if line.strip() and not line.startswith("#"):
            key, val = line.split()[:2]
            gold[key] = float(val)
    # the printed frequency and phase speed follow from the Langmuir relation Eq. 16
    wbg = np.sqrt(1 + 3 * 0.4 ** 2)
    assert round(wbg, 2) == gold["omega_bohm_gross"]
    assert round(wbg / 0.4, 2) == gold["phase_velocity"]
    t, c, _, _ = _landau_series(64, 256, 5 * np.pi, 10.0, (2, 2, 1, 1), 0.05, 0.1, 250, seed=11)
    w, g = _fit_damped_wave(t, c, gold["fit_t_start"], gold["fit_t_end"])
    assert g == pytest.approx(gold["gamma_fit"], rel=0.05)
    assert w == pytest.approx(P.landau_root(0.4).real, rel=0.01)


def test_two_stream_growth_rate():
    """Two counter-drifting beams (+-3 v_th, half density each), mode 1 at
    k = 0.2, 32 x 256 cells over [-10, 10], 4 markers per cell, dt = 0.05,
    seed amplitude 1e-4.  Growth of |E_1| over t in [15, 25] against the
    purely growing dispersion root 0.2845 within 5 % (measured 0.2846)."""
    k = 0.2
    L = 2 * np.pi / k
    sp = O.Species(q=-1.0, m=1.0, nv=(256,), vmin=(-10.0,), vmax=(10.0,))
    sim = O.OracleSim(1, 32, L, 0.05, [sp])
    f0 = O.F0(beams=[(0.5, (3.0,), (1.0,)), (0.5, (-3.0,), (1.0,))], modes=[(1, 1e-4, 0.0)])
    sim.init_markers(0, (2, 2, 1, 1), f0, seed=7, jitter=1.0)
    sim.refresh()
    amps = [P.mode_amplitude(sim.E, 1)]
    for _ in range(500):
        sim.step()
        amps.append(P.mode_amplitude(sim.E, 1))
    t = np.arange(len(amps)) * 0.05
    sel = (t >= 15) & (t <= 25)
    growth = np.polyfit(t[sel], np.log(np.array(amps)[sel]), 1)[0]
    assert growth == pytest.approx(P.two_stream_root(k).imag, rel=0.05)


def test_uniform_maxwellian_lattice_has_no_field():
    """An unperturbed Maxwellian on an unjittered lattice is uniform in x and
    stays so: every cell sees the same markers shifted alike, E is roundoff."""
    sp = O.Species(q=-1.0, m=1.0, nv=(32,), vmin=(-5.0,), vmax=(5.0,))
    sim = O.OracleSim(1, 16, 8.0, 0.1, [sp])
    sim.init_markers(0, (2, 2, 1, 1), O.F0(beams=[(1.0, (0.0,), (1.0,))]), seed=3, jitter=0.0)
    sim.refresh()
    for _ in range(20):
        sim.step()
        assert np.max(np.abs(sim.E)) < 1e-13


def test_two_species_neutral_plasma_has_no_field():
    """Electrons and ions with identical unperturbed density profiles cancel
    in rho (Eq. 14), so E vanishes even with jitter."""
    el = O.Species(q=-1.0, m=1.0, nv=(16,), vmin=(-5.0,), vmax=(5.0,))
    io = O.Species(q=1.0, m=1836.0, nv=(16,), vmin=(-5.0,), vmax=(5.0,))
    sim = O.OracleSim(1, 8, 4.0, 0.1, [el, io])
    f0 = O.F0(beams=[(1.0, (0.0,), (1.0,))], modes=[(1, 0.1, 0.0)])
    sim.init_markers(0, (2, 2, 1, 1), f0, seed=5, jitter=1.0)
    sim.init_markers(1, (2, 2, 1, 1), f0, seed=5, jitter=1.0)
    # same seed, different species index: different jitter, so copy electrons' markers
    sim.set_markers(1, sim.x[0], sim.v[0], sim.fl[0])
    sim.refresh()
    assert np.max(np.abs(sim.rho)) < 1e-14
    assert np.max(np.abs(sim.E)) < 1e-14


@pytest.mark.slow
def test_two_stream_config_geometry_growth_of_modes_5_to_9():
    """The two-stream workload's own geometry (L = 0.4 nx = 204.8 with
    nx = 512, beams at +-3 v_th of half density, mobile ions of mass 1836,
    modes 1-16 seeded at 1e-4 with random phases, dt = 0.05), with fewer
    markers than the benchmark (nv = 256 instead of 1024; 2 x 2 electrons and
    2 x 1 ions per cell).  The growth of |E_m| fitted over t in [8, 20] for
    the modes 5-9 (k = 0.153 ... 0.276, around the fastest mode 7) matches
    the purely growing root of the two-beam dispersion relation within 10 %
    (measured at most 9 % with 4 x 4 ions; the root table: 0.266, 0.281,
    0.285, 0.277, 0.259)."""
    from paper_1804_03901_gb300 import inputs
    w = inputs.two_stream(nv=256, lattice=(2, 2, 1, 1))
    w["lattice"][1] = (2, 1, 1, 1)
    sim = O.OracleSim(1, w["nx"], w["L"], w["dt"], [O.Species(**s) for s in w["species"]])
    for s, (f0, la) in enumerate(zip(w["f0"], w["lattice"])):
        sim.init_markers(s, la, O.F0(f0["beams"], f0["modes"]), w["seed"], w["jitter"])
    sim.refresh()
    Es = [sim.E.copy()]
    for _ in range(400):
        sim.step()
        Es.append(sim.E.copy())
    t = np.arange(len(Es)) * w["dt"]
    sel = (t >= 8.0) & (t <= 20.0)
    for m in range(5, 10):
        k = 2 * np.pi * m / w["L"]
        a = np.array([P.mode_amplitude(E, m) for E in Es])
        growth = np.polyfit(t[sel], np.log(a[sel]), 1)[0]
        assert growth == pytest.approx(P.two_stream_root(k).imag, rel=0.10), (m, growth)
