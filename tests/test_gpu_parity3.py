"""GPU parity of the 1d3v path (three velocity dimensions, no magnetic
field) through the C ABI against the FP64 oracle.

Tolerances (relative L2 over the grid, per step from identical states):
  FP64 path  1e-10 for f, n, rho, E
  FP32 path  1e-5  for f, n, rho, E
Markers are matched by their (distinct) values.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1804_03901_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_03901_gb300 import build
    build.build()
    from paper_1804_03901_gb300 import avl
    return avl


def rel(a, b):
    n = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (n if n > 0 else 1.0)


def make_pair(A, nx, L, dt, species, prec, softening=True, cP=1.0):
    dom = A.make_domain(3, nx, L, dt, cP, softening, prec)
    sim = A.Simulation(dom, [A.make_species(**sp) for sp in species])
    orc = O.OracleSim(3, nx, L, dt, [O.Species(**sp) for sp in species], cP, softening)
    return sim, orc


def sync_oracle_to_gpu(sim, orc):
    for s in range(len(orc.species)):
        if sim.marker_count(s):
            x, v, f = sim.get_markers(s)
            orc.set_markers(s, x, v, f)
    orc.refresh()


def compare_grids(sim, orc, tol, what=""):
    for s in range(len(orc.species)):
        f, n = sim.get_f(s, with_n=True)
        assert f.shape == orc.f[s].shape
        assert rel(f, orc.f[s]) < tol, (what, "f", s, rel(f, orc.f[s]))
        assert rel(n, orc.den[s]) < tol, (what, "n", s, rel(n, orc.den[s]))
    rho, E = sim.get_rho(), sim.get_E()
    assert rel(rho, orc.rho) < tol, (what, "rho", rel(rho, orc.rho))
    assert rel(E, orc.E) < tol, (what, "E", rel(E, orc.E))
    # diagnostics (Sec. 3.4.1): W_E, W_kin, W_total, per species W_kin, N, S
    d, do = sim.get_diag(), orc.diag()
    err = np.abs(d - do) / np.maximum(np.abs(do), 1e-300)
    assert np.all(err < tol), (what, "diag", err)


def compare_markers(sim, orc, tol_x, tol_v, L):
    for s in range(len(orc.species)):
        if not sim.marker_count(s):
            continue
        x, v, f = sim.get_markers(s)
        i1 = np.argsort(f, kind="stable")
        i2 = np.argsort(orc.fl[s], kind="stable")
        np.testing.assert_array_equal(f[i1], orc.fl[s][i2])
        d = (x[i1] - orc.x[s][i2] + L / 2) % L - L / 2
        assert np.max(np.abs(d)) < tol_x, np.max(np.abs(d))
        for k in range(3):
            assert np.max(np.abs(v[k][i1] - orc.v[s][k][i2])) < tol_v, k


def species2(nv):
    return [dict(q=-1.0, m=1.0, nv=nv, vmin=(-3.0, -2.0, -2.5), vmax=(3.0, 2.0, 1.5)),
            dict(q=0.7, m=5.0, nv=(nv[0] // 2 + 3, nv[2], nv[1]), vmin=(-1.0, -1.0, -1.0), vmax=(2.0, 1.0, 1.0))]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("nx,nv,n", [(16, (8, 6, 5), 20011), (12, (4, 3, 7), 3001), (256, (6, 4, 4), 40000),
                                     (300, (5, 3, 3), 9001), (4, (2, 2, 2), 9)])
def test_step_parity_random_markers3(A, prec, nx, nv, n):
    """Random 1d3v marker states (some beyond the velocity grid in every
    component, values over 12 decades), two species of different grids,
    power-of-two (FFT) and other (DFT) x grids, one and two columns per
    thread; set + refresh and three steps, each compared from identical
    states."""
    L, dt = 7.3, 0.07
    species = species2(nv)
    sim, orc = make_pair(A, nx, L, dt, species, prec)
    for s, sp in enumerate(species):
        x, v, f = inputs.random_markers3(100 * nx + s, n, L, sp["vmin"], sp["vmax"])
        sim.set_markers(s, x, v, f)
    sync_oracle_to_gpu(sim, orc)
    compare_grids(sim, orc, TOL[prec], "set")
    dx = L / nx
    for k in range(3):
        sync_oracle_to_gpu(sim, orc)
        sim.step(1)
        orc.step(1)
        compare_grids(sim, orc, TOL[prec], f"step {k}")
        compare_markers(sim, orc, 1e-12 * L if prec == 0 else 2e-6 * dx, 1e-12 if prec == 0 else 1e-5, L)
    sim.synchronize()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_resort_under_strong_field3(A, prec):
    """A strong field moves many markers off their v_x rows every step, so
    the pencils are re-sorted; parity holds through the re-sorts."""
    nx, nv, n, L, dt = 32, (10, 4, 4), 30000, 3.0, 0.2
    species = [dict(q=-4.0, m=1.0, nv=nv, vmin=(-3.0, -2.0, -2.0), vmax=(3.0, 2.0, 2.0))]
    sim, orc = make_pair(A, nx, L, dt, species, prec)
    x, v, f = inputs.random_markers3(5, n, L, species[0]["vmin"], species[0]["vmax"])
    sim.set_markers(0, x, v, f)
    for k in range(6):
        sync_oracle_to_gpu(sim, orc)
        sim.step(1)
        orc.step(1)
        compare_grids(sim, orc, TOL[prec], f"step {k}")
    st = sim.get_stats()
    assert st[0, 1] >= 1, st       # re-sorts happened
    assert st[0, 3] == 6
    sim.synchronize()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_lattice_init_parity3(A, prec):
    """Jittered lattice markers weighted to a bump-on-tail f0 (the generator
    of both sides follows the same definition): grids after creation, then
    a free run of a few steps (FP64: E every step)."""
    wl = inputs.bump_on_tail(nx=16, nv=6)
    wl["L"] = 2 * math.pi / 0.3
    sp = dict(wl["species"][0])
    sp["nv"] = (8, 6, 5)
    species = [sp]
    sim, orc = make_pair(A, wl["nx"], wl["L"], wl["dt"], species, prec)
    f0d = wl["f0"][0]
    lat = (2, 1, 2, 1)
    sim.init_markers(0, lat, A.make_f0(**f0d), wl["seed"], wl["jitter"])
    orc.init_markers(0, lat, O.F0(**f0d), wl["seed"], wl["jitter"])
    orc.refresh()
    assert sim.marker_count(0) == orc.x[0].size
    compare_grids(sim, orc, TOL[prec] if prec == 0 else 2e-6, "init")
    for k in range(5):
        sim.step(1)
        orc.step(1)
        tol = 1e-9 if prec == 0 else 1e-4
        assert rel(sim.get_E(), orc.E) < tol, (k, rel(sim.get_E(), orc.E))
    sim.synchronize()


def test_errors3(A):
    """Argument checks of the 1d3v path."""
    dom = A.make_domain(3, 1024, 1.0, 0.1, 1.0, True, A.AVL_FP64)
    sp = A.make_species(-1.0, 1.0, (4, 4, 4), (-1, -1, -1), (1, 1, 1))
    with pytest.raises(A.AvlError):
        A.Simulation(dom, [sp])
    dom = A.make_domain(3, 16, 1.0, 0.1, 1.0, True, A.AVL_FP32)
    sim = A.Simulation(dom, [sp])
    f0 = A.make_f0([(1.0, (0, 0, 0), (1, 1, 1))])
    with pytest.raises(A.AvlError):
        sim.init_markers(0, (2, 1, 0, 1), f0, 1)
    with pytest.raises(A.AvlError):
        A.Simulation(dom, [A.make_species(-1.0, 1.0, (4, 1, 4), (-1, -1, -1), (1, 1, 1))])
    sim.init_markers(0, (1, 1, 1, 1), f0, 1)
    sim.step(2)
    sim.synchronize()


@pytest.mark.parametrize("prec,nx", [(1, 1024), (0, 512)], ids=["fp32-nx1024", "fp64-nx512"])
def test_step_parity_at_the_largest_nx3(A, prec, nx):
    """The largest x grids of the 1d3v path (FP32 1024: four columns per
    thread; FP64 512: two, with the FP64 gather's shared-memory row planes at
    their largest); one larger is rejected when the context is created."""
    L, dt = 7.3, 0.07
    species = species2((5, 3, 3))
    sim, orc = make_pair(A, nx, L, dt, species, prec)
    for s, sp in enumerate(species):
        x, v, f = inputs.random_markers3(7 * nx + s, 20011, L, sp["vmin"], sp["vmax"])
        sim.set_markers(s, x, v, f)
    for k in range(2):
        sync_oracle_to_gpu(sim, orc)
        sim.step(1)
        orc.step(1)
        compare_grids(sim, orc, TOL[prec], f"nx {nx} step {k}")
    sim.close()
    dom = A.make_domain(3, nx + 1, L, dt, 1.0, True, prec)
    with pytest.raises(A.AvlError) as e:
        A.Simulation(dom, [A.make_species(**species[0])])
    assert e.value.status == A.AVL_EINVAL


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_boundary_positions_and_rows3(A, prec):
    """Markers placed where the cloud-in-cell and the dual velocity rows
    decide a cell: x at 0, at cell edges and centres, one rounding below L;
    velocity components at dual-row boundaries (weight 0 or 1), on the grid's
    first and last rows and just outside it (the FP64 deposit keeps positions
    and rows as fixed-point counts, so these are the cases where its
    rounding could pick another cell).  They sit among random markers that
    give every reached cell a weight well above rounding: a weight that is 0
    in exact arithmetic may come out as 0 or as 2^-52 on either side, and a
    cell reached by such weights alone takes f = num / den = the marker's f
    or 0 (Eq. 4), which no tolerance separates.  Set + refresh and two
    steps, compared with the oracle from identical states."""
    nx, L, dt = 16, 7.3, 0.07
    species = species2((8, 6, 5))
    sim, orc = make_pair(A, nx, L, dt, species, prec)
    dx = L / nx
    for s, sp in enumerate(species):
        xb, vb, fb = inputs.boundary_markers3(77 + s, 1500, nx, L, sp["nv"], sp["vmin"], sp["vmax"])
        xr, vr, fr = inputs.random_markers3(177 + s, 30000, L, sp["vmin"], sp["vmax"], fmin=1e-3)
        sim.set_markers(s, np.concatenate([xb, xr]), np.concatenate([vb, vr], axis=1), np.concatenate([fb, fr]))
    sync_oracle_to_gpu(sim, orc)
    compare_grids(sim, orc, TOL[prec], "set")
    for k in range(2):
        sync_oracle_to_gpu(sim, orc)
        sim.step(1)
        orc.step(1)
        compare_grids(sim, orc, TOL[prec], f"step {k}")
        compare_markers(sim, orc, 1e-12 * L if prec == 0 else 2e-6 * dx, 1e-12 if prec == 0 else 1e-5, L)
    sim.synchronize()
