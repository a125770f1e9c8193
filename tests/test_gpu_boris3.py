"""GPU parity of the magnetized 1d3v path (Boris push with a static
background magnetic field, Sec. 3.2) through the C ABI against the FP64
oracle.

Tolerances as in the field-free 1d3v tests (relative L2 over the grid, per
step from identical states): FP64 1e-10, FP32 1e-5.  Markers are matched
by their (distinct) values.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1804_03901_gb300 import inputs

from test_gpu_parity3 import TOL, compare_grids, compare_markers, make_pair, rel, species2, sync_oracle_to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_03901_gb300 import build
    build.build()
    from paper_1804_03901_gb300 import avl
    return avl


def set_b(sim, orc, B):
    sim.set_bfield(B)
    orc.B = np.asarray(B, dtype=np.float64)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("nx,nv,n,B", [(16, (8, 6, 5), 20011, (0.3, -0.9, 1.4)),
                                       (12, (4, 3, 7), 3001, (0.0, 0.0, 2.0)),
                                       (256, (6, 4, 4), 40000, (1.5, 0.0, 0.0)),
                                       (300, (5, 3, 3), 9001, (0.0, -3.0, 0.5)),
                                       (4, (2, 2, 2), 9, (0.2, 0.2, 0.2))])
def test_boris_step_parity_random_markers(A, prec, nx, nv, n, B):
    """Random 1d3v states (beyond the velocity grid in every component) of two
    species with different charge-to-mass ratios and grids; B along one axis,
    two axes or all three; three steps, each from identical states, with the
    markers (turned velocities, new positions) compared too."""
    L, dt = 7.3, 0.07
    species = species2(nv)
    sim, orc = make_pair(A, nx, L, dt, species, prec)
    for s, sp in enumerate(species):
        x, v, f = inputs.random_markers3(100 * nx + s, n, L, sp["vmin"], sp["vmax"])
        sim.set_markers(s, x, v, f)
    set_b(sim, orc, B)
    dx = L / nx
    for k in range(3):
        sync_oracle_to_gpu(sim, orc)
        sim.step(1)
        orc.step(1)
        compare_grids(sim, orc, TOL[prec], f"step {k}")
        compare_markers(sim, orc, 1e-12 * L if prec == 0 else 2e-6 * dx, 1e-12 if prec == 0 else 1e-5, L)
    st = sim.get_stats()
    assert np.all(st[:, 1] == 3), st      # every magnetized step re-sorts every mobile species
    sim.synchronize()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_boris_free_run_from_lattice(A, prec):
    """Maxwellian electrons with a density ripple in B = B_z (the geometry of
    electron Bernstein waves, Sec. 4.4) over an immobile ion background: a
    free run of 10 steps from the same jittered lattice, E compared every step
    (the two runs drift apart only by rounding)."""
    nx, L, dt = 32, 2 * math.pi / 0.4, 0.1
    species = [dict(q=-1.0, m=1.0, nv=(8, 8, 6), vmin=(-4.0,) * 3, vmax=(4.0,) * 3),
               dict(q=1.0, m=1836.0, nv=(2, 2, 2), vmin=(-0.1,) * 3, vmax=(0.1,) * 3, mobile=False)]
    f0e = dict(beams=[(1.0, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))], modes=[(1, 0.05, 0.0), (3, 0.02, 1.0)])
    f0i = dict(beams=[(1.0, (0.0, 0.0, 0.0), (0.02, 0.02, 0.02))])
    sim, orc = make_pair(A, nx, L, dt, species, prec)
    lat = [(2, 1, 1, 2), (1, 1, 1, 1)]
    for s, f0 in enumerate((f0e, f0i)):
        sim.init_markers(s, lat[s], A.make_f0(**f0), 7, 0.5)
        orc.init_markers(s, lat[s], O.F0(**f0), 7, 0.5)
    orc.refresh()
    set_b(sim, orc, (0.0, 0.0, 0.8))
    for k in range(10):
        sim.step(1)
        orc.step(1)
        tol = 1e-9 if prec == 0 else 2e-4
        assert rel(sim.get_E(), orc.E) < tol, (k, rel(sim.get_E(), orc.E))
    d = sim.get_diag()
    assert np.all(np.isfinite(d))
    sim.synchronize()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_boris_on_then_off(A, prec):
    """Switching B on mid-run (from a layout with markers off their segment
    rows after field-free steps) and off again (back to the field-free push
    from the globally re-sorted layout); parity holds throughout."""
    nx, nv, n, L, dt = 32, (10, 4, 4), 30000, 3.0, 0.2
    species = [dict(q=-4.0, m=1.0, nv=nv, vmin=(-3.0, -2.0, -2.0), vmax=(3.0, 2.0, 2.0))]
    sim, orc = make_pair(A, nx, L, dt, species, prec)
    x, v, f = inputs.random_markers3(9, n, L, species[0]["vmin"], species[0]["vmax"])
    sim.set_markers(0, x, v, f)
    for k, B in enumerate([(0, 0, 0), (0, 0, 0), (0.5, 1.0, 0.0), (0.5, 1.0, 0.0), (0, 0, 0), (0, 0, 0)]):
        set_b(sim, orc, B)
        sync_oracle_to_gpu(sim, orc)
        sim.step(1)
        orc.step(1)
        compare_grids(sim, orc, TOL[prec], f"step {k} B {B}")
    sim.synchronize()


def test_boris_errors(A):
    dom = A.make_domain(1, 16, 1.0, 0.1, 1.0, True, A.AVL_FP64)
    sim = A.Simulation(dom, [A.make_species(-1.0, 1.0, (8,), (-1,), (1,))])
    with pytest.raises(A.AvlError):
        sim.set_bfield((0.0, 0.0, 1.0))     # 1d1v has no magnetic field
    dom = A.make_domain(3, 16, 1.0, 0.1, 1.0, True, A.AVL_FP32)
    sim = A.Simulation(dom, [A.make_species(-1.0, 1.0, (4, 4, 4), (-1, -1, -1), (1, 1, 1))])
    with pytest.raises(A.AvlError):
        sim.set_bfield((0.0, math.inf, 1.0))
    sim.set_bfield((0.0, 0.0, 1.0))
    sim.init_markers(0, (1, 1, 1, 1), A.make_f0([(1.0, (0, 0, 0), (1, 1, 1))]), 1)
    sim.step(2)
    sim.synchronize()
