"""GPU marker refinement by tracing back to the initial state (Sec. 2)
through the C ABI (avl_record_history, avl_refine_markers) against the
oracle's refinement (orc_refine_markers) run on the GPU's own field history.

Tolerances as in the other 1d1v parity tests (relative L2 over the grids):
FP64 1e-10, FP32 1e-5.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

NX, L, DT, SEED = 32, 4 * math.pi, 0.1, 7
TOL = {0: 1e-10, 1: 1e-5}
SPECIES = [dict(q=-1.0, m=1.0, nv=(48,), vmin=(-5.0,), vmax=(5.0,)),
           dict(q=1.0, m=100.0, nv=(8,), vmin=(-0.5,), vmax=(0.5,), mobile=False)]
F0 = [dict(beams=[(0.5, (1.5,), (0.6,)), (0.5, (-1.5,), (0.6,))], modes=[(1, 0.05, 0.3), (2, 0.02, 1.1)]),
      dict(beams=[(1.0, (0.0,), (0.1,))], modes=[])]


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


def start(A, prec, nsteps, history=True):
    dom = A.make_domain(1, NX, L, DT, 1.0, True, prec)
    sim = A.Simulation(dom, [A.make_species(**sp) for sp in SPECIES])
    if history:
        sim.record_history(nsteps + 4)
    for s in range(2):
        sim.init_markers(s, (2, 2, 1, 1) if s == 0 else (1, 1, 1, 1), A.make_f0(**F0[s]), SEED, 1.0)
    hist = [sim.get_E()]
    for _ in range(nsteps):
        sim.step(1)
        hist.append(sim.get_E())
    return sim, np.array(hist)


@pytest.mark.parametrize("prec,nsteps,box,lat", [(0, 20, (5, 13, 10, 30), (2, 3)), (0, 0, (0, 32, 0, 48), (1, 1)),
                                                (1, 20, (5, 13, 10, 30), (2, 3)), (0, 35, (20, 32, 0, 17), (3, 1))],
                         ids=["fp64", "fp64-no-steps", "fp32", "fp64-seam-and-edge"])
def test_refine_matches_oracle(A, prec, nsteps, box, lat):
    """New markers in a box of cells after nsteps steps: their number, their
    values (f0 at the traced-back foot) and the grids of the enlarged set."""
    sim, hist = start(A, prec, nsteps)
    x_old, v_old, f_old = sim.get_markers(0)
    x_ion, v_ion, f_ion = sim.get_markers(1)
    added = sim.refine_markers(0, box, lat, 123)
    xr, vr, fr = O.refine_markers(NX, L, O.Species(**SPECIES[0]), box, lat, O.F0(**F0[0]), 0, 123, 1.0, DT,
                                  hist[:nsteps])
    assert added == xr.size
    assert sim.marker_count(0) == x_old.size + added
    # the GPU's marker values are the old ones and the oracle's new ones
    x_new, v_new, f_new = sim.get_markers(0)
    want_f = np.concatenate([f_old, fr.astype(np.float32).astype(np.float64) if prec else fr])
    np.testing.assert_allclose(np.sort(f_new), np.sort(want_f), rtol=1e-12 if prec == 0 else 1e-6, atol=0)
    # grids of the enlarged marker set
    orc = O.OracleSim(1, NX, L, DT, [O.Species(**sp) for sp in SPECIES])
    orc.set_markers(0, x_new, v_new, f_new)
    orc.set_markers(1, x_ion, v_ion, f_ion)
    orc.refresh()
    f, n = sim.get_f(0, with_n=True)
    assert rel(f, orc.f[0]) < TOL[prec] and rel(n, orc.den[0]) < TOL[prec]
    assert rel(sim.get_E(), orc.E) < TOL[prec]
    # the refined markers against the oracle's, paired by value (FP64): the
    # old markers are exact copies, the new ones agree to rounding
    if prec == 0:
        sel = ~np.isin(f_new, f_old)
        assert sel.sum() == fr.size
        i1, i2 = np.argsort(f_new[sel]), np.argsort(fr)
        np.testing.assert_allclose(x_new[sel][i1], xr[i2], rtol=0, atol=1e-12 * L)
        np.testing.assert_allclose(v_new[0][sel][i1], vr[0][i2], rtol=0, atol=1e-12)
    # one more step from identical states
    sim.step(1)
    orc.step(1)
    assert rel(sim.get_E(), orc.E) < 10 * TOL[prec]
    sim.synchronize()


def test_refine_twice_and_errors(A):
    sim, hist = start(A, 0, 10)
    a1 = sim.refine_markers(0, (0, 4, 0, 10), (1, 1), 5)
    sim.step(3)
    a2 = sim.refine_markers(0, (4, 8, 0, 10), (2, 1), 6)   # traced back through 13 steps
    assert (a1, a2) == (40, 80)
    with pytest.raises(A.AvlError):
        sim.refine_markers(0, (0, 33, 0, 10), (1, 1), 5)     # box beyond the grid
    with pytest.raises(A.AvlError):
        sim.refine_markers(0, (0, 4, 0, 10), (0, 1), 5)
    x, v, f = sim.get_markers(1)
    sim.set_markers(1, x, v, f)
    with pytest.raises(A.AvlError):
        sim.refine_markers(1, (0, 4, 0, 4), (1, 1), 5)       # caller markers: no f0 to trace to
    sim2, _ = start(A, 0, 3, history=False)
    with pytest.raises(A.AvlError):
        sim2.refine_markers(0, (0, 4, 0, 10), (1, 1), 5)     # no field history
    sim.synchronize()
