"""GPU output moments (avl_get_moments) and field residual (avl_get_residual)
against the oracle's definitions on the same reconstructed state, 1d1v and
1d3v, after a step from random markers.  Tolerances as the parity tests:
FP64 1e-10, FP32 1e-5 relative L2 per row."""
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


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("nvdim", [1, 3])
def test_moments_and_residual_match_oracle(A, prec, nvdim):
    nx, L, dt, cP = 24, 6.1, 0.08, 4 * np.pi
    if nvdim == 1:
        species = [dict(q=-1.0, m=1.0, nv=(40,), vmin=(-3.0,), vmax=(4.0,)),
                   dict(q=0.5, m=9.0, nv=(17,), vmin=(-1.0,), vmax=(1.5,))]
    else:
        species = [dict(q=-1.0, m=1.0, nv=(8, 6, 5), vmin=(-3.0, -2.0, -1.0), vmax=(4.0, 2.0, 1.5)),
                   dict(q=0.5, m=9.0, nv=(5, 4, 4), vmin=(-1.0, -1.0, -1.0), vmax=(1.5, 1.0, 0.5))]
    dom = A.make_domain(nvdim, nx, L, dt, cP, True, prec)
    sim = A.Simulation(dom, [A.make_species(**sp) for sp in species])
    orc = O.OracleSim(nvdim, nx, L, dt, [O.Species(**sp) for sp in species], cP, True)
    for s, sp in enumerate(species):
        if nvdim == 1:
            x, v, f = inputs.random_markers(40 + s, 9000, L, sp["vmin"][0], sp["vmax"][0])
        else:
            x, v, f = inputs.random_markers3(40 + s, 20000, L, sp["vmin"], sp["vmax"])
        sim.set_markers(s, x, v, f)
    sim.step(2)
    for s in range(len(species)):
        x, v, f = sim.get_markers(s)
        orc.set_markers(s, x, v, f)
    orc.refresh()
    for s, sp in enumerate(species):
        m = sim.get_moments(s)
        mo = O.moments(nvdim, nx, L, orc.species[s], orc.f[s])
        assert m.shape == mo.shape == (2 + nvdim, nx)
        for r in range(m.shape[0]):
            assert rel(m[r], mo[r]) < TOL[prec], (s, r, rel(m[r], mo[r]))
    res = sim.get_residual()
    ro = O.field_residual(nx, L, cP, orc.rho, orc.E)
    assert rel(res, ro) < TOL[prec] * 10, rel(res, ro)
    sim.synchronize()
