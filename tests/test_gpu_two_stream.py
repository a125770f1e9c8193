"""Linear theory of the two-stream workload on the GPU (Sec. 4: dispersion
tests), in the benchmarked FP32 production form at full size.

Electrons of two counter-drifting beams (+-3 v_th, half density each) and
mobile ions (m = 1836), nx = 512, L = 204.8, nv = 1024, 4 x 4 markers per
cell (16.8 M markers), modes 1-16 seeded at 1e-4 with random phases,
dt = 0.05.  The growth of |E_m| fitted over t in [8, 20] for the modes 5-9
(k = 0.153 ... 0.276, around the fastest mode 7) matches the purely growing
root of the two-beam dispersion relation (Faddeeva-function roots computed
in plasma_theory) within 10 %, as the oracle does at this geometry
(test_oracle_physics).
"""
import numpy as np
import pytest

from paper_1804_03901_gb300 import inputs

import plasma_theory as P

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


def test_two_stream_full_size_growth_of_modes_5_to_9(A):
    w = inputs.two_stream()
    dom = A.make_domain(1, w["nx"], w["L"], w["dt"], 1.0, True, A.AVL_FP32)
    sim = A.Simulation(dom, [A.make_species(**sp) for sp in w["species"]])
    for s, (f0, lat) in enumerate(zip(w["f0"], w["lattice"])):
        sim.init_markers(s, lat, A.make_f0(f0["beams"], f0["modes"]), w["seed"], w["jitter"])
    Es = [sim.get_E()]
    for _ in range(400):
        sim.step(1)
        Es.append(sim.get_E())
    sim.close()
    t = np.arange(len(Es)) * w["dt"]
    sel = (t >= 8.0) & (t <= 20.0)
    fits = {}
    for m in range(5, 10):
        k = 2 * np.pi * m / w["L"]
        a = np.array([P.mode_amplitude(E, m) for E in Es])
        fits[m] = (np.polyfit(t[sel], np.log(a[sel]), 1)[0], P.two_stream_root(k).imag)
    print({m: f"{g:.4f} vs {th:.4f}" for m, (g, th) in fits.items()})
    for m, (g, th) in fits.items():
        assert g == pytest.approx(th, rel=0.10), (m, g, th)
