"""GPU adjoint (avl_adjoint) against the oracle's discrete adjoint and
against central finite differences of the GPU's own forward run (avl_step).

Tolerances: FP64 J within 1e-10 and the gradient within 1e-8 (relative to
its largest component) of the oracle; FP32 within 2e-3; finite differences
of the FP64 forward at h = 1e-6 within 1e-6.
"""
import math

import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import oracle as O

pytestmark = pytest.mark.gpu

NX, L, DT, SEED = 16, 10.0, 0.1, 11


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_03901_gb300 import build
    build.build()
    from paper_1804_03901_gb300 import avl
    return avl


def problem(amps=(0.02, 0.01), u=1.5):
    species = [dict(q=-1.0, m=1.0, nv=(24,), vmin=(-5.0,), vmax=(5.0,), mobile=True),
               dict(q=1.0, m=100.0, nv=(8,), vmin=(-0.5,), vmax=(0.5,), mobile=False)]
    f0s = [dict(beams=[(0.5, (u,), (0.6,)), (0.5, (-u,), (0.6,))], modes=[(1, amps[0], 0.3), (2, amps[1], 1.1)]),
           dict(beams=[(1.0, (0.0,), (0.1,))], modes=[(1, 0.005, 0.0)])]
    lattices = [(2, 2, 1, 1), (1, 1, 1, 1)]
    return species, f0s, lattices


def make_sim(A, prec, species, f0s, lattices, jitter=1.0):
    dom = A.make_domain(1, NX, L, DT, 1.0, True, prec)
    sim = A.Simulation(dom, [A.make_species(**sp) for sp in species])
    for s in range(len(species)):
        sim.init_markers(s, lattices[s], A.make_f0(**f0s[s]), SEED, jitter)
    return sim


def oracle_gradient(species, f0s, lattices, nsteps, jitter=1.0):
    osp = [O.Species(**sp) for sp in species]
    of0 = [O.F0(**f) for f in f0s]
    J, ga, gu, _ = AD.field_energy_gradient(NX, L, DT, osp, of0, lattices, SEED, jitter, 0, nsteps)
    return J, np.concatenate([ga, gu])


@pytest.mark.parametrize("prec,nsteps,ckpt", [(0, 25, 7), (0, 25, 25), (0, 0, 1), (1, 25, 7)],
                         ids=["fp64-k7", "fp64-k25", "fp64-0steps", "fp32-k7"])
def test_adjoint_matches_oracle(A, prec, nsteps, ckpt):
    species, f0s, lattices = problem()
    sim = make_sim(A, prec, species, f0s, lattices)
    J, ga, gu = sim.adjoint(0, A.make_f0(**f0s[0]), nsteps, ckpt)
    Jo, go = oracle_gradient(species, f0s, lattices, nsteps)
    g = np.concatenate([ga, gu])
    tolJ, tolg = (1e-10, 1e-8) if prec == 0 else (2e-3, 2e-3)
    assert J == pytest.approx(Jo, rel=tolJ)
    assert np.max(np.abs(g - go)) < tolg * np.max(np.abs(go)), (g, go)
    sim.synchronize()


def test_checkpoint_interval_does_not_change_the_gradient(A):
    species, f0s, lattices = problem()
    sim = make_sim(A, 0, species, f0s, lattices)
    th = A.make_f0(**f0s[0])
    ref = None
    for k in (1, 4, 25, 100):
        J, ga, gu = sim.adjoint(0, th, 25, k)
        g = np.concatenate([[J], ga, gu])
        if ref is None:
            ref = g
        assert np.max(np.abs(g - ref)) < 1e-12 * np.max(np.abs(ref)), k


def test_adjoint_matches_finite_differences_of_the_forward(A):
    """Central differences of J from the library's own FP64 forward run
    (avl_init_markers + avl_step + avl_get_E) at h = 1e-6."""
    species, f0s, lattices = problem()
    nsteps, h = 25, 1e-6
    sim = make_sim(A, 0, species, f0s, lattices)
    J, ga, gu = sim.adjoint(0, A.make_f0(**f0s[0]), nsteps, 10)
    g = np.concatenate([ga, gu])

    def J_of(amps, drifts):
        f = dict(f0s[0])
        f["modes"] = [(m, amps[k], ph) for k, (m, _, ph) in enumerate(f0s[0]["modes"])]
        f["beams"] = [(n, (drifts[b],), vth) for b, (n, _, vth) in enumerate(f0s[0]["beams"])]
        s2 = make_sim(A, 0, species, [f] + f0s[1:], lattices)
        s2.step(nsteps)
        E = s2.get_E()
        s2.close()
        return 0.5 * float(np.sum(E ** 2)) * (L / NX)

    amps = [a for (_, a, _) in f0s[0]["modes"]]
    drifts = [u[0] for (_, u, _) in f0s[0]["beams"]]
    assert J == pytest.approx(J_of(amps, drifts), rel=1e-10)
    fd = []
    for k in range(len(amps)):
        ap, am = list(amps), list(amps)
        ap[k] += h
        am[k] -= h
        fd.append((J_of(ap, drifts) - J_of(am, drifts)) / (2 * h))
    for b in range(len(drifts)):
        dp, dm = list(drifts), list(drifts)
        dp[b] += h
        dm[b] -= h
        fd.append((J_of(amps, dp) - J_of(amps, dm)) / (2 * h))
    fd = np.array(fd)
    assert np.max(np.abs(fd - g)) < 1e-6 * np.max(np.abs(g)), (fd, g)


def test_autograd_function(A):
    torch = pytest.importorskip("torch")
    from paper_1804_03901_gb300.autograd import FieldEnergy
    species, f0s, lattices = problem()
    sim = make_sim(A, 0, species, f0s, lattices)
    amps = torch.tensor([a for (_, a, _) in f0s[0]["modes"]], dtype=torch.float64, requires_grad=True)
    drifts = torch.tensor([u[0] for (_, u, _) in f0s[0]["beams"]], dtype=torch.float64, requires_grad=True)
    J = FieldEnergy.apply(amps, drifts, sim, 0, f0s[0], 25, 7)
    (3.0 * J).backward()
    J2, ga, gu = sim.adjoint(0, A.make_f0(**f0s[0]), 25, 7)
    assert float(J.detach()) == pytest.approx(J2, rel=1e-12)
    np.testing.assert_allclose(amps.grad.numpy(), 3.0 * ga, rtol=1e-12)
    np.testing.assert_allclose(drifts.grad.numpy(), 3.0 * gu, rtol=1e-12)


def test_adjoint_errors(A):
    species, f0s, lattices = problem()
    dom = A.make_domain(1, NX, L, DT, 1.0, True, A.AVL_FP64)
    sim = A.Simulation(dom, [A.make_species(**sp) for sp in species])
    sim.init_markers(0, lattices[0], A.make_f0(**f0s[0]), SEED, 1.0)
    rng = np.random.default_rng(1)
    sim.set_markers(1, rng.uniform(0, L, 50), rng.uniform(-0.4, 0.4, 50), rng.uniform(0.1, 1, 50))
    with pytest.raises(A.AvlError):       # species 1 came from caller arrays
        sim.adjoint(0, A.make_f0(**f0s[0]), 5, 2)
    sim.init_markers(1, lattices[1], A.make_f0(**f0s[1]), SEED, 1.0)
    with pytest.raises(A.AvlError):
        sim.adjoint(0, A.make_f0(**f0s[0]), 5, 0)
    sim.adjoint(0, A.make_f0(**f0s[0]), 5, 2)
    sim.synchronize()


_CONFIG4 = {}


def _config4_oracle(nsteps):
    """The oracle adjoint of the two-stream adjoint workload at its full size
    (nx = 256, nv = 512, 2 x 4 markers per cell: 1048576 electrons and as
    many immobile ions, 16 mode amplitudes and 2 beam drifts), over nsteps
    steps (all states held in memory)."""
    if nsteps not in _CONFIG4:
        from paper_1804_03901_gb300 import inputs
        w = inputs.two_stream_adjoint()
        osp = [O.Species(**sp) for sp in w["species"]]
        of0 = [O.F0(f["beams"], f["modes"]) for f in w["f0"]]
        J, ga, gu, _ = AD.field_energy_gradient(w["nx"], w["L"], w["dt"], osp, of0, w["lattice"], w["seed"],
                                                w["jitter"], 0, nsteps)
        _CONFIG4[nsteps] = (w, J, np.concatenate([ga, gu]))
    return _CONFIG4[nsteps]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_adjoint_matches_oracle_at_config4_size(A, prec):
    """FP64: J within 1e-10 and the gradient within 1e-8 of the oracle
    adjoint (relative to its largest component) at the workload's full size
    over 30 steps with checkpoints every 10; FP32: the same comparison, its
    error printed (stated in the design notes) and held to 2e-3."""
    nsteps, ckpt = 30, 10
    w, Jo, go = _config4_oracle(nsteps)
    dom = A.make_domain(1, w["nx"], w["L"], w["dt"], 1.0, True, prec)
    sim = A.Simulation(dom, [A.make_species(**sp) for sp in w["species"]])
    for s, (f0, lat) in enumerate(zip(w["f0"], w["lattice"])):
        sim.init_markers(s, lat, A.make_f0(f0["beams"], f0["modes"]), w["seed"], w["jitter"])
    f0 = w["f0"][0]
    J, ga, gu = sim.adjoint(0, A.make_f0(f0["beams"], f0["modes"]), nsteps, ckpt)
    sim.close()
    g = np.concatenate([ga, gu])
    errJ = abs(J - Jo) / abs(Jo)
    errg = float(np.max(np.abs(g - go)) / np.max(np.abs(go)))
    print(f"config-4 size adjoint ({'fp64' if prec == 0 else 'fp32'}): J rel err {errJ:.2e}, "
          f"gradient rel err {errg:.2e}")
    tolJ, tolg = (1e-10, 1e-8) if prec == 0 else (2e-3, 2e-3)
    assert errJ < tolJ
    assert errg < tolg


def test_adjoint_matches_finite_differences_at_config4_size(A):
    """The two-stream adjoint workload at full size (1048576 electrons,
    nx = 256, nv = 512, 16 mode amplitudes and 2 beam drifts): the FP64
    adjoint against central differences of the library's FP64 forward run
    at h = 1e-10, over 100 steps (linear phase) and the full 500 steps
    (T = 25, checkpoints every 50).  The differences carry an O(h) error of
    their own from markers crossing cloud-in-cell kinks (it sets the 1e-5
    disagreement at h = 1e-6) and a roundoff error O(eps J / h) that takes
    over below h = 1e-10.  Measured: 1.6e-7 (100 steps) and 1.0e-6
    (500 steps) relative to the largest component."""
    from paper_1804_03901_gb300 import inputs
    w = inputs.two_stream_adjoint()
    f0 = w["f0"][0]

    def sim_of(f0e):
        dom = A.make_domain(1, w["nx"], w["L"], w["dt"], 1.0, True, A.AVL_FP64)
        sim = A.Simulation(dom, [A.make_species(**sp) for sp in w["species"]])
        for s, (ff, lat) in enumerate(zip([f0e] + w["f0"][1:], w["lattice"])):
            sim.init_markers(s, lat, A.make_f0(ff["beams"], ff["modes"]), w["seed"], w["jitter"])
        return sim

    amps = [a for (_, a, _) in f0["modes"]]
    drifts = [u[0] for (_, u, _) in f0["beams"]]

    def J_of(a, d, n):
        f0e = {"beams": [(nb, (d[b],) + tuple(u[1:]), vth) for b, (nb, u, vth) in enumerate(f0["beams"])],
               "modes": [(m, a[k], ph) for k, (m, _, ph) in enumerate(f0["modes"])]}
        sim = sim_of(f0e)
        sim.step(n)
        E = sim.get_E()
        sim.close()
        return 0.5 * float(np.sum(E ** 2)) * (w["L"] / w["nx"])

    h = 1e-10
    for n, tol in ((100, 1e-6), (500, 1.5e-6)):
        sim = sim_of(f0)
        _, ga, gu = sim.adjoint(0, A.make_f0(f0["beams"], f0["modes"]), n, 50)
        sim.close()
        g = np.concatenate([ga, gu])
        fd = []
        for k in range(len(amps)):
            ap, am = list(amps), list(amps)
            ap[k] += h
            am[k] -= h
            fd.append((J_of(ap, drifts, n) - J_of(am, drifts, n)) / (2 * h))
        for b in range(len(drifts)):
            dp, dm = list(drifts), list(drifts)
            dp[b] += h
            dm[b] -= h
            fd.append((J_of(amps, dp, n) - J_of(amps, dm, n)) / (2 * h))
        err = float(np.max(np.abs(np.array(fd) - g)) / np.max(np.abs(g)))
        print(f"config-4 size adjoint vs central differences (h = 1e-10), {n} steps: {err:.2e}")
        assert err < tol, (n, err)
