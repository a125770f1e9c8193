"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative L2 over the grid, per step from identical states):
  FP64 path  1e-10 for f, n, rho, E
  FP32 path  1e-5  for f, n, rho, E
Marker positions and velocities are matched by their (distinct) values.
"""
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
    dom = A.make_domain(1, nx, L, dt, cP, softening, prec)
    sim = A.Simulation(dom, [A.make_species(**sp) for sp in species])
    orc = O.OracleSim(1, nx, L, dt, [O.Species(**sp) for sp in species], cP, softening)
    return sim, orc


def sync_oracle_to_gpu(sim, orc):
    """Give the oracle the GPU's exact marker state (per-step parity)."""
    for s in range(len(orc.species)):
        if sim.marker_count(s):
            x, v, f = sim.get_markers(s)
            orc.set_markers(s, x, v, f)
    orc.refresh()


def compare_grids(sim, orc, tol, what=""):
    for s in range(len(orc.species)):
        f, n = sim.get_f(s, with_n=True)
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
        assert np.max(np.abs(v[0][i1] - orc.v[s][0][i2])) < tol_v


SPECIES2 = lambda nv: [dict(q=-1.0, m=1.0, nv=(nv,), vmin=(-3.0,), vmax=(3.0,)),
                       dict(q=0.7, m=5.0, nv=(nv // 2 + 3,), vmin=(-1.0,), vmax=(2.0,))]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("nx,nv,n,chunk", [(64, 96, 20011, 1024), (48, 40, 5003, 640), (64, 96, 20011, 0),
                                            (4, 2, 7, 0), (32, 64, 30000, 64), (15, 24, 3001, 0),
                                            (13, 30, 5003, 256)])
def test_step_parity_random_markers(A, monkeypatch, prec, nx, nv, n, chunk):
    """Random marker states (some beyond the velocity grid, values over 12
    decades), many chunks and a ragged last chunk, power-of-two (FFT) and
    other (DFT) grids, odd nx (deposit windows of an odd number of cells,
    padded to 16-byte bulk copies; E staged without the bulk copy); one set +
    refresh and three steps (each re-sorting the markers), each compared from
    identical states."""
    if chunk:
        monkeypatch.setenv("AVL_CHUNK_M", str(chunk))
    L, dt = 7.3, 0.07
    species = SPECIES2(nv)
    sim, orc = make_pair(A, nx, L, dt, species, prec)
    for s, sp in enumerate(species):
        x, v, f = inputs.random_markers(100 * nx + s, n, L, sp["vmin"][0], sp["vmax"][0])
        sim.set_markers(s, x, v, f)
    sync_oracle_to_gpu(sim, orc)
    compare_grids(sim, orc, TOL[prec], "set")
    for k in range(3):
        sync_oracle_to_gpu(sim, orc)
        sim.step(1)
        orc.step(1)
        compare_grids(sim, orc, TOL[prec], f"step {k}")
        dx = L / nx
        compare_markers(sim, orc, 1e-12 * L if prec == 0 else 2e-6 * dx,
                        1e-12 if prec == 0 else 1e-5, L)
    sim.synchronize()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_set_markers_matches_oracle_inputs(A, prec):
    """Without any step: the reconstruction of caller markers (FP64 inputs,
    rounded to the FP32 storage in the FP32 path) against the oracle on the
    unrounded inputs."""
    nx, nv, n, L = 32, 50, 9000, 5.0
    species = SPECIES2(nv)
    sim, orc = make_pair(A, nx, L, 0.1, species, prec)
    for s, sp in enumerate(species):
        x, v, f = inputs.random_markers(7 + s, n, L, sp["vmin"][0], sp["vmax"][0])
        sim.set_markers(s, x, v, f)
        orc.set_markers(s, x, v, f)
    orc.refresh()
    compare_grids(sim, orc, TOL[prec], "set")


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_lattice_init_parity(A, prec):
    """avl_init_markers against the oracle's lattice: same SplitMix64 jitter,
    same f0 values, same reconstruction."""
    w = inputs.landau(nx=32, nv=48)
    sp = w["species"][0]
    sim, orc = make_pair(A, w["nx"], w["L"], w["dt"], w["species"], prec)
    f0 = w["f0"][0]
    sim.init_markers(0, w["lattice"][0], A.make_f0(f0["beams"], f0["modes"]), w["seed"], w["jitter"])
    orc.init_markers(0, w["lattice"][0], O.F0(f0["beams"], f0["modes"]), w["seed"], w["jitter"])
    orc.refresh()
    compare_grids(sim, orc, TOL[prec], "init")
    x, v, f = sim.get_markers(0)
    assert x.size == orc.x[0].size
    key_g = np.lexsort((np.round(v[0], 9), np.round(x, 9)))
    key_o = np.lexsort((np.round(orc.v[0][0], 9), np.round(orc.x[0], 9)))
    tol = 1e-12 if prec == 0 else 1e-6
    assert np.max(np.abs(x[key_g] - orc.x[0][key_o])) < tol * w["L"]
    assert np.max(np.abs(v[0][key_g] - orc.v[0][0][key_o])) < tol * 10
    assert rel(f[key_g], orc.fl[0][key_o]) < (1e-14 if prec == 0 else 1e-7)


def test_landau_free_running_fp64(A):
    """The Landau workload at its full size (32768 markers, 200 steps), GPU
    and oracle each running on their own: E stays within 1e-9 relative L2
    (stable, damped problem: no chaotic growth of roundoff), diagnostics
    agree, and the GPU's own damping fit matches the dispersion root."""
    import plasma_theory as P
    w = inputs.landau()
    sim, orc = make_pair(A, w["nx"], w["L"], w["dt"], w["species"], 0)
    f0 = w["f0"][0]
    sim.init_markers(0, w["lattice"][0], A.make_f0(f0["beams"], f0["modes"]), w["seed"], w["jitter"])
    orc.init_markers(0, w["lattice"][0], O.F0(f0["beams"], f0["modes"]), w["seed"], w["jitter"])
    orc.refresh()
    amps = [P.mode_amplitude(sim.get_E(), 1)]
    for k in range(w["steps"]):
        sim.step(1)
        orc.step(1)
        E = sim.get_E()
        amps.append(P.mode_amplitude(E, 1))
        if k % 20 == 19:
            assert rel(E, orc.E) < 1e-9, (k, rel(E, orc.E))
            np.testing.assert_allclose(sim.get_diag(), orc.diag(), rtol=1e-9, atol=1e-15)
    t = np.arange(len(amps)) * w["dt"]
    sel = (t >= 1.5) & (t <= 18)
    pk = P.peaks(t, np.array(amps))
    pk = pk[sel[pk]][:5]
    g = np.polyfit(t[pk], np.log(np.array(amps)[pk]), 1)[0]
    assert g == pytest.approx(P.landau_root(0.5).imag, rel=0.05)


@pytest.mark.parametrize("drift", [1, 0], ids=["drift_trigger", "miss_only"])
def test_strong_field_resort_and_overflow(A, monkeypatch, drift):
    """A light, strongly perturbed species: markers cross many velocity rows
    per step, exercising far keys in the re-sort and the out-of-window
    deposit; parity holds at every step.  With the drift trigger every step
    that drifts markers a row re-sorts; by default only the share of
    markers outside their windows decides."""
    monkeypatch.setenv("AVL_CHUNK_M", "256")
    monkeypatch.setenv("AVL_RESORT_DRIFT", str(drift))
    nx, nv, L, dt = 32, 64, 4.0, 0.2
    species = [dict(q=-1.0, m=0.05, nv=(nv,), vmin=(-4.0,), vmax=(4.0,))]
    for prec in (0, 1):
        sim, orc = make_pair(A, nx, L, dt, species, prec)
        f0 = A.make_f0([(1.0, (0.0,), (1.0,))], [(1, 0.5, 0.0), (2, 0.3, 1.0)])
        sim.init_markers(0, (2, 2, 1, 1), f0, 99, 1.0)
        for k in range(6):
            sync_oracle_to_gpu(sim, orc)
            sim.step(1)
            orc.step(1)
            compare_grids(sim, orc, TOL[prec], f"prec {prec} step {k}")
        st = sim.get_stats()
        # markers leave their chunks' windows quickly: most steps re-sort
        assert (3 if drift else 0) <= st[0, 1] <= 6
        sim.synchronize()


def test_edge_cases(A):
    nx, L = 16, 2.0
    sp = [dict(q=-1.0, m=1.0, nv=(8,), vmin=(-1.0,), vmax=(1.0,))]
    for prec in (0, 1):
        sim, orc = make_pair(A, nx, L, 0.1, sp, prec)
        # every marker beyond the velocity grid: nothing deposits, f = rho = E = 0
        x = np.linspace(0, L, 50, endpoint=False)
        v = np.full(50, 3.0)
        f = np.linspace(0.1, 1.0, 50)
        sim.set_markers(0, x, v, f)
        assert np.all(sim.get_f(0) == 0.0) and np.all(sim.get_rho() == 0.0)
        assert np.all(sim.get_E() == 0.0)
        # markers on the periodic seam and on cell centres
        x = np.array([0.0, L - 1e-9, 0.5 * L / nx, L / 2])
        v = np.array([0.0, 0.125, -0.875, 0.999])
        f = np.array([1.0, 2.0, 3.0, 4.0])
        sim.set_markers(0, x, v, f)
        orc.set_markers(0, x, v, f)
        orc.refresh()
        compare_grids(sim, orc, TOL[prec], "seam")
        sim.step(2)
        orc.step(2)
        compare_grids(sim, orc, 1e-9 if prec == 0 else 1e-5, "seam steps")


def test_immobile_species_and_unsoftened_cgs(A):
    """A fixed, perturbed ion background (never pushed, still in rho) and the
    unsoftened Eq. 5 with the CGS Poisson constant 4 pi."""
    nx, nv, L, dt = 32, 40, 6.0, 0.05
    species = [dict(q=-1.0, m=1.0, nv=(nv,), vmin=(-5.0,), vmax=(5.0,)),
               dict(q=1.0, m=100.0, nv=(16,), vmin=(-0.5,), vmax=(0.5,), mobile=False)]
    for prec in (0, 1):
        sim, orc = make_pair(A, nx, L, dt, species, prec, softening=False, cP=4 * np.pi)
        sim.init_markers(0, (2, 2, 1, 1), A.make_f0([(1.0, (0.0,), (1.0,))], [(1, 0.05, 0.0)]), 5, 1.0)
        sim.init_markers(1, (1, 2, 1, 1), A.make_f0([(1.0, (0.0,), (0.1,))], [(2, 0.1, 0.3)]), 6, 1.0)
        ions_before = sim.get_markers(1)
        for k in range(3):
            sync_oracle_to_gpu(sim, orc)
            sim.step(1)
            orc.step(1)
            compare_grids(sim, orc, TOL[prec], f"step {k}")
        ions_after = sim.get_markers(1)
        for a, b in zip(ions_before, ions_after):
            np.testing.assert_array_equal(a, b)


def test_errors_are_reported(A):
    from paper_1804_03901_gb300.avl import AvlError, AVL_EINVAL, AVL_ESTATE
    sim, _ = make_pair(A, 16, 2.0, 0.1, [dict(q=-1.0, m=1.0, nv=(8,), vmin=(-1.0,), vmax=(1.0,))], 0)
    with pytest.raises(AvlError) as e:
        sim.step(1)
    assert e.value.status == AVL_ESTATE
    with pytest.raises(AvlError) as e:
        sim.set_markers(0, np.array([2.5]), np.array([0.0]), np.array([1.0]))   # x beyond L
    assert e.value.status == AVL_EINVAL
    with pytest.raises(AvlError) as e:
        sim.init_markers(0, (0, 1, 1, 1), A.make_f0([(1.0, (0.0,), (1.0,))]), 1, 1.0)
    assert e.value.status == AVL_EINVAL
    sim.synchronize()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_diag_async_rows_match_blocking_reads(A, prec):
    """avl_get_diag_async enqueues the diagnostics row behind the steps: a
    row per step into page-locked memory, read after avl_synchronize, equals
    the blocking avl_get_diag of the same state and the oracle's row."""
    import torch
    nx, nv, L, dt = 32, 40, 6.0, 0.1
    species = [dict(q=-1.0, m=1.0, nv=(nv,), vmin=(-5.0,), vmax=(5.0,))]
    sim, orc = make_pair(A, nx, L, dt, species, prec)
    sim.init_markers(0, (2, 2, 1, 1), A.make_f0([(1.0, (0.0,), (1.0,))], [(1, 0.05, 0.0)]), 5, 1.0)
    nd = 3 + 3 * len(species)
    rows = torch.zeros((5, nd), dtype=torch.float64).pin_memory()
    ref = []
    for k in range(5):
        sim.step(1)
        sim.get_diag_async(rows[k].data_ptr())
        ref.append(sim.get_diag())
    sim.step(1)
    sim.get_diag_async(rows[4].data_ptr())   # overwritten in stream order
    sim.synchronize()
    got = rows.numpy()
    assert np.array_equal(got[:4], np.array(ref[:4]))
    last = sim.get_diag()
    assert np.array_equal(got[4], last)
    sync_oracle_to_gpu(sim, orc)
    err = np.abs(last - orc.diag()) / np.maximum(np.abs(orc.diag()), 1e-300)
    assert np.all(err < TOL[prec]), err


def test_conservation_drift_fp32_within_oracle_drift(A):
    """The Landau workload (32768 markers, 200 steps) in the FP32 path,
    free running beside the FP64 oracle: the drifts of N (integral of f)
    and of the total energy over the run stay within 1.5 times the oracle's
    own drift (the ratio reconstruction does not conserve N exactly, Sec.
    3.4.1), with an FP32 rounding floor of 1e-6."""
    w = inputs.landau()
    sim, orc = make_pair(A, w["nx"], w["L"], w["dt"], w["species"], 1)
    f0 = w["f0"][0]
    sim.init_markers(0, w["lattice"][0], A.make_f0(f0["beams"], f0["modes"]), w["seed"], w["jitter"])
    orc.init_markers(0, w["lattice"][0], O.F0(f0["beams"], f0["modes"]), w["seed"], w["jitter"])
    orc.refresh()
    g0, o0 = sim.get_diag(), orc.diag()
    sim.step(w["steps"])
    orc.step(w["steps"])
    g1, o1 = sim.get_diag(), orc.diag()
    for q, what in ((4, "N"), (2, "W_total")):
        dg = abs(g1[q] - g0[q]) / abs(g0[q])
        do = abs(o1[q] - o0[q]) / abs(o0[q])
        assert dg <= 1.5 * do + 1e-6, (what, dg, do)


def test_largest_deposit_window(A):
    """A wide x grid (nx = 2048): the FP32 deposit window of 8 velocity rows
    (numerator, denominator and the reference plane: 196 KB) still fits one
    CTA's shared memory and the step matches the oracle.  In FP64 creating
    the markers reports AVL_EINVAL instead of launching: at nx = 2048 for
    the fixed-point positions (nx 2^52 must stay below 2^63), at nx = 2040
    because the window (8 bytes per plane cell, 7 rows at least) does not
    fit."""
    nx, L, dt = 2048, 7.3, 0.07
    species = SPECIES2(64)
    sim, orc = make_pair(A, nx, L, dt, species, A.AVL_FP32)
    for s, sp in enumerate(species):
        x, v, f = inputs.random_markers(31 + s, 20011, L, sp["vmin"][0], sp["vmax"][0])
        sim.set_markers(s, x, v, f)
    for k in range(2):
        sync_oracle_to_gpu(sim, orc)
        sim.step(1)
        orc.step(1)
        compare_grids(sim, orc, TOL[1], f"nx 2048 step {k}")
    sim.close()
    for nxd, why in ((2048, "nx < 2048"), (2040, "shared memory")):
        sim, _ = make_pair(A, nxd, L, dt, species, A.AVL_FP64)
        x, v, f = inputs.random_markers(31, 20011, L, species[0]["vmin"][0], species[0]["vmax"][0])
        with pytest.raises(A.AvlError) as e:
            sim.set_markers(0, x, v, f)
        assert e.value.status == A.AVL_EINVAL and why in str(e.value), (nxd, str(e.value))
        sim.close()
