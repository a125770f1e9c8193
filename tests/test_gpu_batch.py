"""Batched ensemble (avl_create_batch): every run of a batch advanced by the
batched launches matches the FP64 oracle per step (FP64 1e-10, FP32 1e-5
relative L2 of f, n, rho, E) and matches the same run stepped on its own;
the chunk-size autotuner leaves the state as it found it."""
import math

import numpy as np
import pytest

from oracle import oracle as O

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


# (nx, L, dt, nv, vmax, f0, lattice): Landau-like and two-stream-like runs of uneven sizes
RUNS = [
    (16, 4 * math.pi, 0.1, 32, 6.0, dict(beams=[(1.0, (0.0,), (1.0,))], modes=[(1, 0.05, 0.0)]), (2, 2, 1, 1)),
    (32, 12.8, 0.05, 48, 8.0, dict(beams=[(0.5, (2.5,), (0.8,)), (0.5, (-2.5,), (0.8,))],
                                  modes=[(1, 0.01, 0.4), (3, 0.02, 1.0)]), (2, 4, 1, 1)),
    (24, 9.0, 0.1, 40, 6.0, dict(beams=[(1.0, (0.5,), (1.2,))], modes=[(2, 0.03, 2.0)]), (4, 4, 1, 1)),
    (64, 25.6, 0.05, 96, 10.0, dict(beams=[(0.5, (3.0,), (1.0,)), (0.5, (-3.0,), (1.0,))],
                                   modes=[(m, 1e-3, 0.3 * m) for m in range(1, 6)]), (2, 2, 1, 1)),
]


def species_of(nv, vmax):
    return dict(q=-1.0, m=1.0, nv=(nv,), vmin=(-vmax,), vmax=(vmax,), mobile=True)


def make_batch(A, prec, runs=RUNS):
    doms = [A.make_domain(1, nx, L, dt, 1.0, True, prec) for (nx, L, dt, *_rest) in runs]
    sps = [[A.make_species(**species_of(nv, vmax))] for (_, _, _, nv, vmax, _, _) in runs]
    b = A.Batch(doms, sps)
    for r, (nx, L, dt, nv, vmax, f0, lat) in enumerate(runs):
        b.runs[r].init_markers(0, lat, A.make_f0(**f0), 100 + r, 1.0)
    return b


def oracle_of(run):
    nx, L, dt, nv, vmax, f0, lat = run
    return O.OracleSim(1, nx, L, dt, [O.Species(**species_of(nv, vmax))])


def sync(sim, orc):
    x, v, f = sim.get_markers(0)
    orc.set_markers(0, x, v, f)
    orc.refresh()


def compare(sim, orc, tol, what):
    f, n = sim.get_f(0, with_n=True)
    assert rel(f, orc.f[0]) < tol, (what, "f", rel(f, orc.f[0]))
    assert rel(n, orc.den[0]) < tol, (what, "n", rel(n, orc.den[0]))
    assert rel(sim.get_rho(), orc.rho) < tol, (what, "rho")
    assert rel(sim.get_E(), orc.E) < tol, (what, "E", rel(sim.get_E(), orc.E))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_batch_runs_match_oracle(A, prec):
    b = make_batch(A, prec)
    orcs = [oracle_of(run) for run in RUNS]
    for k in range(3):
        for r in range(len(RUNS)):
            sync(b.runs[r], orcs[r])
        b.step(1)
        for r in range(len(RUNS)):
            orcs[r].step(1)
            compare(b.runs[r], orcs[r], TOL[prec], f"run {r} step {k}")
    b.synchronize()
    b.close()


def test_batch_equals_runs_stepped_alone(A):
    b = make_batch(A, 0)
    b.step(10)
    for r, (nx, L, dt, nv, vmax, f0, lat) in enumerate(RUNS):
        sim = A.Simulation(A.make_domain(1, nx, L, dt, 1.0, True, 0), [A.make_species(**species_of(nv, vmax))])
        sim.init_markers(0, lat, A.make_f0(**f0), 100 + r, 1.0)
        sim.step(10)
        assert rel(b.runs[r].get_E(), sim.get_E()) < 1e-11, r
        np.testing.assert_allclose(b.runs[r].get_diag(), sim.get_diag(), rtol=1e-11)
        sim.close()
    b.close()


def test_autotune_restores_the_state(A):
    b = make_batch(A, 1)
    b.step(2)
    E0 = [b.runs[r].get_E() for r in range(len(RUNS))]
    m = b.autotune(2)
    assert m in (0, 1024, 2048, 4096, 8192, 16384)
    for r in range(len(RUNS)):
        assert rel(b.runs[r].get_E(), E0[r]) < 1e-5, r
    orcs = [oracle_of(run) for run in RUNS]
    for r in range(len(RUNS)):
        sync(b.runs[r], orcs[r])
    b.step(1)
    for r in range(len(RUNS)):
        orcs[r].step(1)
        compare(b.runs[r], orcs[r], TOL[1], f"run {r} after autotune")
    b.close()


def test_batch_errors(A):
    d64 = A.make_domain(1, 16, 5.0, 0.1, 1.0, True, 0)
    d32 = A.make_domain(1, 16, 5.0, 0.1, 1.0, True, 1)
    sp = [A.make_species(**species_of(16, 4.0))]
    with pytest.raises(A.AvlError):
        A.Batch([d64, d32], [sp, sp])
    d3 = A.make_domain(3, 16, 5.0, 0.1, 1.0, True, 1)
    with pytest.raises(A.AvlError):
        A.Batch([d3], [[A.make_species(-1.0, 1.0, (4, 4, 4), (-1, -1, -1), (1, 1, 1))]])
    b = A.Batch([d64, d64], [sp, sp])
    with pytest.raises(A.AvlError):   # run 1 has no markers
        b.runs[0].init_markers(0, (2, 2, 1, 1), A.make_f0([(1.0, (0.0,), (1.0,))]), 1)
        b.step(1)
    # the diagnostics rows belong to the runs, not to the batch
    import numpy as np
    row = np.zeros(6)
    ptr = row.ctypes.data_as(A.C.POINTER(A.C.c_double))
    assert A.avl_get_diag(b.ctx, ptr) == A.AVL_EINVAL
    assert A.avl_get_diag_async(b.ctx, row.ctypes.data) == A.AVL_EINVAL
    b.close()
