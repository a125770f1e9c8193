"""Failure detection without a GPU fault, and replay.

The deposit kernels wait for their bulk copies (TMA) on an mbarrier with a
bounded number of polls.  avl_set_wait_limit(ctx, 0) makes every such first
wait give up at once: the kernel sets the AVL_ETIMEOUT flag, drains the copy
with the default limit (no copy is left in flight into shared memory) and the
step goes on.  The test checks that the host sees AVL_ETIMEOUT at the next
synchronisation, that the step itself is still the oracle's step, and that
with the default limit restored the context steps on without an error.
Nothing here traps, faults or hangs the GPU.

Replay: the same input run twice gives the same state up to the rounding of
sums whose order the shared-memory and global reductions leave open (the
atomics are unordered), i.e. agreement at the 1e-13 level in FP64, not
bitwise identity.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1804_03901_gb300 import inputs

import test_gpu_parity as P1
import test_gpu_parity3 as P3

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


def pair_1d1v(A, prec):
    species = P1.SPECIES2(64)
    sim, orc = P1.make_pair(A, 32, 7.3, 0.07, species, prec)
    for s, sp in enumerate(species):
        x, v, f = inputs.random_markers(900 + s, 6001, 7.3, sp["vmin"][0], sp["vmax"][0])
        sim.set_markers(s, x, v, f)
    return sim, orc, P1


def pair_1d3v(A, prec):
    species = P3.species2((8, 6, 5))
    sim, orc = P3.make_pair(A, 16, 7.3, 0.07, species, prec)
    for s, sp in enumerate(species):
        x, v, f = inputs.random_markers3(910 + s, 8001, 7.3, sp["vmin"], sp["vmax"])
        sim.set_markers(s, x, v, f)
    return sim, orc, P3


@pytest.mark.parametrize("nvdim,prec", [(1, 1), (1, 0), (3, 1), (3, 0)],
                         ids=["1d1v-fp32", "1d1v-fp64", "1d3v-fp32", "1d3v-fp64"])
def test_bounded_wait_timeout_is_reported_and_the_context_recovers(A, nvdim, prec):
    sim, orc, P = (pair_1d1v if nvdim == 1 else pair_1d3v)(A, prec)
    tol = P.TOL[prec]
    P.sync_oracle_to_gpu(sim, orc)
    sim.set_wait_limit(0)               # every first wait on a bulk copy gives up at once
    sim.step(1)
    orc.step(1)
    with pytest.raises(A.AvlError) as err:
        sim.synchronize()
    assert err.value.status == A.AVL_ETIMEOUT, err.value
    # the copies were drained before the kernels went on: the step is intact
    P.compare_grids(sim, orc, tol, "step with the timeout path taken")
    sim.synchronize()                   # the flag was reported once and cleared
    sim.set_wait_limit(-1)              # default limit again
    P.sync_oracle_to_gpu(sim, orc)
    sim.step(2)
    orc.step(2)
    sim.synchronize()
    P.compare_grids(sim, orc, tol, "steps after the default limit is restored")
    sim.close()


def test_wait_limit_rejects_null_context(A):
    assert A.avl_set_wait_limit(None, 0) == A.AVL_EINVAL


@pytest.mark.parametrize("nvdim", [1, 3])
def test_replay_fp64_agrees_to_rounding(A, nvdim):
    """Two contexts fed the same markers and stepped the same way."""
    runs = []
    for _ in range(2):
        sim, _, _ = (pair_1d1v if nvdim == 1 else pair_1d3v)(A, 0)
        sim.step(5)
        sim.synchronize()
        runs.append((sim, [sim.get_f(s) for s in range(2)], sim.get_E(), sim.get_diag(),
                     [sim.get_markers(s) for s in range(2)]))
    (s1, f1, E1, d1, m1), (s2, f2, E2, d2, m2) = runs
    for s in range(2):
        assert P1.rel(f2[s], f1[s]) < 1e-13
        x1, v1, g1 = m1[s]
        x2, v2, g2 = m2[s]
        i1, i2 = np.argsort(g1, kind="stable"), np.argsort(g2, kind="stable")
        np.testing.assert_array_equal(g1[i1], g2[i2])
        assert np.max(np.abs(x1[i1] - x2[i2])) < 1e-12
        assert np.max(np.abs(v1[:, i1] - v2[:, i2])) < 1e-12
    assert P1.rel(E2, E1) < 1e-12
    assert np.all(np.abs(d2 - d1) <= 1e-12 * np.abs(d1) + 1e-300)
    s1.close()
    s2.close()
