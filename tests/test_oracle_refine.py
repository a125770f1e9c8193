"""Pins of the oracle's marker refinement by tracing back (Sec. 2: a patch of
phase space that needs more resolution later is traced back to the initial
state and given more markers there), against things that do not share its
code: free streaming, the closed form of the inverse kick-drift under a
uniform field, and the oracle's own forward push run over the same fields."""
import math

import numpy as np

from oracle import oracle as O

NX, L, DT = 16, 6.0, 0.1


def species():
    return O.Species(q=-1.3, m=0.8, nv=(20,), vmin=(-4.0,), vmax=(4.0,))


def f0():
    return O.F0(beams=[(0.6, (0.7,), (0.9,)), (0.4, (-1.1,), (0.5,))], modes=[(1, 0.05, 0.3), (3, 0.02, -1.0)])


def test_count_and_placement():
    sp = species()
    box, lat = (3, 7, 5, 9), (2, 3)
    x, v, f = O.refine_markers(NX, L, sp, box, lat, f0(), 0, 99, 1.0, DT, np.zeros((0, NX)))
    assert x.size == (7 - 3) * (9 - 5) * 2 * 3
    dx, dv = L / NX, 8.0 / 20
    assert np.all((x >= 3 * dx) & (x < 7 * dx))
    assert np.all((v[0] >= -4.0 + 5 * dv) & (v[0] < -4.0 + 9 * dv))
    # no steps since the initial state: the values are f0 at the new markers
    want = np.array([O.f0_eval(f0(), 1, L, x[k], [v[0][k]]) for k in range(x.size)])
    np.testing.assert_allclose(f, want, rtol=1e-14)


def test_free_streaming_closed_form():
    """E = 0 in every stored state: the foot is (x - v N dt mod L, v) and
    f = f0 there (the exact solution f0(x - v t, v) of the field-free Vlasov
    equation)."""
    sp = species()
    N = 37
    x, v, f, x0, v0 = O.refine_markers(NX, L, sp, (0, NX, 2, 18), (1, 2), f0(), 1, 5, 0.5, DT,
                                       np.zeros((N, NX)), feet=True)
    np.testing.assert_allclose(v0, v[0], rtol=0, atol=0)
    d = (x0 - (x - v[0] * N * DT)) / L
    assert np.max(np.abs(d - np.round(d))) < 1e-12
    want = np.array([O.f0_eval(f0(), 1, L, (x[k] - v[0][k] * N * DT) % L, [v[0][k]]) for k in range(x.size)])
    np.testing.assert_allclose(f, want, rtol=1e-10, atol=1e-14)


def test_uniform_field_closed_form():
    """E = E0 everywhere: v_{N-k} = v - k a, a = (q/m) E0 dt, so the foot is
    v0 = v - N a and x0 = x - dt (N v - a N (N - 1) / 2) (mod L)."""
    sp = species()
    N, E0 = 25, 0.37
    a = sp.q / sp.m * E0 * DT
    x, v, f, x0, v0 = O.refine_markers(NX, L, sp, (4, 9, 6, 12), (2, 2), f0(), 2, 7, 1.0, DT,
                                       np.full((N, NX), E0), feet=True)
    np.testing.assert_allclose(v0, v[0] - N * a, rtol=0, atol=1e-12)
    xw = x - DT * (N * v[0] - a * N * (N - 1) / 2)
    d = (x0 - xw) / L
    assert np.max(np.abs(d - np.round(d))) < 1e-12


def test_reversible_against_the_forward_push():
    """A non-uniform field history: pushing the feet forward with the oracle's
    kick-drift step (E^n in step n) returns the refined markers."""
    sp = species()
    N = 30
    rng = np.random.default_rng(3)
    hist = np.array([0.4 * np.sin(2 * math.pi * (np.arange(NX) + 0.5) / NX + 0.2 * n)
                     + 0.1 * rng.normal(size=NX) for n in range(N)])
    x, v, f, x0, v0 = O.refine_markers(NX, L, sp, (0, NX, 0, 20), (2, 1), f0(), 3, 11, 1.0, DT, hist, feet=True)
    xs, vs = x0.copy(), v0.reshape(1, -1).copy()
    for n in range(N):
        O.push(1, NX, L, sp, xs, vs, DT, hist[n])
    d = (xs - x) / L
    assert np.max(np.abs(d - np.round(d))) < 1e-11
    np.testing.assert_allclose(vs[0], v[0], rtol=0, atol=1e-11)
    # and the values are f0 at the feet
    want = np.array([O.f0_eval(f0(), 1, L, x0[k], [v0[k]]) for k in range(x.size)])
    np.testing.assert_allclose(f, want, rtol=1e-14)
