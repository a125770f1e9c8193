"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper it checks and the independent fact
it checks against: a published test vector, a closed form, a brute-force
evaluation of the paper's definition, or an invariant.
"""
import itertools
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Counter-based generator for the lattice jitter
# --------------------------------------------------------------------------
def test_splitmix64_published_vector():
    """SplitMix64 from state 0 reproduces the published reference outputs."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt"))
            if l.strip() and not l.startswith("#")]
    for n, hexval in rows:
        assert O.splitmix64(0, int(n)) == int(hexval, 16)


def test_jitter_uniform_statistics():
    u = np.array([O.lib().orc_jitter_uniform(12345, 1, m, d) for m in range(4000) for d in range(4)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1.0 / 12.0) < 0.005
    hist, _ = np.histogram(u, bins=16, range=(0, 1))
    chi2 = np.sum((hist - u.size / 16) ** 2 / (u.size / 16))
    assert chi2 < 40.0       # 15 dof: p ~ 5e-4


# --------------------------------------------------------------------------
# Initial distribution and markers (Sec. 2, Sec. 3.1, Sec. 3.3, Eq. 17)
# --------------------------------------------------------------------------
def test_f0_velocity_integral_is_density():
    f0 = O.F0(beams=[(0.7, (1.5, 0, 0), (0.8, 1, 1)), (0.3, (-2.0, 0, 0), (0.5, 1, 1))],
              modes=[(2, 0.1, 0.3)])
    L = 10.0
    for x in (0.0, 1.3, 7.7):
        val, _ = integrate.quad(lambda v: O.f0_eval(f0, 1, L, x, [v]), -15, 15, limit=200)
        pert = 1.0 + 0.1 * np.cos(2 * np.pi * 2 * x / L + 0.3)
        assert val == pytest.approx(1.0 * pert, rel=1e-9)


def test_f0_3v_integral_is_density():
    f0 = O.F0(beams=[(0.95, (0, 0, 0), (1, 1, 1)), (0.05, (4.0, 0, 0), (0.5, 0.5, 0.5))])
    # separable: integrate each beam's x-component, others by symmetry
    val, _ = integrate.tplquad(lambda z, y, x: O.f0_eval(f0, 3, 1.0, 0.0, [x, y, z]),
                               -8, 8, -8, 8, -8, 8, epsabs=1e-7)
    assert val == pytest.approx(1.0, rel=1e-5)


def test_marker_lattice_without_jitter():
    sp = O.Species(q=-1, m=1, nv=(4,), vmin=(-2.0,), vmax=(2.0,))
    x, v, fl = O.init_markers(1, 3, 6.0, sp, (2, 2, 1, 1), O.F0(beams=[(1, (0,), (1,))]), 0, 7, 0.0)
    assert x.size == 3 * 4 * 4
    dx, dv = 2.0, 1.0
    m = 0
    for i in range(3):
        for j in range(4):
            for a in range(2):
                for b in range(2):
                    assert x[m] == pytest.approx((i + (a + 0.5) / 2) * dx, abs=1e-14)
                    assert v[0, m] == pytest.approx(-2.0 + (j + (b + 0.5) / 2) * dv, abs=1e-14)
                    m += 1


def test_markers_inside_their_subcells_with_jitter():
    sp = O.Species(q=-1, m=1, nv=(5, 3, 2), vmin=(-3, -1, -2), vmax=(3, 2, 2))
    lat = (2, 1, 2, 1)
    f0 = O.F0(beams=[(1, (0, 0, 0), (1, 1, 1))], modes=[(1, 0.05, 0.0)])
    x, v, fl = O.init_markers(3, 4, 8.0, sp, lat, f0, 2, 99, 1.0)
    ppc = 4
    assert x.size == 4 * 5 * 3 * 2 * ppc
    dx = 2.0
    dv = [(sp.vmax[d] - sp.vmin[d]) / sp.nv[d] for d in range(3)]
    m = 0
    for i, jx, jy, jz in itertools.product(range(4), range(5), range(3), range(2)):
        for a, bx, by, bz in itertools.product(range(2), range(1), range(2), range(1)):
            assert i * dx + a * dx / 2 <= x[m] < i * dx + (a + 1) * dx / 2
            for d, (j, b, p) in enumerate(((jx, bx, 1), (jy, by, 2), (jz, bz, 1))):
                lo = sp.vmin[d] + (j + b / p) * dv[d]
                assert lo <= v[d, m] < lo + dv[d] / p + 1e-15
            assert fl[m] == pytest.approx(O.f0_eval(f0, 3, 8.0, x[m], v[:, m]), rel=1e-15)
            m += 1


# --------------------------------------------------------------------------
# Reconstruction (Sec. 2, Fig. 1, Eq. 4) against the overlap-area definition
# --------------------------------------------------------------------------
def _ov(a0, a1, b0, b1):
    return max(0.0, min(a1, b1) - max(a0, b0))


def brute_reconstruct(nvdim, nx, L, sp, x, v, fl):
    """Marker = uniform box of one cell's size; alpha = overlap volume / cell
    volume with every grid cell; periodic images in x; no cells beyond the
    velocity grid."""
    dx = L / nx
    nv = tuple(sp.nv[:nvdim])
    dv = [(sp.vmax[d] - sp.vmin[d]) / sp.nv[d] for d in range(nvdim)]
    num = np.zeros((nx,) + nv)
    den = np.zeros((nx,) + nv)
    for l in range(x.size):
        for i in range(nx):
            ox = sum(_ov(x[l] - dx / 2 + sh, x[l] + dx / 2 + sh, i * dx, (i + 1) * dx)
                     for sh in (-L, 0.0, L)) / dx
            if ox == 0.0:
                continue
            for j in itertools.product(*[range(n) for n in nv]):
                o = ox
                for d in range(nvdim):
                    c0 = sp.vmin[d] + j[d] * dv[d]
                    o *= _ov(v[d, l] - dv[d] / 2, v[d, l] + dv[d] / 2, c0, c0 + dv[d]) / dv[d]
                if o > 0.0:
                    num[(i,) + j] += o * fl[l]
                    den[(i,) + j] += o
    f = np.where(den > 0, num / np.where(den > 0, den, 1), 0.0)
    return f, num, den


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_reconstruct_1d1v_matches_overlap_area(seed):
    rng = np.random.default_rng(seed)
    nx, L = 5, 3.0
    sp = O.Species(q=-1, m=1, nv=(6,), vmin=(-1.5,), vmax=(1.5,))
    n = 12
    x = rng.uniform(0, L, n)
    x[0] = 0.0                       # on the periodic seam
    x[1] = L - 1e-12
    v = rng.uniform(-1.9, 1.9, (1, n))   # some clouds partly or wholly off the v-grid
    v[0, 2] = -1.5 + 0.25            # exactly on a cell centre
    fl = rng.uniform(0.1, 2.0, n)
    f, num, den = O.reconstruct(1, nx, L, sp, x, v, fl)
    fb, numb, denb = brute_reconstruct(1, nx, L, sp, x, v, fl)
    np.testing.assert_allclose(num, numb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(den, denb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(f, fb, rtol=1e-11, atol=1e-14)


def test_reconstruct_1d3v_matches_overlap_volume():
    rng = np.random.default_rng(5)
    nx, L = 3, 2.0
    sp = O.Species(q=-1, m=1, nv=(3, 2, 4), vmin=(-1, -1, -2), vmax=(1, 1, 2))
    n = 8
    x = rng.uniform(0, L, n)
    v = np.stack([rng.uniform(-1.2, 1.2, n), rng.uniform(-1.2, 1.2, n), rng.uniform(-2.3, 2.3, n)])
    fl = rng.uniform(0.1, 2.0, n)
    f, num, den = O.reconstruct(3, nx, L, sp, x, v, fl)
    fb, numb, denb = brute_reconstruct(3, nx, L, sp, x, v, fl)
    np.testing.assert_allclose(num, numb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(den, denb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(f, fb, rtol=1e-11, atol=1e-14)


def test_reconstruct_uniform_value_and_unit_weight():
    rng = np.random.default_rng(3)
    nx, L = 8, 4.0
    sp = O.Species(q=-1, m=1, nv=(8,), vmin=(-2.0,), vmax=(2.0,))
    x = rng.uniform(0, L, 40)
    v = rng.uniform(-1.5, 1.5, (1, 40))
    f, num, den = O.reconstruct(1, nx, L, sp, x, v, np.full(40, 0.37))
    assert np.all(np.abs(f[den > 0] - 0.37) < 1e-15)
    assert np.all(f[den == 0] == 0.0)
    # one interior marker: its weights sum to one
    f1, n1, d1 = O.reconstruct(1, nx, L, sp, np.array([1.3]), np.array([[0.2]]), np.array([2.0]))
    assert d1.sum() == pytest.approx(1.0, abs=1e-15)
    assert n1.sum() == pytest.approx(2.0, abs=1e-15)
    assert np.count_nonzero(d1) == 4


def test_vhs_ratio_does_not_drown_low_values():
    """The defining property of Eq. 4 against the plain sum of Eq. 3: two
    markers sharing cells with values 1 and 1e-10 reconstruct a weighted
    mean, not a sum."""
    sp = O.Species(q=-1, m=1, nv=(4,), vmin=(0.0,), vmax=(4.0,))
    x = np.array([2.5, 2.5])
    v = np.array([[1.5, 1.5]])
    f, num, den = O.reconstruct(1, 4, 4.0, sp, x, v, np.array([1.0, 1e-10]))
    assert f[2, 1] == pytest.approx(0.5 * (1 + 1e-10), rel=1e-14)


# --------------------------------------------------------------------------
# Velocity moment (Eq. 14) and diagnostics (Sec. 3.4.1, Eq. 12, Eq. 13)
# --------------------------------------------------------------------------
def _maxwell_grid(nx, nv, vmax):
    dv = 2 * vmax / nv
    vc = -vmax + (np.arange(nv) + 0.5) * dv
    return np.tile(np.exp(-0.5 * vc ** 2) / np.sqrt(2 * np.pi), (nx, 1)), vc, dv


def test_moment_maxwellian_quadrature():
    f, vc, dv = _maxwell_grid(7, 128, 6.0)
    sp = O.Species(q=-1.0, m=1, nv=(128,), vmin=(-6.0,), vmax=(6.0,))
    rho = O.moment(1, 7, 3.0, sp, f)
    # midpoint rule = integral - (h^2/24) (f'(b) - f'(a)) + O(h^4) (Euler-Maclaurin)
    phi6 = np.exp(-18.0) / np.sqrt(2 * np.pi)
    midpoint = special.erf(6.0 / np.sqrt(2.0)) + dv * dv / 24 * 12.0 * phi6
    # next Euler-Maclaurin term: 7 h^4/5760 |f'''(b) - f'''(a)| ~ 2.3e-13
    np.testing.assert_allclose(rho, -midpoint, rtol=5e-13)


def test_diag_maxwellian_closed_forms():
    nx, L, a = 5, 2.5, 6.0
    f, vc, dv = _maxwell_grid(nx, 256, a)
    sp = O.Species(q=-1.0, m=2.0, nv=(256,), vmin=(-a,), vmax=(a,))
    N, W, S = O.diag(1, nx, L, sp, f)
    phi = np.exp(-0.5 * a * a) / np.sqrt(2 * np.pi)
    h2 = dv * dv / 24       # Euler-Maclaurin: midpoint = integral - h^2/24 (f'(b) - f'(a))
    N_mid = special.erf(a / np.sqrt(2)) + h2 * 2 * a * phi
    W_mid = (special.erf(a / np.sqrt(2)) - 2 * a * phi) + h2 * 2 * (a ** 3 - 2 * a) * phi
    assert N == pytest.approx(L * N_mid, rel=1e-12)
    assert W == pytest.approx(0.5 * 2.0 * L * W_mid, rel=1e-11)
    ent, _ = integrate.quad(lambda v: (np.exp(-0.5 * v * v) / np.sqrt(2 * np.pi))
                            * (-0.5 * v * v - 0.5 * np.log(2 * np.pi)), -a, a)
    assert S == pytest.approx(L * ent, rel=1e-6)


def test_field_energy_single_mode():
    nx, L = 32, 7.0
    x = (np.arange(nx) + 0.5) * L / nx
    E = 0.3 * np.sin(2 * np.pi * 3 * x / L)
    assert O.field_energy(nx, L, 1.0, E) == pytest.approx(0.09 * L / 4, rel=1e-13)
    assert O.field_energy(nx, L, 4 * np.pi, E) == pytest.approx(0.09 * L / 2 / (8 * np.pi), rel=1e-13)


# --------------------------------------------------------------------------
# Spectral Poisson solve (Sec. 3.1, Eq. 5, Eq. 6a-c)
# --------------------------------------------------------------------------
def _modes(nx, L, coeffs):
    x = (np.arange(nx) + 0.5) * L / nx
    rho = np.zeros(nx)
    for m, a, b in coeffs:
        k = 2 * np.pi * m / L
        rho += a * np.cos(k * x) + b * np.sin(k * x)
    return x, rho


@pytest.mark.parametrize("nx", [16, 15, 64])
def test_poisson_unsoftened_modes_closed_form(nx):
    L, cP = 5.0, 1.7
    coeffs = [(1, 0.4, -0.2), (3, -0.1, 0.25), (nx // 2 - 1, 0.05, 0.01)]
    x, rho = _modes(nx, L, coeffs)
    E = O.poisson(nx, L, cP, False, rho + 3.0)        # constant part removed by k = 0
    Eex = np.zeros(nx)
    for m, a, b in coeffs:
        k = 2 * np.pi * m / L
        Eex += cP / k * (a * np.sin(k * x) - b * np.cos(k * x))
    np.testing.assert_allclose(E, Eex, atol=1e-12)


@pytest.mark.parametrize("nx", [16, 15, 64])
def test_poisson_softened_modes_closed_form(nx):
    L, cP = 5.0, 1.0
    dx = L / nx
    coeffs = [(1, 0.4, -0.2), (5, -0.1, 0.25)]
    x, rho = _modes(nx, L, coeffs)
    E = O.poisson(nx, L, cP, True, rho)
    Eex = np.zeros(nx)
    for m, a, b in coeffs:
        k = 2 * np.pi * m / L
        kappa = np.sin(k * dx) / dx
        K2 = (2 * np.sin(k * dx / 2) / dx) ** 2
        Eex += cP * kappa / K2 * (a * np.sin(k * x) - b * np.cos(k * x))
    np.testing.assert_allclose(E, Eex, atol=1e-12)


@pytest.mark.parametrize("nx", [8, 9, 32])
def test_poisson_softened_equals_finite_difference_solve(nx):
    """Eq. 6 with kappa = sin(k dx)/dx and K^2 = (2 sin(k dx/2)/dx)^2 is the
    spectral form of E = -(phi_{i+1} - phi_{i-1})/(2 dx) with
    -(phi_{i+1} - 2 phi_i + phi_{i-1})/dx^2 = cP (rho_i - <rho>); solved here
    by a dense least-squares solve, no Fourier transform involved."""
    rng = np.random.default_rng(nx)
    L, cP = 3.0, 4 * np.pi
    dx = L / nx
    rho = rng.normal(size=nx)
    A = np.zeros((nx, nx))
    for i in range(nx):
        A[i, i] = 2.0 / dx ** 2
        A[i, (i + 1) % nx] -= 1.0 / dx ** 2
        A[i, (i - 1) % nx] -= 1.0 / dx ** 2
    Aug = np.vstack([A, np.ones((1, nx))])
    rhs = np.concatenate([cP * (rho - rho.mean()), [0.0]])
    phi = np.linalg.lstsq(Aug, rhs, rcond=None)[0]
    Efd = -(np.roll(phi, -1) - np.roll(phi, 1)) / (2 * dx)
    E = O.poisson(nx, L, cP, True, rho)
    np.testing.assert_allclose(E, Efd, atol=1e-10 * np.abs(Efd).max())


def test_poisson_constant_and_nyquist_give_zero():
    nx, L = 16, 2.0
    rho = np.full(nx, 0.7) + 0.3 * (-1.0) ** np.arange(nx)
    for soft in (True, False):
        E = O.poisson(nx, L, 1.0, soft, rho)
        assert np.max(np.abs(E)) < 1e-14


# --------------------------------------------------------------------------
# Push (Sec. 2, Fig. 2): gather with the reconstruction weights, kick, drift
# --------------------------------------------------------------------------
def test_push_free_streaming_closed_form():
    rng = np.random.default_rng(1)
    nx, L, dt = 16, 5.0, 0.1
    sp = O.Species(q=-1, m=1, nv=(8,), vmin=(-4,), vmax=(4,))
    x0 = rng.uniform(0, L, 50)
    v0 = rng.uniform(-4, 4, (1, 50))
    x, v = x0.copy(), v0.copy()
    for _ in range(37):
        O.push(1, nx, L, sp, x, v, dt, np.zeros(nx))
    np.testing.assert_array_equal(v, v0)
    d = (x - np.mod(x0 + v0[0] * 37 * dt, L) + L / 2) % L - L / 2
    assert np.max(np.abs(d)) < 1e-12
    assert np.all((x >= 0) & (x < L))


def test_push_uniform_field_discrete_parabola():
    rng = np.random.default_rng(2)
    nx, L, dt, E0 = 16, 50.0, 0.05, 0.3
    sp = O.Species(q=-2.0, m=4.0, nv=(8,), vmin=(-4,), vmax=(4,))
    a = sp.q / sp.m * E0
    x0 = rng.uniform(0, L, 20)
    v0 = rng.uniform(-1, 1, (1, 20))
    x, v = x0.copy(), v0.copy()
    n = 25
    for _ in range(n):
        O.push(1, nx, L, sp, x, v, dt, np.full(nx, E0))
    np.testing.assert_allclose(v[0], v0[0] + a * n * dt, atol=1e-13)
    xe = np.mod(x0 + n * v0[0] * dt + a * dt * dt * n * (n + 1) / 2, L)
    d = (x - xe + L / 2) % L - L / 2
    assert np.max(np.abs(d)) < 1e-12


def test_push_gathers_with_cic_weights_linear_field():
    """A field linear between two cell centres is interpolated exactly."""
    nx, L = 10, 10.0
    sp = O.Species(q=1, m=1, nv=(4,), vmin=(-1,), vmax=(1,))
    E = np.zeros(nx)
    E[3], E[4] = 2.0, 5.0              # centres at 3.5 and 4.5
    x = np.array([3.5, 3.75, 4.0, 4.5])
    v = np.zeros((1, 4))
    O.push(1, nx, L, sp, x, v, 1.0, E)
    np.testing.assert_allclose(v[0], [2.0, 2.75, 3.5, 5.0], atol=1e-14)


# --- output moments and the field residual (Sec. 3.4.2) ------------------------
def test_moments_of_a_flat_distribution_are_exact():
    """f = c on the velocity grid: the midpoint rule integrates v exactly and
    v^2 with the known -h^2/24 error per cell: j = q c (b^2 - a^2)/2,
    M2 = q c [(b^3 - a^3)/3 - (b - a) h^2 / 12]."""
    nx, L = 5, 3.0
    sp = O.Species(q=-1.5, m=1.0, nv=(17,), vmin=(-2.0,), vmax=(5.0,))
    c = 0.7
    f = np.full((nx, 17), c)
    m = O.moments(1, nx, L, sp, f)
    a, b = -2.0, 5.0
    h = (b - a) / 17
    np.testing.assert_allclose(m[0], sp.q * c * (b - a), rtol=1e-14)
    np.testing.assert_allclose(m[1], sp.q * c * (b * b - a * a) / 2, rtol=1e-13)
    np.testing.assert_allclose(m[2], sp.q * c * ((b ** 3 - a ** 3) / 3 - (b - a) * h * h / 12), rtol=1e-13)


def test_moments_1d3v_separate_by_component():
    """1d3v: f = g(vx) h(vy) k(vz) gives j_d = q (prod of the other
    integrals) (first moment of its own factor), and M2 the sum over d."""
    nx, L = 3, 2.0
    sp = O.Species(q=1.0, m=1.0, nv=(6, 5, 4), vmin=(-1.0, -2.0, 0.5), vmax=(2.0, 1.0, 1.5))
    rng = np.random.default_rng(2)
    fac = [rng.uniform(0.1, 1.0, n) for n in sp.nv]
    f = np.einsum("i,j,k->ijk", *fac)[None].repeat(nx, axis=0)
    dv = [(sp.vmax[d] - sp.vmin[d]) / sp.nv[d] for d in range(3)]
    vc = [sp.vmin[d] + (np.arange(sp.nv[d]) + 0.5) * dv[d] for d in range(3)]
    I0 = [fac[d].sum() * dv[d] for d in range(3)]
    I1 = [(fac[d] * vc[d]).sum() * dv[d] for d in range(3)]
    I2 = [(fac[d] * vc[d] ** 2).sum() * dv[d] for d in range(3)]
    m = O.moments(3, nx, L, sp, f)
    np.testing.assert_allclose(m[0], np.prod(I0), rtol=1e-13)
    for d in range(3):
        others = np.prod([I0[e] for e in range(3) if e != d])
        np.testing.assert_allclose(m[1 + d], I1[d] * others, rtol=1e-13)
    M2 = sum(I2[d] * np.prod([I0[e] for e in range(3) if e != d]) for d in range(3))
    np.testing.assert_allclose(m[4], M2, rtol=1e-13)


@pytest.mark.parametrize("softening", [True, False])
def test_field_residual_of_a_single_mode(softening):
    """rho = cos(k x): E from Eq. 5 / Eq. 6 is c kappa/K^2 sin(k x), its
    centred difference c (kappa/K^2)(sin(k dx)/dx) cos(k x) / c, so the
    residual is cos(k x) (1 - kappa sin(k dx) / (dx K^2))."""
    nx, L, cP, m = 32, 7.0, 4 * np.pi, 3
    dx = L / nx
    x = (np.arange(nx) + 0.0) * dx
    k = 2 * np.pi * m / L
    rho = np.cos(k * x)
    E = O.poisson(nx, L, cP, softening, rho)
    kappa = np.sin(k * dx) / dx if softening else k
    K2 = (2 * np.sin(k * dx / 2) / dx) ** 2 if softening else k * k
    expect = rho * (1 - kappa * np.sin(k * dx) / (dx * K2))
    np.testing.assert_allclose(O.field_residual(nx, L, cP, rho, E), expect, atol=1e-12)


# --- Boris push with a background magnetic field (1d3v) -----------------------
def _rodrigues(v, axis, ang):
    k = axis / np.linalg.norm(axis)
    return v * np.cos(ang) + np.cross(k, v) * np.sin(ang) + k * np.dot(k, v) * (1 - np.cos(ang))


def _boris_sp():
    return O.Species(q=-1.3, m=0.7, nv=(4, 4, 4), vmin=(-5.0,) * 3, vmax=(5.0,) * 3)


def test_boris_pure_gyration_closed_form():
    """E = 0: each step rotates v about B by the Boris angle 2 atan(|t|),
    t = (q/m)(dt/2) B, in the sense of dv/dt = (q/m) v x B (about -sign(q/m) B);
    after n steps v = R(n angle) v0, |v| and v . B unchanged."""
    sp = _boris_sp()
    nx, L, dt = 8, 3.0, 0.37
    B = np.array([0.4, -1.1, 0.7])
    qm = sp.q / sp.m
    t = 0.5 * qm * dt * B
    ang = 2 * np.arctan(np.linalg.norm(t))
    v0 = np.array([[0.3], [1.2], [-0.8]])
    x = np.array([1.0])
    v = v0.copy()
    E = np.zeros(nx)
    for n in range(1, 41):
        O.push_boris(nx, L, sp, x, v, dt, E, B)
        expect = _rodrigues(v0[:, 0], -np.sign(qm) * B, n * ang)
        np.testing.assert_allclose(v[:, 0], expect, rtol=0, atol=1e-13)
    # free streaming along x with the rotating v_x
    assert 0 <= x[0] < L


def test_boris_exb_drift_is_a_fixed_point():
    """Uniform E along x perpendicular to B: the drift velocity E x B / B^2
    (force q (E + v x B) = 0) is left unchanged by every Boris step."""
    sp = _boris_sp()
    nx, L, dt = 8, 3.0, 0.2
    E0 = 0.35
    B = np.array([0.0, 0.6, -0.9])
    vd = np.cross(np.array([E0, 0.0, 0.0]), B) / np.dot(B, B)
    v = vd.reshape(3, 1).copy()
    x = np.array([0.5])
    E = np.full(nx, E0)
    for _ in range(50):
        O.push_boris(nx, L, sp, x, v, dt, E, B)
        np.testing.assert_allclose(v[:, 0], vd, rtol=0, atol=1e-13)


def test_boris_without_field_is_the_kick_push():
    """B = 0: the Boris push is the kick-drift push of Sec. 2 (two half kicks)."""
    sp = _boris_sp()
    nx, L, dt = 16, 5.0, 0.1
    rng = np.random.default_rng(4)
    n = 50
    x = rng.uniform(0, L, n)
    v = rng.uniform(-3, 3, (3, n))
    E = rng.normal(size=nx)
    x2, v2 = x.copy(), v.copy()
    O.push_boris(nx, L, sp, x, v, dt, E, np.zeros(3))
    O.push(3, nx, L, sp, x2, v2, dt, E)
    np.testing.assert_allclose(v, v2, rtol=0, atol=1e-14)
    np.testing.assert_allclose(x, x2, rtol=0, atol=1e-12)
