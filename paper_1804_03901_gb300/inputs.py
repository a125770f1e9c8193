"""Seeded synthetic workloads and marker states.

This module only holds parameters and random draws (numpy's PCG64 seeded per
workload); it contains none of the method's arithmetic.  Both the GPU tests
and the CPU oracle tests take their inputs from here.

Workloads (normalised units: omega_p = 1, lambda_D = 1, v_th,e = 1, electron
charge -1 and mass 1, Poisson constant 1):

landau      Landau damping 1d1v, FP64: electrons only (immobile neutralising
            ions are the removed k = 0 mode); nx = 64, L = 4 pi (k = 0.5),
            nv = 128 on [-6, 6]; 2 x 2 markers per cell (32768); f0 =
            Maxwellian (1 + 0.01 cos 0.5 x); dt = 0.1; 200 steps.
two_stream  Two-stream instability 1d1v, FP32: electrons 0.5 M(v-3) + 0.5
            M(v+3) with 1e-4 density perturbations in modes 1-16 (seeded
            random phases); mobile ions (m = 1836, T_i = T_e, v range
            +-10 v_th,i, unperturbed); nx = 512, L = 0.4 nx = 204.8,
            nv = 1024 on [-10, 10] v_th; 4 x 4 markers per cell (8388608 per
            species); dt = 0.05; 2000 steps.
landau_paper  The paper's own Landau run (Sec. 4.2): k = 0.4, L = 5 pi,
            nx = 512, nv = 6600 on [-10, 10], alpha = 0.05, dt = 0.1, FP64,
            2 x 2 markers per cell (13516800), 1000 steps (t = 100: linear
            damping and the first trapping oscillation).
ensemble    Batched ensemble of 256 independent 1d1v FP32 runs (run r seeded with
            the workload seed + r): nx from {64, 128, 256, 512}, nv from
            {128, 256, 512, 1024}, markers per cell from {4, 8, 16} (2x2, 2x4,
            4x4), each a Landau run (Maxwellian drifting at u, v range u +- 6,
            L = 4 pi, mode 1, dt = 0.1) or a two-stream run (beams at +-u,
            v range +-10, L = 0.4 nx, modes 1-4 with seeded phases,
            dt = 0.05) with probability 1/2; amplitude log-uniform in
            [1e-4, 1e-2], drift u uniform in [0, 4]; immobile ions as the
            removed k = 0 mode; 1000 steps.
two_stream_adjoint  Gradient of the field energy at T = 25 of a two-stream
            run, 1d1v: electrons 0.5 M(v-u) + 0.5 M(v+u), u = 3, with 16 mode
            amplitudes around 1e-4 (1e-4 (1 + 0.1 N(0,1)), seeded) and
            seeded phases; immobile ions; nx = 256, L = 102.4, nv = 512 on
            [-10, 10]; 2 x 4 markers per cell (1048576 electrons); dt = 0.05;
            500 steps; checkpoints every 50 steps.
bump_on_tail  Bump-on-tail 1d3v, FP32: electrons 0.95 M3(v; 1) + 0.05
            M3(v - 4 e_x; 0.5) (isotropic Maxwellians), density perturbation
            1e-3 cos(0.3 x); immobile ions (the removed k = 0 mode);
            nx = 256, L = 2 pi / 0.3 (k = 0.3 is mode 1), nv = 64^3 on
            [-8, 8]^3; 2 markers per cell along x (134217728); dt = 0.05;
            500 steps.
bernstein   Magnetized 1d3v, FP32, in the geometry of the electron Bernstein
            test (Sec. 4.4: a uniform field perpendicular to x): electrons
            M3(v; 1) with density perturbations 1e-3 in modes 1-8 (seeded
            phases), B = e_z with |q B / m| = 1 = omega_p (63 steps per
            gyration at dt = 0.1, above the 2 pi of Sec. 3.3); immobile
            ions (the removed k = 0 mode); nx = 256, L = 0.5 nx = 128,
            nv = 64^3 on [-6, 6]^3; 2 markers per cell along x (134217728);
            500 steps.  The paper's own run (128^3 velocity cells, about
            700 GB) does not fit one GPU.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 1804_03901


def _maxwell(n, u, vth):
    return (n, (u, 0.0, 0.0), (vth, 1.0, 1.0))


def landau(nx=64, nv=128, steps=200):
    return {
        "name": f"landau_1d1v_fp64_nx{nx}_nv{nv}",
        "nvdim": 1, "nx": nx, "L": 4 * math.pi, "dt": 0.1, "precision": "fp64",
        "species": [dict(q=-1.0, m=1.0, nv=(nv,), vmin=(-6.0,), vmax=(6.0,), mobile=True)],
        "f0": [dict(beams=[_maxwell(1.0, 0.0, 1.0)], modes=[(1, 0.01, 0.0)])],
        "lattice": [(2, 2, 1, 1)],
        "seed": BASE_SEED + 0, "jitter": 1.0, "steps": steps,
    }


def two_stream(nx=512, nv=1024, lattice=(4, 4, 1, 1), steps=2000, nmodes=16, amp=1e-4):
    rng = np.random.default_rng(BASE_SEED + 1)
    phases = rng.uniform(0.0, 2 * math.pi, nmodes)
    vthi = 1836.0 ** -0.5
    return {
        "name": f"two_stream_1d1v_fp32_nx{nx}_nv{nv}",
        "nvdim": 1, "nx": nx, "L": 0.4 * nx, "dt": 0.05, "precision": "fp32",
        "species": [dict(q=-1.0, m=1.0, nv=(nv,), vmin=(-10.0,), vmax=(10.0,), mobile=True),
                    dict(q=1.0, m=1836.0, nv=(nv,), vmin=(-10.0 * vthi,), vmax=(10.0 * vthi,),
                         mobile=True)],
        "f0": [dict(beams=[_maxwell(0.5, 3.0, 1.0), _maxwell(0.5, -3.0, 1.0)],
                    modes=[(m + 1, amp, float(phases[m])) for m in range(nmodes)]),
               dict(beams=[_maxwell(1.0, 0.0, vthi)], modes=[])],
        "lattice": [tuple(lattice), tuple(lattice)],
        "seed": BASE_SEED + 1, "jitter": 1.0, "steps": steps,
    }


def landau_paper(nx=512, nv=6600, steps=1000, lattice=(2, 2, 1, 1)):
    return {
        "name": f"landau_paper_1d1v_fp64_nx{nx}_nv{nv}",
        "nvdim": 1, "nx": nx, "L": 5 * math.pi, "dt": 0.1, "precision": "fp64",
        "species": [dict(q=-1.0, m=1.0, nv=(nv,), vmin=(-10.0,), vmax=(10.0,), mobile=True)],
        "f0": [dict(beams=[_maxwell(1.0, 0.0, 1.0)], modes=[(1, 0.05, 0.0)])],
        "lattice": [tuple(lattice)],
        "seed": BASE_SEED + 5, "jitter": 1.0, "steps": steps,
    }


def ensemble(nrun=256, steps=1000):
    rng = np.random.default_rng(BASE_SEED + 4)
    runs = []
    for r in range(nrun):
        nx = int(rng.choice([64, 128, 256, 512]))
        nv = int(rng.choice([128, 256, 512, 1024]))
        lat = [(2, 2, 1, 1), (2, 4, 1, 1), (4, 4, 1, 1)][int(rng.integers(3))]
        amp = float(math.exp(rng.uniform(math.log(1e-4), math.log(1e-2))))
        u = float(rng.uniform(0.0, 4.0))
        if rng.uniform() < 0.5:
            run = {"type": "landau", "nx": nx, "L": 4 * math.pi, "dt": 0.1,
                   "species": [dict(q=-1.0, m=1.0, nv=(nv,), vmin=(u - 6.0,), vmax=(u + 6.0,), mobile=True)],
                   "f0": [dict(beams=[_maxwell(1.0, u, 1.0)], modes=[(1, amp, 0.0)])]}
        else:
            ph = rng.uniform(0.0, 2 * math.pi, 4)
            run = {"type": "two_stream", "nx": nx, "L": 0.4 * nx, "dt": 0.05,
                   "species": [dict(q=-1.0, m=1.0, nv=(nv,), vmin=(-10.0,), vmax=(10.0,), mobile=True)],
                   "f0": [dict(beams=[_maxwell(0.5, u, 1.0), _maxwell(0.5, -u, 1.0)],
                               modes=[(m + 1, amp, float(ph[m])) for m in range(4)])]}
        run["lattice"] = [lat]
        run["seed"] = BASE_SEED + 4 + r
        runs.append(run)
    return {"name": f"ensemble_{nrun}_runs_1d1v_fp32", "nvdim": 1, "precision": "fp32", "runs": runs,
            "jitter": 1.0, "steps": steps}


def two_stream_adjoint(nx=256, nv=512, lattice=(2, 4, 1, 1), steps=500, ckpt=50, nmodes=16):
    rng = np.random.default_rng(BASE_SEED + 3)
    amps = 1e-4 * (1.0 + 0.1 * rng.standard_normal(nmodes))
    phases = rng.uniform(0.0, 2 * math.pi, nmodes)
    vthi = 1836.0 ** -0.5
    return {
        "name": f"two_stream_adjoint_1d1v_nx{nx}_nv{nv}",
        "nvdim": 1, "nx": nx, "L": 0.4 * nx, "dt": 0.05, "precision": "fp32",
        "species": [dict(q=-1.0, m=1.0, nv=(nv,), vmin=(-10.0,), vmax=(10.0,), mobile=True),
                    dict(q=1.0, m=1836.0, nv=(nv,), vmin=(-10.0 * vthi,), vmax=(10.0 * vthi,),
                         mobile=False)],
        "f0": [dict(beams=[_maxwell(0.5, 3.0, 1.0), _maxwell(0.5, -3.0, 1.0)],
                    modes=[(m + 1, float(amps[m]), float(phases[m])) for m in range(nmodes)]),
               dict(beams=[_maxwell(1.0, 0.0, vthi)], modes=[])],
        "lattice": [tuple(lattice), tuple(lattice)],
        "seed": BASE_SEED + 3, "jitter": 1.0, "steps": steps, "ckpt": ckpt,
    }


def bump_on_tail(nx=256, nv=64, lattice=(2, 1, 1, 1), steps=500):
    return {
        "name": f"bump_on_tail_1d3v_fp32_nx{nx}_nv{nv}^3",
        "nvdim": 3, "nx": nx, "L": 2 * math.pi / 0.3, "dt": 0.05, "precision": "fp32",
        "species": [dict(q=-1.0, m=1.0, nv=(nv,) * 3, vmin=(-8.0,) * 3, vmax=(8.0,) * 3, mobile=True)],
        "f0": [dict(beams=[(0.95, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)),
                           (0.05, (4.0, 0.0, 0.0), (0.5, 0.5, 0.5))],
                    modes=[(1, 1e-3, 0.0)])],
        "lattice": [tuple(lattice)],
        "seed": BASE_SEED + 2, "jitter": 1.0, "steps": steps,
    }


def bernstein(nx=256, nv=64, lattice=(2, 1, 1, 1), steps=500, nmode=8):
    rng = np.random.default_rng(BASE_SEED + 5)
    phases = rng.uniform(0.0, 2 * math.pi, nmode)
    return {
        "name": f"bernstein_1d3v_fp32_nx{nx}_nv{nv}^3_Bz1",
        "nvdim": 3, "nx": nx, "L": 0.5 * nx, "dt": 0.1, "precision": "fp32",
        "species": [dict(q=-1.0, m=1.0, nv=(nv,) * 3, vmin=(-6.0,) * 3, vmax=(6.0,) * 3, mobile=True)],
        "f0": [dict(beams=[(1.0, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))],
                    modes=[(m + 1, 1e-3, float(phases[m])) for m in range(nmode)])],
        "lattice": [tuple(lattice)],
        "B": (0.0, 0.0, 1.0),
        "seed": BASE_SEED + 6, "jitter": 1.0, "steps": steps,
    }


def random_markers(seed, n, L, vmin, vmax, v_overhang=0.05, fmin=1e-12, fmax=1.0):
    """Markers scattered uniformly in x and v (a few percent of them beyond
    the velocity grid), values log-uniform over [fmin, fmax]; values are made
    distinct so that two marker sets can be matched by value."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, L, n)
    span = vmax - vmin
    v = rng.uniform(vmin - v_overhang * span, vmax + v_overhang * span, n)
    f = np.exp(rng.uniform(math.log(fmin), math.log(fmax), n))
    # distinct values even after rounding to FP32
    f = np.unique(f.astype(np.float32)).astype(np.float64)
    while f.size < n:
        extra = np.exp(rng.uniform(math.log(fmin), math.log(fmax), n - f.size)).astype(np.float32)
        f = np.unique(np.concatenate([f.astype(np.float32), extra])).astype(np.float64)
    f = rng.permutation(f[:n])
    return x, v, f


def boundary_markers3(seed, n, nx, L, nv, vmin, vmax):
    """1d3v markers on the places where a cloud-in-cell weight is 0 or 1:
    x at 0, at the cell edges and centres and one rounding below L; each
    velocity component at the dual-row boundaries (cell centres), at vmin,
    at vmax, one rounding below vmax and a quarter cell below vmin.  f over
    three decades, distinct for every marker."""
    rng = np.random.default_rng(seed)
    dx = L / nx
    nv, vmin, vmax = np.asarray(nv), np.asarray(vmin, float), np.asarray(vmax, float)
    dv = (vmax - vmin) / nv
    xs = np.concatenate([[0.0, np.nextafter(L, 0.0)], dx * np.arange(nx), dx * (np.arange(nx) + 0.5)])
    x = xs[rng.integers(0, xs.size, n)]
    v = np.empty((3, n))
    for d in range(3):
        rows = np.concatenate([vmin[d] + dv[d] * (np.arange(-1, nv[d] + 1) + 0.5),
                               [vmin[d], vmax[d], np.nextafter(vmax[d], -np.inf), vmin[d] - 0.25 * dv[d]]])
        v[d] = rows[rng.integers(0, rows.size, n)]
    f = np.exp(rng.uniform(-3.0 * math.log(10.0), 0.0, n)) * (1.0 + 1e-9 * np.arange(n))
    return x, v, f


def random_markers3(seed, n, L, vmin, vmax, v_overhang=0.05, fmin=1e-12, fmax=1.0):
    """1d3v version of random_markers: v has shape (3, n), each component
    uniform over its range widened by v_overhang on both sides."""
    rng = np.random.default_rng(seed)
    x, _, f = random_markers(seed + 7919, n, L, vmin[0], vmax[0], v_overhang, fmin, fmax)
    v = np.empty((3, n))
    for d in range(3):
        span = vmax[d] - vmin[d]
        v[d] = rng.uniform(vmin[d] - v_overhang * span, vmax[d] + v_overhang * span, n)
    return x, v, f

