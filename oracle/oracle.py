"""Python face of the FP64 CPU oracle (oracle/vhs_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check of
__graft_entry__ and by bench.py's cpu_baseline / reference leg.  Never imported
by the product package.  Marshals numpy arrays into the C routines and strings
them together in the order of the paper's time loop (Sec. 2, Fig. 2):

    init:  markers -> reconstruct f (Eq. 4) -> rho (Eq. 14) -> E (Eq. 6)
    step:  gather E at the markers + push -> reconstruct f -> rho -> E

so that after every call the stored f, rho and E belong to the current
markers.  Species with ``mobile=False`` are never pushed; their reconstructed
density stays fixed and still contributes to rho.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vhs_oracle.c")
_LIB = os.path.join(_HERE, "libvhs_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fused multiply-add)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "vhs_oracle.h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("nvdim", C.c_int32), ("nx", C.c_int32), ("L", C.c_double),
                ("nv", C.c_int32 * 3), ("vmin", C.c_double * 3), ("vmax", C.c_double * 3)]


class _F0(C.Structure):
    _fields_ = [("nbeam", C.c_int32), ("beam_n", C.c_double * 4),
                ("beam_u", (C.c_double * 3) * 4), ("beam_vth", (C.c_double * 3) * 4),
                ("nmode", C.c_int32), ("mode", C.c_int32 * 64),
                ("amp", C.c_double * 64), ("phase", C.c_double * 64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        gp = C.POINTER(_Grid)
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_jitter_uniform.restype = C.c_double
        L.orc_jitter_uniform.argtypes = [C.c_uint64, C.c_int32, C.c_int64, C.c_int32]
        L.orc_f0_eval.restype = C.c_double
        L.orc_f0_eval.argtypes = [C.POINTER(_F0), C.c_int32, C.c_double, C.c_double, dp]
        L.orc_marker_count.restype = C.c_int64
        L.orc_marker_count.argtypes = [gp, C.POINTER(C.c_int32)]
        L.orc_init_markers.restype = C.c_int64
        L.orc_init_markers.argtypes = [gp, C.POINTER(C.c_int32), C.POINTER(_F0), C.c_int32,
                                       C.c_uint64, C.c_double, dp, dp, dp]
        L.orc_reconstruct.restype = None
        L.orc_reconstruct.argtypes = [gp, C.c_int64, dp, dp, dp, dp, dp, dp]
        L.orc_moment.restype = None
        L.orc_moment.argtypes = [gp, C.c_double, dp, dp]
        L.orc_poisson.restype = None
        L.orc_poisson.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_int32, dp, dp]
        L.orc_push.restype = None
        L.orc_push.argtypes = [gp, C.c_int64, dp, dp, C.c_double, C.c_double, dp]
        L.orc_push_boris.restype = None
        L.orc_push_boris.argtypes = [gp, C.c_int64, dp, dp, C.c_double, C.c_double, dp, dp]
        L.orc_refine_markers.restype = C.c_int64
        L.orc_refine_markers.argtypes = [gp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(_F0), C.c_int32,
                                         C.c_uint64, C.c_double, C.c_double, C.c_double, C.c_int32, dp, dp, dp,
                                         dp, dp, dp]
        L.orc_diag.restype = None
        L.orc_diag.argtypes = [gp, C.c_double, dp, dp]
        L.orc_field_energy.restype = C.c_double
        L.orc_field_energy.argtypes = [C.c_int32, C.c_double, C.c_double, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class Species:
    """One plasma species: charge, mass, velocity grid (Sec. 3.1, Fig. 3)."""
    q: float
    m: float
    nv: tuple
    vmin: tuple
    vmax: tuple
    mobile: bool = True


@dataclass
class F0:
    """Initial distribution: beams x (1 + sum of cosine modes)."""
    beams: list = field(default_factory=list)   # (n, (ux,uy,uz), (vthx,vthy,vthz))
    modes: list = field(default_factory=list)   # (mode number, amplitude, phase)

    def to_c(self) -> _F0:
        s = _F0()
        s.nbeam = len(self.beams)
        assert s.nbeam <= 4 and len(self.modes) <= 64
        for b, (n, u, vth) in enumerate(self.beams):
            s.beam_n[b] = n
            for d in range(3):
                s.beam_u[b][d] = u[d] if d < len(u) else 0.0
                s.beam_vth[b][d] = vth[d] if d < len(vth) else 1.0
        s.nmode = len(self.modes)
        for k, (mnum, amp, ph) in enumerate(self.modes):
            s.mode[k] = int(mnum)
            s.amp[k] = amp
            s.phase[k] = ph
        return s


def make_grid(nvdim: int, nx: int, L: float, sp: Species) -> _Grid:
    g = _Grid()
    g.nvdim = nvdim
    g.nx = nx
    g.L = L
    for d in range(3):
        if d < nvdim:
            g.nv[d] = int(sp.nv[d])
            g.vmin[d] = float(sp.vmin[d])
            g.vmax[d] = float(sp.vmax[d])
        else:
            g.nv[d] = 1
            g.vmin[d] = -0.5
            g.vmax[d] = 0.5
    return g


def splitmix64(seed: int, n: int) -> int:
    return int(lib().orc_splitmix64(seed, n))


def f0_eval(f0: F0, nvdim: int, L: float, x: float, v) -> float:
    vv = np.zeros(3)
    vv[:len(v)] = v
    c = f0.to_c()
    return float(lib().orc_f0_eval(C.byref(c), nvdim, L, x, _dp(vv)))


def init_markers(nvdim, nx, L, sp: Species, lattice, f0: F0, species_index, seed, jitter):
    g = make_grid(nvdim, nx, L, sp)
    lat = (C.c_int32 * 4)(*[int(a) for a in lattice])
    n = int(lib().orc_marker_count(C.byref(g), lat))
    x = np.zeros(n)
    v = np.zeros(nvdim * n)
    fl = np.zeros(n)
    c = f0.to_c()
    lib().orc_init_markers(C.byref(g), lat, C.byref(c), species_index, seed, jitter,
                           _dp(x), _dp(v), _dp(fl))
    return x, v.reshape(nvdim, n), fl


def reconstruct(nvdim, nx, L, sp: Species, x, v, fl):
    """Returns (f, num, den), each shaped (nx, *nv[:nvdim])."""
    g = make_grid(nvdim, nx, L, sp)
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(nvdim, -1))
    fl = np.ascontiguousarray(fl, dtype=np.float64)
    shape = (nx,) + tuple(int(a) for a in sp.nv[:nvdim])
    f = np.zeros(shape)
    num = np.zeros(shape)
    den = np.zeros(shape)
    lib().orc_reconstruct(C.byref(g), x.size, _dp(x), _dp(v), _dp(fl), _dp(num), _dp(den), _dp(f))
    return f, num, den


def moment(nvdim, nx, L, sp: Species, f, rho=None):
    g = make_grid(nvdim, nx, L, sp)
    rho = np.zeros(nx) if rho is None else rho
    f = np.ascontiguousarray(f, dtype=np.float64)
    lib().orc_moment(C.byref(g), sp.q, _dp(f), _dp(rho))
    return rho


def poisson(nx, L, cP, softening, rho):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    E = np.zeros(nx)
    lib().orc_poisson(nx, L, cP, int(softening), _dp(rho), _dp(E))
    return E


def push(nvdim, nx, L, sp: Species, x, v, dt, E):
    """In place on x (n,) and v (nvdim, n)."""
    g = make_grid(nvdim, nx, L, sp)
    assert x.dtype == np.float64 and v.dtype == np.float64 and v.flags.c_contiguous
    lib().orc_push(C.byref(g), x.size, _dp(x), _dp(v), sp.q / sp.m, dt,
                   _dp(np.ascontiguousarray(E, dtype=np.float64)))


def push_boris(nx, L, sp: Species, x, v, dt, E, B):
    """1d3v Boris push with background field B (3,), in place on x (n,) and
    v (3, n)."""
    g = make_grid(3, nx, L, sp)
    assert x.dtype == np.float64 and v.dtype == np.float64 and v.flags.c_contiguous
    Bv = np.ascontiguousarray(B, dtype=np.float64)
    lib().orc_push_boris(C.byref(g), x.size, _dp(x), _dp(v), sp.q / sp.m, dt,
                         _dp(np.ascontiguousarray(E, dtype=np.float64)), _dp(Bv))


def refine_markers(nx, L, sp: Species, box, lattice, f0: F0, species_index, seed, jitter, dt, Ehist,
                   feet=False):
    """1d1v marker refinement by tracing back (orc_refine_markers): new markers
    on a jittered lattice[0] x lattice[1] sub-lattice of every cell of the box
    [box[0], box[1]) x [box[2], box[3]) at the current time, traced back through
    the fields Ehist (nhist, nx) of the states since the initial one, with
    f = f0 at the foot.  Returns x, v (1, n), f and, with feet=True, x0, v0."""
    g = make_grid(1, nx, L, sp)
    n = (box[1] - box[0]) * (box[3] - box[2]) * lattice[0] * lattice[1]
    Eh = np.ascontiguousarray(Ehist, dtype=np.float64).reshape(-1, nx)
    x, v, fl = np.zeros(n), np.zeros(n), np.zeros(n)
    x0, v0 = np.zeros(n), np.zeros(n)
    b = (C.c_int32 * 4)(*[int(q) for q in box])
    lat = (C.c_int32 * 2)(*[int(q) for q in lattice])
    c = f0.to_c()
    got = lib().orc_refine_markers(C.byref(g), b, lat, C.byref(c), species_index, seed, jitter, sp.q / sp.m, dt,
                                   Eh.shape[0], _dp(Eh), _dp(x), _dp(v), _dp(fl), _dp(x0), _dp(v0))
    assert got == n
    out = (x, v.reshape(1, n), fl)
    return out + (x0, v0) if feet else out


def diag(nvdim, nx, L, sp: Species, f):
    g = make_grid(nvdim, nx, L, sp)
    out = np.zeros(3)
    lib().orc_diag(C.byref(g), sp.m, _dp(np.ascontiguousarray(f, dtype=np.float64)), _dp(out))
    return out


def moments(nvdim, nx, L, sp: Species, f):
    """Velocity moments of one species' reconstructed f (Sec. 3.4.2 output
    quantities), midpoint rule over the cell-centred velocity grid like the
    charge of Eq. 14: rows [rho_s, j_x, (j_y, j_z,) M2], each (nx,):
      rho_s = q sum f dv,  j_d = q sum v_d f dv,  M2 = q sum |v|^2 f dv
    (M2 = q n <v^2>, the trace of the second moment in 1d3v)."""
    f = np.asarray(f, dtype=np.float64).reshape((nx,) + tuple(sp.nv[:nvdim]))
    dv = [(sp.vmax[d] - sp.vmin[d]) / sp.nv[d] for d in range(nvdim)]
    centres = [sp.vmin[d] + (np.arange(sp.nv[d]) + 0.5) * dv[d] for d in range(nvdim)]
    grids = np.meshgrid(*centres, indexing="ij")
    dvol = float(np.prod(dv))
    axes = tuple(range(1, nvdim + 1))
    out = [sp.q * dvol * f.sum(axis=axes)]
    for d in range(nvdim):
        out.append(sp.q * dvol * (f * grids[d]).sum(axis=axes))
    v2 = sum(g * g for g in grids)
    out.append(sp.q * dvol * (f * v2).sum(axis=axes))
    return np.array(out)


def field_residual(nx, L, cP, rho, E):
    """Charge the field solve leaves unexplained (Sec. 3.4.2):
    rho_i - (E_{i+1} - E_{i-1}) / (2 dx cP), centred difference, periodic."""
    dx = L / nx
    E = np.asarray(E, dtype=np.float64)
    return np.asarray(rho, dtype=np.float64) - (np.roll(E, -1) - np.roll(E, 1)) / (2.0 * dx * cP)


def field_energy(nx, L, cP, E):
    return float(lib().orc_field_energy(nx, L, cP, _dp(np.ascontiguousarray(E, dtype=np.float64))))


class OracleSim:
    """The whole Vlasov-Hybrid step on the CPU, in the order of Fig. 2."""

    def __init__(self, nvdim, nx, L, dt, species, cP=1.0, softening=True):
        self.nvdim, self.nx, self.L, self.dt = nvdim, nx, float(L), float(dt)
        self.cP, self.softening = float(cP), bool(softening)
        self.species = list(species)
        self.x = [None] * len(self.species)
        self.v = [None] * len(self.species)
        self.fl = [None] * len(self.species)
        self.f = [None] * len(self.species)
        self.den = [None] * len(self.species)
        self.rho_s = [np.zeros(nx) for _ in self.species]
        self.rho = np.zeros(nx)
        self.E = np.zeros(nx)
        self.B = np.zeros(3)     # background magnetic field (1d3v)
        self.nstep = 0

    def init_markers(self, s, lattice, f0: F0, seed, jitter=1.0):
        self.x[s], self.v[s], self.fl[s] = init_markers(
            self.nvdim, self.nx, self.L, self.species[s], lattice, f0, s, seed, jitter)

    def set_markers(self, s, x, v, fl):
        self.x[s] = np.array(x, dtype=np.float64)
        self.v[s] = np.array(v, dtype=np.float64).reshape(self.nvdim, -1).copy()
        self.fl[s] = np.array(fl, dtype=np.float64)

    def _reconstruct(self, s):
        sp = self.species[s]
        if self.x[s] is None:
            shape = (self.nx,) + tuple(sp.nv[:self.nvdim])
            self.f[s] = np.zeros(shape)
            self.den[s] = np.zeros(shape)
        else:
            self.f[s], _, self.den[s] = reconstruct(self.nvdim, self.nx, self.L, sp,
                                                    self.x[s], self.v[s], self.fl[s])
        self.rho_s[s] = moment(self.nvdim, self.nx, self.L, sp, self.f[s])

    def _field(self):
        rho = np.zeros(self.nx)
        for s in range(len(self.species)):
            rho += self.rho_s[s]
        self.rho = rho
        self.E = poisson(self.nx, self.L, self.cP, self.softening, rho)

    def refresh(self):
        """Reconstruct every species from its markers, then rho and E."""
        for s in range(len(self.species)):
            self._reconstruct(s)
        self._field()

    def step(self, n=1):
        for _ in range(n):
            for s, sp in enumerate(self.species):
                if sp.mobile and self.x[s] is not None:
                    if self.nvdim == 3 and np.any(self.B != 0):
                        push_boris(self.nx, self.L, sp, self.x[s], self.v[s], self.dt, self.E, self.B)
                    else:
                        push(self.nvdim, self.nx, self.L, sp, self.x[s], self.v[s], self.dt, self.E)
            for s, sp in enumerate(self.species):
                if sp.mobile:
                    self._reconstruct(s)
            self._field()
            self.nstep += 1

    def diag(self):
        """[W_E, W_kin, W_total, then per species W_kin_s, N_s, S_s]."""
        we = field_energy(self.nx, self.L, self.cP, self.E)
        per = [diag(self.nvdim, self.nx, self.L, sp, self.f[s]) for s, sp in enumerate(self.species)]
        wk = sum(p[1] for p in per)
        out = [we, wk, we + wk]
        out += [p[1] for p in per] + [p[0] for p in per] + [p[2] for p in per]
        return np.array(out)


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
