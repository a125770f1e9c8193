"""ctypes binding of the C ABI in include/avl.h (argument marshalling only).

Every function of the C library is exposed under its own name and returns
the avl_status integer; ``check`` turns a failing status into AvlError with
the library's message.  ``Simulation`` is a thin convenience wrapper that
moves numpy arrays or torch tensors in and out; all computation happens in
the CUDA kernels of libavl.so.  If libavl.so is missing or cannot be loaded,
importing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libavl.so")

AVL_OK, AVL_EINVAL, AVL_ENOMEM, AVL_ECUDA, AVL_ETIMEOUT, AVL_ESTATE, AVL_ENUMERIC = range(7)
AVL_FP64, AVL_FP32 = 0, 1
AVL_MAX_SPECIES = 8
STATUS_NAMES = {0: "AVL_OK", 1: "AVL_EINVAL", 2: "AVL_ENOMEM", 3: "AVL_ECUDA",
                4: "AVL_ETIMEOUT", 5: "AVL_ESTATE", 6: "AVL_ENUMERIC"}

EXPORTED = ["avl_create", "avl_destroy", "avl_last_error", "avl_init_markers", "avl_set_markers",
            "avl_marker_count", "avl_get_markers", "avl_step", "avl_get_f", "avl_get_rho",
            "avl_get_E", "avl_get_diag", "avl_get_diag_async", "avl_get_stats", "avl_field_solve", "avl_field_solve_noalloc",
            "avl_profile_steps", "avl_adjoint", "avl_create_batch", "avl_batch_run", "avl_autotune",
            "avl_get_moments", "avl_get_residual", "avl_set_bfield", "avl_record_history", "avl_refine_markers",
            "avl_synchronize", "avl_set_wait_limit"]


class avl_domain(C.Structure):
    _fields_ = [("nvdim", C.c_int32), ("nx", C.c_int32), ("L", C.c_double), ("dt", C.c_double),
                ("poisson_const", C.c_double), ("softening", C.c_int32), ("precision", C.c_int32)]


class avl_species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("mobile", C.c_int32),
                ("nv", C.c_int32 * 3), ("vmin", C.c_double * 3), ("vmax", C.c_double * 3)]


class avl_f0(C.Structure):
    _fields_ = [("nbeam", C.c_int32), ("beam_n", C.c_double * 4),
                ("beam_u", (C.c_double * 3) * 4), ("beam_vth", (C.c_double * 3) * 4),
                ("nmode", C.c_int32), ("mode", C.c_int32 * 64),
                ("amp", C.c_double * 64), ("phase", C.c_double * 64)]


class AvlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libavl.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, dp, i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)
    sig = {
        "avl_create": (C.c_int, [C.POINTER(avl_domain), C.POINTER(avl_species), C.c_int32, vp,
                                 C.POINTER(vp)]),
        "avl_destroy": (None, [vp]),
        "avl_last_error": (C.c_char_p, [vp]),
        "avl_init_markers": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(avl_f0),
                                       C.c_uint64, C.c_double]),
        "avl_set_markers": (C.c_int, [vp, C.c_int32, C.c_int64, vp, vp, vp, C.c_int32]),
        "avl_marker_count": (C.c_int, [vp, C.c_int32, i64p]),
        "avl_get_markers": (C.c_int, [vp, C.c_int32, vp, vp, vp, C.c_int32]),
        "avl_step": (C.c_int, [vp, C.c_int32]),
        "avl_get_f": (C.c_int, [vp, C.c_int32, vp, vp, C.c_int32]),
        "avl_get_rho": (C.c_int, [vp, vp, C.c_int32]),
        "avl_get_E": (C.c_int, [vp, vp, C.c_int32]),
        "avl_get_diag": (C.c_int, [vp, dp]),
        "avl_get_diag_async": (C.c_int, [vp, vp]),
        "avl_get_stats": (C.c_int, [vp, i64p]),
        "avl_field_solve": (C.c_int, [C.c_int32, C.c_double, C.c_double, C.c_int32, vp, vp, vp]),
        "avl_field_solve_noalloc": (C.c_int, [C.c_int32, C.c_double, C.c_double, C.c_int32, vp, vp, vp]),
        "avl_profile_steps": (C.c_int, [vp, C.c_int32, dp, C.c_int32]),
        "avl_adjoint": (C.c_int, [vp, C.c_int32, C.POINTER(avl_f0), C.c_int32, C.c_int32, dp, dp, dp]),
        "avl_create_batch": (C.c_int, [C.c_int32, C.POINTER(avl_domain), C.POINTER(avl_species),
                                       C.POINTER(C.c_int32), vp, C.POINTER(vp)]),
        "avl_batch_run": (C.c_int, [vp, C.c_int32, C.POINTER(vp)]),
        "avl_autotune": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_int32)]),
        "avl_get_moments": (C.c_int, [vp, C.c_int32, vp, C.c_int32]),
        "avl_get_residual": (C.c_int, [vp, vp, C.c_int32]),
        "avl_set_bfield": (C.c_int, [vp, vp]),
        "avl_record_history": (C.c_int, [vp, C.c_int32]),
        "avl_refine_markers": (C.c_int, [vp, C.c_int32, vp, vp, C.c_uint64, C.c_double, vp]),
        "avl_synchronize": (C.c_int, [vp]),
        "avl_set_wait_limit": (C.c_int, [vp, C.c_int64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()

# same names as the C ABI
avl_create = lib.avl_create
avl_destroy = lib.avl_destroy
avl_last_error = lib.avl_last_error
avl_init_markers = lib.avl_init_markers
avl_set_markers = lib.avl_set_markers
avl_marker_count = lib.avl_marker_count
avl_get_markers = lib.avl_get_markers
avl_step = lib.avl_step
avl_get_f = lib.avl_get_f
avl_get_rho = lib.avl_get_rho
avl_get_E = lib.avl_get_E
avl_get_diag = lib.avl_get_diag
avl_get_diag_async = lib.avl_get_diag_async
avl_get_stats = lib.avl_get_stats
avl_field_solve = lib.avl_field_solve
avl_field_solve_noalloc = lib.avl_field_solve_noalloc
avl_profile_steps = lib.avl_profile_steps
avl_adjoint = lib.avl_adjoint
avl_create_batch = lib.avl_create_batch
avl_batch_run = lib.avl_batch_run
avl_autotune = lib.avl_autotune
avl_get_moments = lib.avl_get_moments
avl_get_residual = lib.avl_get_residual
avl_set_bfield = lib.avl_set_bfield
avl_record_history = lib.avl_record_history
avl_refine_markers = lib.avl_refine_markers
avl_synchronize = lib.avl_synchronize
avl_set_wait_limit = lib.avl_set_wait_limit


def check(status, ctx=None):
    if status != AVL_OK:
        msg = avl_last_error(ctx)
        raise AvlError(status, msg.decode() if msg else "")
    return status


def make_domain(nvdim, nx, L, dt, poisson_const=1.0, softening=True, precision=AVL_FP64):
    return avl_domain(nvdim, nx, L, dt, poisson_const, int(bool(softening)), precision)


def make_species(q, m, nv, vmin, vmax, mobile=True):
    s = avl_species()
    s.q, s.m, s.mobile = q, m, int(bool(mobile))
    nv = list(nv) + [1] * (3 - len(nv))
    vmin = list(vmin) + [-0.5] * (3 - len(vmin))
    vmax = list(vmax) + [0.5] * (3 - len(vmax))
    for d in range(3):
        s.nv[d], s.vmin[d], s.vmax[d] = int(nv[d]), float(vmin[d]), float(vmax[d])
    return s


def make_f0(beams, modes=()):
    """beams: [(n, (ux,uy,uz), (vthx,vthy,vthz))], modes: [(mode, amp, phase)]."""
    f = avl_f0()
    f.nbeam = len(beams)
    for b, (n, u, vth) in enumerate(beams):
        f.beam_n[b] = n
        for d in range(3):
            f.beam_u[b][d] = u[d] if d < len(u) else 0.0
            f.beam_vth[b][d] = vth[d] if d < len(vth) else 1.0
    f.nmode = len(modes)
    for k, (m, a, ph) in enumerate(modes):
        f.mode[k], f.amp[k], f.phase[k] = int(m), a, ph
    return f


def _ptr(a):
    """Address of a contiguous float64 numpy array or torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data, 0
    # torch tensor
    assert a.dtype.__str__() == "torch.float64" and a.is_contiguous()
    return a.data_ptr(), int(a.is_cuda)


class Simulation:
    """Owns one avl context; numpy in/out on the host, torch tensors on the device."""

    def __init__(self, domain, species, stream=None):
        self.nvdim = domain.nvdim
        self.nx = domain.nx
        self.species = list(species)
        arr = (avl_species * len(species))(*species)
        ctx = C.c_void_p()
        st = stream if stream is not None else None
        check(avl_create(C.byref(domain), arr, len(species), st, C.byref(ctx)))
        self.ctx = ctx

    def close(self):
        if self.ctx:
            avl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        return check(st, self.ctx)

    def init_markers(self, s, lattice, f0, seed, jitter=1.0):
        lat = (C.c_int32 * 4)(*[int(a) for a in lattice])
        self._chk(avl_init_markers(self.ctx, s, lat, C.byref(f0), seed, jitter))

    def set_markers(self, s, x, v, f):
        n = x.shape[0]
        px, dx = _ptr(x)
        pv, dv = _ptr(v)
        pf, df = _ptr(f)
        assert dx == dv == df
        self._chk(avl_set_markers(self.ctx, s, n, px, pv, pf, dx))

    def marker_count(self, s):
        n = C.c_int64()
        self._chk(avl_marker_count(self.ctx, s, C.byref(n)))
        return n.value

    def get_markers(self, s):
        n = self.marker_count(s)
        x = np.zeros(n)
        v = np.zeros((self.nvdim, n))
        f = np.zeros(n)
        self._chk(avl_get_markers(self.ctx, s, x.ctypes.data, v.ctypes.data, f.ctypes.data, 0))
        return x, v, f

    def step(self, n=1):
        self._chk(avl_step(self.ctx, n))

    def profile_steps(self, n):
        """Milliseconds summed over n steps per kernel class:
        [key count + scan, push + deposit + re-sorted write, finalize, field]."""
        ms = np.zeros(4)
        self._chk(avl_profile_steps(self.ctx, n, ms.ctypes.data_as(C.POINTER(C.c_double)), 4))
        return ms

    def adjoint(self, s, theta, nsteps, ckpt_every):
        """(J, dJ/d amp (nmode,), dJ/d beam x-drift (nbeam,)) of the field
        energy after nsteps steps with the f0 of species s set to theta."""
        ga = (C.c_double * max(1, theta.nmode))()
        gu = (C.c_double * max(1, theta.nbeam))()
        J = C.c_double()
        self._chk(avl_adjoint(self.ctx, s, C.byref(theta), nsteps, ckpt_every, ga, gu, C.byref(J)))
        return J.value, np.array(ga[:theta.nmode]), np.array(gu[:theta.nbeam])

    def synchronize(self):
        self._chk(avl_synchronize(self.ctx))

    def set_wait_limit(self, polls):
        """Polls of the first bounded wait of the deposit kernels (0: give up
        at once and flag AVL_ETIMEOUT; negative: the default)."""
        self._chk(avl_set_wait_limit(self.ctx, int(polls)))

    def get_f(self, s, with_n=False):
        sp = self.species[s]
        shape = (self.nx,) + tuple(sp.nv[d] for d in range(self.nvdim))
        f = np.zeros(shape)
        n = np.zeros(shape) if with_n else None
        self._chk(avl_get_f(self.ctx, s, f.ctypes.data, n.ctypes.data if with_n else None, 0))
        return (f, n) if with_n else f

    def get_moments(self, s):
        """(2 + nvdim, nx): rho_s, j_x, (j_y, j_z), M2 of species s."""
        out = np.zeros((2 + self.nvdim, self.nx))
        self._chk(avl_get_moments(self.ctx, s, out.ctypes.data, 0))
        return out

    def record_history(self, max_steps):
        """Keep E of every state from now on (for refine_markers)."""
        self._chk(avl_record_history(self.ctx, int(max_steps)))

    def refine_markers(self, s, box, lattice, seed, jitter=1.0):
        """Add markers to the box [x0, x1) x [v0, v1) of cells of species s,
        traced back to the creation for their values; returns the count."""
        b = np.ascontiguousarray(box, dtype=np.int32).reshape(4)
        lat = np.ascontiguousarray(lattice, dtype=np.int32).reshape(2)
        added = C.c_int64(0)
        self._chk(avl_refine_markers(self.ctx, int(s), b.ctypes.data, lat.ctypes.data, int(seed), float(jitter),
                                     C.byref(added)))
        return int(added.value)

    def set_bfield(self, B):
        """Static background magnetic field (B_x, B_y, B_z) of a 1d3v run: the
        following steps use the Boris push."""
        b = np.ascontiguousarray(B, dtype=np.float64).reshape(3)
        self._chk(avl_set_bfield(self.ctx, b.ctypes.data))

    def get_residual(self):
        out = np.zeros(self.nx)
        self._chk(avl_get_residual(self.ctx, out.ctypes.data, 0))
        return out

    def get_rho(self):
        r = np.zeros(self.nx)
        self._chk(avl_get_rho(self.ctx, r.ctypes.data, 0))
        return r

    def get_E(self):
        e = np.zeros(self.nx)
        self._chk(avl_get_E(self.ctx, e.ctypes.data, 0))
        return e

    def get_diag(self):
        d = np.zeros(3 + 3 * len(self.species))
        self._chk(avl_get_diag(self.ctx, d.ctypes.data_as(C.POINTER(C.c_double))))
        return d

    def get_diag_async(self, out_ptr):
        """Enqueue the copy of the current diagnostics row to the host address
        out_ptr (page-locked, 3 + 3 nspecies doubles); valid after synchronize()."""
        self._chk(avl_get_diag_async(self.ctx, out_ptr))

    def get_stats(self):
        d = np.zeros(4 * len(self.species), dtype=np.int64)
        self._chk(avl_get_stats(self.ctx, d.ctypes.data_as(C.POINTER(C.c_int64))))
        return d.reshape(len(self.species), 4)


class Batch:
    """Independent 1d1v runs advanced together (avl_create_batch).
    runs[r] is a Simulation view of run r (owned by the batch)."""

    def __init__(self, domains, species_lists, stream=None):
        n = len(domains)
        doms = (avl_domain * n)(*domains)
        flat = [sp for lst in species_lists for sp in lst]
        sps = (avl_species * len(flat))(*flat)
        ns = (C.c_int32 * n)(*[len(lst) for lst in species_lists])
        ctx = C.c_void_p()
        check(avl_create_batch(n, doms, sps, ns, stream, C.byref(ctx)))
        self.ctx = ctx
        self.runs = []
        for r in range(n):
            sub = C.c_void_p()
            check(avl_batch_run(ctx, r, C.byref(sub)), ctx)
            v = Simulation.__new__(Simulation)
            v.nvdim, v.nx, v.species, v.ctx = 1, domains[r].nx, list(species_lists[r]), sub
            v._view = True
            self.runs.append(v)

    def _chk(self, st):
        return check(st, self.ctx)

    def step(self, n=1):
        self._chk(avl_step(self.ctx, n))

    def profile_steps(self, n):
        ms = (C.c_double * 4)()
        self._chk(avl_profile_steps(self.ctx, n, ms, 4))
        return np.array(ms[:])

    def autotune(self, trial_steps=5):
        m = C.c_int32()
        self._chk(avl_autotune(self.ctx, trial_steps, C.byref(m)))
        return m.value

    def synchronize(self):
        self._chk(avl_synchronize(self.ctx))

    def close(self):
        if self.ctx:
            for v in self.runs:
                v.ctx = None
            avl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
