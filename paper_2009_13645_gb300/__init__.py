"""Python binding of libmithra (include/mithra.h): argument marshalling only.

Every step of the FDTD/PIC time step runs in the CUDA kernels of libmithra.so.  There is no
CPU fallback: importing this package loads the library and raises if it is missing or
cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = ["lib", "Grid", "Undulator", "Bunch", "Run", "MithraError", "load", "FIELD", "KERNELS",
           "grid_from", "undulator_from", "bunch_from", "use_torch_allocator"]

OK, EINVAL, ENOMEM, ERANGE, ETIMEDOUT, EDIVERGED, ENOTFOUND, EAGAIN, ECUDA = 0, -1, -2, -3, -4, -5, -6, -7, -8
FIELD = {"Ax": 0, "Ay": 1, "Az": 2, "phi": 3, "Jx": 4, "Jy": 5, "Jz": 6, "rho": 7,
         "Ex": 8, "Ey": 9, "Ez": 10, "Bx": 11, "By": 12, "Bz": 13}
KERNELS = ("emit_eb", "push_deposit", "stencil", "mur", "power", "sort", "clear_sources")
INFO_KEYS = ("gamma0", "beta0", "dx", "dy", "dz", "dt", "dtb", "A", "x0", "y0", "z0", "T0",
             "omega_h", "M", "kp", "z_ref", "q", "kstar", "kb")


class MithraError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmithra error {code}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double),
                ("solver", C.c_int32), ("courant", C.c_double), ("mur_order", C.c_int32),
                ("space_charge", C.c_int32), ("precision", C.c_int32), ("substeps", C.c_int32),
                ("power_plane_dist", C.c_double), ("norm_freq", C.c_double), ("sort_every", C.c_int32),
                ("nf_min", C.c_double), ("nf_max", C.c_double), ("nf_points", C.c_int32),
                ("bunch_every", C.c_int32), ("optimize_position", C.c_int32)]


class Undulator(C.Structure):
    _fields_ = [("kind", C.c_int32), ("K", C.c_double), ("lambda_", C.c_double),
                ("n_periods", C.c_double), ("pol_deg", C.c_double), ("waist", C.c_double),
                ("pulse_fwhm", C.c_double), ("signal", C.c_int32), ("dist_to_bunch_head", C.c_double),
                ("gap", C.c_double), ("n_modules", C.c_int32), ("taper", C.c_double)]


class Ellipsoid(C.Structure):
    _fields_ = [("uniform", C.c_int32), ("gamma", C.c_double), ("sig", C.c_double * 3),
                ("sig_u", C.c_double * 3), ("cse_sigma", C.c_double), ("lambda_r", C.c_double),
                ("bunching", C.c_double), ("bunching_phase", C.c_double), ("shot_noise", C.c_int32),
                ("charge_e", C.c_double)]


class Seed(C.Structure):
    _fields_ = [("type", C.c_int32), ("a0", C.c_double), ("lambda_", C.c_double), ("pol_deg", C.c_double),
                ("waist", C.c_double), ("focus", C.c_double), ("offset", C.c_double),
                ("pulse_fwhm", C.c_double), ("cep_deg", C.c_double)]


class Bunch(C.Structure):
    _fields_ = [("n", C.c_int64), ("charge_e", C.c_double), ("gamma", C.c_double),
                ("sig_z", C.c_double), ("lab_particles", C.POINTER(C.c_double)),
                ("uniform", C.c_int32), ("rel_espread", C.c_double), ("sig_x", C.c_double),
                ("sig_y", C.c_double), ("eps_n_x", C.c_double), ("eps_n_y", C.c_double),
                ("cse_sigma", C.c_double), ("lambda_r", C.c_double), ("bunching", C.c_double),
                ("bunching_phase", C.c_double), ("shot_noise", C.c_int32), ("seed", C.c_uint64)]


_lib = None
_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


def load(rebuild: bool = False):
    """Load (building first when needed) paper_2009_13645_gb300/_build/libmithra.so."""
    global _lib
    if _lib is not None and not rebuild:
        return _lib
    path = _build.LIB
    if rebuild or not _build.up_to_date():
        path = _build.build(force=rebuild)
    if not os.path.exists(path):
        raise ImportError(f"libmithra.so not found at {path}")
    L = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    vp = C.c_void_p
    L.mithra_set_allocator.argtypes = [_ALLOC, _FREE, vp]
    L.mithra_create.argtypes = [C.POINTER(Grid), C.c_double, C.POINTER(Undulator), C.POINTER(Bunch), C.POINTER(vp)]
    L.mithra_set_stream.argtypes = [vp, vp]
    L.mithra_step.argtypes = [vp, C.c_int64]
    L.mithra_sync.argtypes = [vp]
    L.mithra_fields.argtypes = [vp, C.c_int, C.c_int, dp, C.c_size_t]
    L.mithra_set_field.argtypes = [vp, C.c_int, C.c_int, dp, C.c_size_t]
    L.mithra_particles.argtypes = [vp, dp, C.c_size_t]
    L.mithra_set_particles.argtypes = [vp, dp, C.c_size_t]
    L.mithra_radiated_power.argtypes = [vp, dp, dp, C.c_size_t, C.POINTER(C.c_size_t)]
    L.mithra_onaxis_field.argtypes = [vp, dp, C.c_size_t, C.POINTER(C.c_size_t)]
    L.mithra_set_seed.argtypes = [vp, C.POINTER(Seed)]
    L.mithra_ellipsoid_bunch.argtypes = [C.POINTER(Ellipsoid), C.c_int64, dp, vp]
    L.mithra_power_spectrum.argtypes = [vp, dp, dp, C.c_size_t, C.POINTER(C.c_size_t)]
    L.mithra_bunch_series.argtypes = [vp, dp, C.c_size_t, C.POINTER(C.c_size_t)]
    L.mithra_diag.argtypes = [vp, dp, dp]
    L.mithra_info.argtypes = [vp, dp, C.POINTER(C.c_int64)]
    L.mithra_set_profiling.argtypes = [vp, C.c_int]
    L.mithra_kernel_stats.argtypes = [vp, C.c_int, dp, C.POINTER(C.c_int64)]
    L.mithra_kernel_name.restype = C.c_char_p
    L.mithra_kernel_name.argtypes = [C.c_int]
    L.mithra_destroy.argtypes = [vp]
    L.mithra_destroy.restype = None
    L.mithra_last_error.restype = C.c_char_p
    L.mithra_version.restype = C.c_int
    L.mithra_kernel_launches.restype = C.c_int64
    L.mithra_serve_start.argtypes = [C.c_size_t, C.c_int, C.c_int, C.c_int]
    L.mithra_serve_start_grouped.argtypes = [C.c_size_t, C.c_int, C.c_int, C.c_int, C.c_int]
    L.mithra_serve_group_stats.argtypes = [C.POINTER(C.c_int64)]
    L.mithra_submit.argtypes = [C.POINTER(Grid), C.POINTER(Undulator), C.POINTER(Bunch), C.c_int64,
                                C.POINTER(C.c_uint64)]
    L.mithra_poll.argtypes = [C.c_uint64, C.POINTER(C.c_int), C.c_void_p]
    L.mithra_result_series.argtypes = [C.c_uint64, dp, dp, C.c_size_t, C.POINTER(C.c_size_t)]
    L.mithra_release.argtypes = [C.c_uint64]
    L.mithra_serve_stats.argtypes = [C.POINTER(C.c_int64)]
    L.mithra_serve_stop.argtypes = []
    L.mithra_field_energy_noalloc.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_int64, C.c_double,
                                              C.c_void_p, C.c_void_p]
    _lib = L
    return L


def lib():
    return load()


NOALLOC_MAX_NODES = 134217728


def mithra_field_energy_noalloc(eb_ptrs, precision: int, n: int, cell_volume: float, out_ptr: int,
                                stream: int = 0) -> None:
    """Field energy of device E/B arrays into the device double at out_ptr, with no device
    allocation (see include/mithra.h).  eb_ptrs: six device addresses (ints)."""
    L = load()
    arr = (C.c_void_p * 6)(*[C.c_void_p(int(p)) for p in eb_ptrs])
    _check(L.mithra_field_energy_noalloc(arr, int(precision), int(n), float(cell_volume),
                                         C.c_void_p(int(out_ptr)), C.c_void_p(int(stream))))


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("state", C.c_int32), ("steps", C.c_int64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("field_energy", C.c_double), ("bunching", C.c_double), ("power_last", C.c_double),
                ("power_peak", C.c_double), ("hbm_bytes", C.c_int64), ("reserved_bytes", C.c_int64)]


def serve_start(hbm_budget_bytes: int, max_active: int = 8, queue_capacity: int = 256, steps_per_chunk: int = 16,
                grouped: bool = False):
    """Start the serving loop on the current device (see include/mithra.h); grouped: ready requests
    advance together, one graph launch for all of them."""
    _check(load().mithra_serve_start_grouped(C.c_size_t(int(hbm_budget_bytes)), int(max_active), int(queue_capacity),
                                             int(steps_per_chunk), 1 if grouped else 0))


def serve_group_stats() -> dict:
    """Group launches of the running server and the request periods they advanced."""
    out = (C.c_int64 * 2)()
    _check(load().mithra_serve_group_stats(out))
    return {"group_launches": int(out[0]), "group_periods": int(out[1])}


def submit(w, lab6=None, nsteps=None, precision=None) -> int:
    """Queue one run of workload w (lab particles lab6, default: its seeded bunch)."""
    import workloads
    L = load()
    lab6 = workloads.lab_bunch(w) if lab6 is None else lab6
    b, keep = bunch_from(w, lab6)
    g, u = grid_from(w, precision), undulator_from(w)
    t = C.c_uint64()
    _check(L.mithra_submit(C.byref(g), C.byref(u), C.byref(b), int(w.steps if nsteps is None else nsteps),
                           C.byref(t)))
    return t.value


def poll(ticket: int):
    """(done, Result) of a request."""
    d = C.c_int()
    r = Result()
    _check(load().mithra_poll(C.c_uint64(ticket), C.byref(d), C.byref(r)))
    return bool(d.value), r


def result_series(ticket: int):
    L = load()
    n = C.c_size_t()
    _check(L.mithra_result_series(C.c_uint64(ticket), None, None, 0, C.byref(n)))
    p, t = np.zeros(n.value), np.zeros(n.value)
    if n.value:
        _check(L.mithra_result_series(C.c_uint64(ticket), _dp(p), _dp(t), n.value, C.byref(n)))
    return p, t


def release(ticket: int):
    _check(load().mithra_release(C.c_uint64(ticket)))


def serve_stats() -> dict:
    s = (C.c_int64 * 6)()
    _check(load().mithra_serve_stats(s))
    return dict(zip(("completed", "active", "queued", "reserved", "pool_in_use", "pool_peak"), list(s)))


def serve_stop():
    _check(load().mithra_serve_stop())


def kernel_launches() -> int:
    """CUDA kernels launched by libmithra in this process so far."""
    return int(load().mithra_kernel_launches())


def _check(rc):
    if rc != OK:
        msg = _lib.mithra_last_error().decode(errors="replace")
        raise MithraError(rc, msg)
    return rc


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


_torch_hooks = None


def use_torch_allocator(enable: bool = True):
    """Route libmithra's device allocations through PyTorch's caching allocator."""
    global _torch_hooks
    L = load()
    if not enable:
        _check(L.mithra_set_allocator(_ALLOC(), _FREE(), None))
        _torch_hooks = None
        return
    import torch

    def _alloc(ctx, nbytes):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device()))
        except Exception:
            return None

    def _free(ctx, ptr):
        torch.cuda.caching_allocator_delete(int(ptr))

    _torch_hooks = (_ALLOC(_alloc), _FREE(_free))
    _check(L.mithra_set_allocator(_torch_hooks[0], _torch_hooks[1], None))


def grid_from(w, precision=None, sort_every=0) -> Grid:
    g = Grid()
    g.nx, g.ny, g.nz = w.nx, w.ny, w.nz
    g.dx, g.dy, g.dz = w.dx, w.dy, w.dz
    g.cx = g.cy = g.cz = 0.0
    g.solver, g.courant, g.mur_order = w.solver, w.courant, w.mur_order
    g.space_charge = w.space_charge
    g.precision = w.precision if precision is None else int(precision)
    g.substeps = w.substeps
    g.power_plane_dist, g.norm_freq = w.plane_dist, w.norm_freq
    g.sort_every = int(sort_every)
    g.nf_min, g.nf_max, g.nf_points = w.nf_min, w.nf_max, w.nf_points
    g.bunch_every = w.bunch_every
    g.optimize_position = w.optimize
    return g


def ellipsoid_bunch(e: Ellipsoid, n: int, stream=None) -> np.ndarray:
    """n lab-frame macro-particles (n x 6) of a quasi-random ellipsoid bunch, computed on the GPU."""
    L = load()
    out = np.zeros((int(n), 6))
    _check(L.mithra_ellipsoid_bunch(C.byref(e), int(n), _dp(out) if n else None,
                                    C.c_void_p(int(stream)) if stream is not None else None))
    return out


def seed_from(w) -> Seed:
    s = Seed()
    s.type, s.a0, s.lambda_, s.pol_deg = w.seed_type, w.seed_a0, w.seed_lambda, w.seed_pol_deg
    s.waist, s.focus, s.offset = w.seed_waist, w.seed_focus, w.seed_offset
    s.pulse_fwhm, s.cep_deg = w.seed_pulse_fwhm, w.seed_cep_deg
    return s


def undulator_from(w) -> Undulator:
    u = Undulator()
    u.kind, u.K, u.lambda_, u.n_periods = w.und_kind, w.K, w.lambda_u, w.n_periods
    u.pol_deg, u.waist, u.pulse_fwhm, u.signal = w.pol_deg, w.waist, w.pulse_fwhm, w.signal
    u.dist_to_bunch_head = w.dist_head
    u.gap, u.n_modules, u.taper = w.gap, w.n_modules, w.taper
    return u


def bunch_from(w, lab6: np.ndarray):
    lab6 = np.ascontiguousarray(lab6, dtype=np.float64)
    b = Bunch()
    b.n = lab6.shape[0]
    b.charge_e, b.gamma, b.sig_z = w.charge_e, w.gamma, w.sig_z
    b.lab_particles = _dp(lab6) if lab6.size else C.POINTER(C.c_double)()
    return b, lab6


class Run:
    """One run on the current CUDA device (owns the libmithra handle)."""

    def __init__(self, grid: Grid, und: Undulator, bunch: Bunch, dt_lab: float = 0.0, stream=None):
        self.L = load()
        h = C.c_void_p()
        _check(self.L.mithra_create(C.byref(grid), float(dt_lab), C.byref(und), C.byref(bunch), C.byref(h)))
        self.h = h
        self.grid = grid
        self.np = int(bunch.n)
        self.shape = (grid.nz, grid.ny, grid.nx)
        if stream is not None:
            _check(self.L.mithra_set_stream(self.h, C.c_void_p(int(stream))))

    @classmethod
    def from_workload(cls, w, lab6=None, precision=None, sort_every=0, stream=None):
        import workloads
        lab6 = workloads.lab_bunch(w) if lab6 is None else lab6
        b, keep = bunch_from(w, lab6)
        r = cls(grid_from(w, precision, sort_every), undulator_from(w), b, stream=stream)
        r._keep = keep
        if getattr(w, "seed_type", -1) >= 0:
            r.set_seed(seed_from(w))
        return r

    def set_seed(self, seed: Seed):
        _check(self.L.mithra_set_seed(self.h, C.byref(seed)))

    def close(self):
        if getattr(self, "h", None):
            self.L.mithra_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        _check(self.L.mithra_step(self.h, int(n)))

    def sync(self):
        _check(self.L.mithra_sync(self.h))

    def info(self) -> dict:
        out = np.zeros(19)
        hb = C.c_int64()
        _check(self.L.mithra_info(self.h, _dp(out), C.byref(hb)))
        d = dict(zip(INFO_KEYS, out.tolist()))
        d["hbm_bytes"] = hb.value
        return d

    def field(self, name, lev: int = 1) -> np.ndarray:
        out = np.zeros(self.shape)
        w = FIELD[name] if isinstance(name, str) else int(name)
        _check(self.L.mithra_fields(self.h, w, lev, _dp(out), out.size))
        return out

    def set_field(self, name, lev: int, arr):
        a = np.ascontiguousarray(np.broadcast_to(arr, self.shape), dtype=np.float64)
        w = FIELD[name] if isinstance(name, str) else int(name)
        _check(self.L.mithra_set_field(self.h, w, lev, _dp(a), a.size))

    def particles(self) -> np.ndarray:
        out = np.zeros((self.np, 6))
        _check(self.L.mithra_particles(self.h, _dp(out), self.np))
        return out

    def set_particles(self, rest6):
        a = np.ascontiguousarray(rest6, dtype=np.float64)
        _check(self.L.mithra_set_particles(self.h, _dp(a), a.shape[0]))

    def series(self):
        n = C.c_size_t()
        _check(self.L.mithra_radiated_power(self.h, None, None, 0, C.byref(n)))
        p, t, e = np.zeros(n.value), np.zeros(n.value), np.zeros(n.value)
        if n.value:
            _check(self.L.mithra_radiated_power(self.h, _dp(p), _dp(t), n.value, C.byref(n)))
            _check(self.L.mithra_onaxis_field(self.h, _dp(e), n.value, C.byref(n)))
        return p, t, e

    def spectrum(self):
        """(h, p): the swept normalised frequencies and the lab power per step and frequency."""
        n = C.c_size_t()
        nf = int(self.grid.nf_points)
        h = np.zeros(nf)
        _check(self.L.mithra_power_spectrum(self.h, _dp(h), None, 0, C.byref(n)))
        p = np.zeros((n.value, nf))
        if n.value:
            _check(self.L.mithra_power_spectrum(self.h, None, _dp(p), p.size, C.byref(n)))
        return h, p

    def bunch_series(self):
        """Bunch samples, rows x 15 (see mithra_bunch_series)."""
        n = C.c_size_t()
        _check(self.L.mithra_bunch_series(self.h, None, 0, C.byref(n)))
        out = np.zeros((n.value, 15))
        if n.value:
            _check(self.L.mithra_bunch_series(self.h, _dp(out), n.value, C.byref(n)))
        return out

    def diag(self):
        fe = C.c_double()
        b = np.zeros(3)
        _check(self.L.mithra_diag(self.h, C.byref(fe), _dp(b)))
        return fe.value, float(b[0])

    def bunching_complex(self) -> complex:
        b = np.zeros(3)
        _check(self.L.mithra_diag(self.h, None, _dp(b)))
        return complex(b[1], b[2])

    def set_profiling(self, on: bool):
        _check(self.L.mithra_set_profiling(self.h, 1 if on else 0))

    def kernel_stats(self) -> dict:
        out = {}
        for k, name in enumerate(KERNELS):
            ms, n = C.c_double(), C.c_int64()
            _check(self.L.mithra_kernel_stats(self.h, k, C.byref(ms), C.byref(n)))
            out[name] = (ms.value, n.value)
        return out
