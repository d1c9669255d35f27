"""Python access to the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle is imported by the test-suite, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline leg, and by
nothing else.  It shares no code with the CUDA library: both consume the
lab-frame particle arrays of :mod:`workloads` and nothing more.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

FIELD = {"Ax": 0, "Ay": 1, "Az": 2, "phi": 3, "Jx": 4, "Jy": 5, "Jz": 6, "rho": 7,
         "Ex": 8, "Ey": 9, "Ez": 10, "Bx": 11, "By": 12, "Bz": 13}


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (plain C11, IEEE FP64, no contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    # OpenMP runs the independent loops on all cores (same results); without it, one thread
    if subprocess.call(cmd[:-1] + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL) != 0:
        subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def threads() -> int:
    """Threads the oracle's independent loops run on (OMP_NUM_THREADS, else all cores)."""
    return int(_load().orc_threads())


def set_threads(n: int) -> None:
    """Run later steps on n threads (results do not depend on it)."""
    _load().orc_set_threads(int(n))


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double),
        ("solver", C.c_int32), ("courant", C.c_double), ("mur_order", C.c_int32),
        ("space_charge", C.c_int32), ("substeps", C.c_int32), ("periodic", C.c_int32 * 3),
        ("plane_dist", C.c_double), ("norm_freq", C.c_double),
        ("und_kind", C.c_int32), ("K", C.c_double), ("lambda_u", C.c_double),
        ("n_periods", C.c_double), ("pol_deg", C.c_double), ("waist", C.c_double),
        ("pulse_fwhm", C.c_double), ("signal", C.c_int32), ("dist_head", C.c_double),
        ("gamma", C.c_double), ("charge_e", C.c_double), ("sig_z", C.c_double),
        ("gap", C.c_double), ("n_modules", C.c_int32), ("taper", C.c_double),
        ("nf_min", C.c_double), ("nf_max", C.c_double), ("nf_points", C.c_int32), ("bunch_every", C.c_int32),
        ("seed_type", C.c_int32), ("seed_a0", C.c_double), ("seed_lambda", C.c_double),
        ("seed_pol_deg", C.c_double), ("seed_waist", C.c_double), ("seed_focus", C.c_double),
        ("seed_offset", C.c_double), ("seed_pulse_fwhm", C.c_double), ("seed_cep_deg", C.c_double),
        ("optimize_position", C.c_int32),
    ]


class Ellipsoid(C.Structure):
    _fields_ = [("uniform", C.c_int32), ("gamma", C.c_double), ("sig", C.c_double * 3),
                ("sig_u", C.c_double * 3), ("cse_sigma", C.c_double), ("lambda_r", C.c_double),
                ("bunching", C.c_double), ("bunching_phase", C.c_double), ("shot_noise", C.c_int32),
                ("charge_e", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            lib.orc_threads.restype = C.c_int
            lib.orc_set_threads.argtypes = [C.c_int]
            lib.orc_create.restype = C.c_void_p
            lib.orc_create.argtypes = [C.POINTER(Params), dp, C.c_int64]
            lib.orc_destroy.argtypes = [C.c_void_p]
            lib.orc_step.argtypes = [C.c_void_p, C.c_int64]
            lib.orc_info.argtypes = [C.c_void_p, dp]
            lib.orc_get_field.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
            lib.orc_set_field.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
            lib.orc_get_particles.argtypes = [C.c_void_p, dp]
            lib.orc_set_particles.argtypes = [C.c_void_p, dp]
            lib.orc_num_particles.restype = C.c_int64
            lib.orc_num_particles.argtypes = [C.c_void_p]
            lib.orc_series.restype = C.c_int64
            lib.orc_series.argtypes = [C.c_void_p, dp, dp, dp]
            lib.orc_diag.argtypes = [C.c_void_p, dp, dp]
            lib.orc_spectrum.restype = C.c_int64
            lib.orc_spectrum.argtypes = [C.c_void_p, dp, dp]
            lib.orc_bunch_series.restype = C.c_int64
            lib.orc_bunch_series.argtypes = [C.c_void_p, dp]
            lib.orc_external_field.argtypes = [C.c_void_p] + [C.c_double] * 4 + [dp, dp]
            lib.orc_lab_field.argtypes = [C.c_void_p] + [C.c_double] * 4 + [dp, dp]
            lib.orc_boris.argtypes = [dp, dp, dp, C.c_double]
            lib.orc_halton.restype = C.c_double
            lib.orc_halton.argtypes = [C.c_uint, C.c_uint]
            lib.orc_ellipsoid_bunch.argtypes = [C.POINTER(Ellipsoid), C.c_int64, dp]
            lib.orc_seed_potential.argtypes = [C.c_void_p] + [C.c_double] * 4 + [dp]
            lib.orc_mur.argtypes = [C.c_void_p, C.c_int]
            lib.orc_stencil.argtypes = [C.c_void_p, C.c_int]
            lib.orc_rotate_levels.argtypes = [C.c_void_p]
            lib.orc_deposit_moves.argtypes = [C.c_void_p, dp, dp, C.c_int64]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params_from(w, periodic=(0, 0, 0)) -> Params:
    """Oracle parameters from a :class:`workloads.Workload` (field by field)."""
    p = Params()
    p.nx, p.ny, p.nz = w.nx, w.ny, w.nz
    p.dx, p.dy, p.dz = w.dx, w.dy, w.dz
    p.cx = p.cy = p.cz = 0.0
    p.solver, p.courant, p.mur_order = w.solver, w.courant, w.mur_order
    p.space_charge, p.substeps = w.space_charge, w.substeps
    for a in range(3):
        p.periodic[a] = int(periodic[a])
    p.plane_dist, p.norm_freq = w.plane_dist, w.norm_freq
    p.und_kind, p.K, p.lambda_u, p.n_periods = w.und_kind, w.K, w.lambda_u, w.n_periods
    p.pol_deg, p.waist, p.pulse_fwhm, p.signal = w.pol_deg, w.waist, w.pulse_fwhm, w.signal
    p.dist_head, p.gamma, p.charge_e, p.sig_z = w.dist_head, w.gamma, w.charge_e, w.sig_z
    p.gap, p.n_modules, p.taper = w.gap, w.n_modules, w.taper
    p.nf_min, p.nf_max, p.nf_points, p.bunch_every = w.nf_min, w.nf_max, w.nf_points, w.bunch_every
    p.seed_type, p.seed_a0, p.seed_lambda, p.seed_pol_deg = w.seed_type, w.seed_a0, w.seed_lambda, w.seed_pol_deg
    p.seed_waist, p.seed_focus, p.seed_offset = w.seed_waist, w.seed_focus, w.seed_offset
    p.seed_pulse_fwhm, p.seed_cep_deg = w.seed_pulse_fwhm, w.seed_cep_deg
    p.optimize_position = w.optimize
    return p


def halton(i: int, j: int) -> float:
    return _load().orc_halton(i, j)


def ellipsoid_bunch(e: Ellipsoid, n: int) -> np.ndarray:
    out = np.zeros((n, 6))
    if n:
        _load().orc_ellipsoid_bunch(C.byref(e), n, _dp(out))
    return out


INFO_KEYS = ("gamma0", "beta0", "dx", "dy", "dz", "dt", "dtb", "A", "x0", "y0", "z0", "T0",
             "omega_h", "M", "kp", "z_ref", "q", "kstar", "kb")


class Run:
    """One oracle run (owns the C object)."""

    def __init__(self, params: Params, lab6: np.ndarray | None = None):
        self.lib = _load()
        self.p = params
        lab6 = np.zeros((0, 6)) if lab6 is None else np.ascontiguousarray(lab6, dtype=np.float64)
        self.h = self.lib.orc_create(C.byref(params), _dp(lab6), lab6.shape[0])
        self.shape = (params.nz, params.ny, params.nx)

    def close(self):
        if self.h:
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        self.lib.orc_step(self.h, int(n))

    def info(self) -> dict:
        out = np.zeros(19)
        self.lib.orc_info(self.h, _dp(out))
        return dict(zip(INFO_KEYS, out.tolist()))

    def field(self, name, lev: int = 1) -> np.ndarray:
        out = np.zeros(self.shape)
        self.lib.orc_get_field(self.h, FIELD[name] if isinstance(name, str) else int(name), lev, _dp(out))
        return out

    def set_field(self, name, lev: int, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape)
        self.lib.orc_set_field(self.h, FIELD[name] if isinstance(name, str) else int(name), lev, _dp(a))

    def particles(self) -> np.ndarray:
        n = self.lib.orc_num_particles(self.h)
        out = np.zeros((n, 6))
        if n:
            self.lib.orc_get_particles(self.h, _dp(out))
        return out

    def set_particles(self, rest6: np.ndarray):
        a = np.ascontiguousarray(rest6, dtype=np.float64)
        assert a.shape == (self.lib.orc_num_particles(self.h), 6)
        self.lib.orc_set_particles(self.h, _dp(a))

    def series(self):
        n = self.lib.orc_series(self.h, None, None, None)
        p, t, e = np.zeros(n), np.zeros(n), np.zeros(n)
        if n:
            self.lib.orc_series(self.h, _dp(p), _dp(t), _dp(e))
        return p, t, e

    def spectrum(self):
        """(h, p): normalised frequencies (nf) and lab power per step and frequency (steps x nf)."""
        nf = self.p.nf_points
        n = self.lib.orc_spectrum(self.h, None, None)
        h, p = np.zeros(max(nf, 0)), np.zeros((n, max(nf, 0)))
        if nf and n:
            self.lib.orc_spectrum(self.h, _dp(h), _dp(p))
        return h, p

    def bunch_series(self):
        """Bunch samples (rows x 15), see orc_bunch_series."""
        n = self.lib.orc_bunch_series(self.h, None)
        out = np.zeros((n, 15))
        if n:
            self.lib.orc_bunch_series(self.h, _dp(out))
        return out

    def diag(self):
        fe, b = C.c_double(), np.zeros(3)
        self.lib.orc_diag(self.h, C.byref(fe), _dp(b))
        return fe.value, float(b[0])

    def bunching_complex(self) -> complex:
        fe, b = C.c_double(), np.zeros(3)
        self.lib.orc_diag(self.h, C.byref(fe), _dp(b))
        return complex(b[1], b[2])

    def external_field(self, x, y, z, t):
        E, B = np.zeros(3), np.zeros(3)
        self.lib.orc_external_field(self.h, x, y, z, t, _dp(E), _dp(B))
        return E, B

    def seed_potential(self, x, y, z, t):
        A = np.zeros(2)
        self.lib.orc_seed_potential(self.h, x, y, z, t, _dp(A))
        return A

    def lab_field(self, x, y, zeta, t):
        E, B = np.zeros(3), np.zeros(3)
        self.lib.orc_lab_field(self.h, x, y, zeta, t, _dp(E), _dp(B))
        return E, B

    def stencil(self, c: int):
        self.lib.orc_stencil(self.h, c)

    def mur(self, c: int):
        self.lib.orc_mur(self.h, c)

    def rotate(self):
        self.lib.orc_rotate_levels(self.h)

    def deposit_moves(self, old6: np.ndarray, new6: np.ndarray):
        a = np.ascontiguousarray(old6, dtype=np.float64)
        b = np.ascontiguousarray(new6, dtype=np.float64)
        self.lib.orc_deposit_moves(self.h, _dp(a), _dp(b), a.shape[0])


def boris(u, E, B, dtb):
    """One Boris step of the normalised momentum u (electron), returns the new u."""
    lib = _load()
    u = np.array(u, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lib.orc_boris(_dp(u), _dp(E), _dp(B), float(dtb))
    return u
