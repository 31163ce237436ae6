"""FP64 CPU oracle of the phase-field lattice Boltzmann step (arXiv:1710.09541).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of ``bench.py`` may build and call this package; the product library never
does.  It shares no code with the CUDA path.

The arithmetic lives in ``lbm_oracle.c`` (plain C, double precision, one node
at a time, in the order of the paper's Sec. II).  This module compiles it with
gcc on first use and exposes it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None


class OracleParams(ctypes.Structure):
    """Mirror of ``orc_params`` in lbm_oracle.c."""

    _fields_ = [
        ("rho_l", ctypes.c_double),
        ("rho_g", ctypes.c_double),
        ("nu_l", ctypes.c_double),
        ("nu_g", ctypes.c_double),
        ("visc_mode", ctypes.c_int),
        ("sigma", ctypes.c_double),
        ("W", ctypes.c_double),
        ("tau_h", ctypes.c_double),
        ("Gx", ctypes.c_double),
        ("Gy", ctypes.c_double),
        ("bc_y", ctypes.c_int),
        ("normal_scheme", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FP contraction so the
    x86 and Arm builds round identically, OpenMP over rows)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d = ctypes.c_double
            pd = ctypes.POINTER(ctypes.c_double)
            pi = ctypes.POINTER(ctypes.c_int)
            vp = ctypes.c_void_p
            L.orc_lattice_constants.argtypes = [pi, pi, pd, pi]
            L.orc_feq.argtypes = [d, d, d, pd]
            L.orc_geq.argtypes = [d, d, d, d, pd]
            L.orc_source_f.argtypes = [d, d, d, d, d, d, pd]
            L.orc_force_g.argtypes = [d, d, d, d, d, d, d, d, pd]
            L.orc_viscosity.argtypes = [ctypes.POINTER(OracleParams), d]
            L.orc_viscosity.restype = d
            L.orc_grad_lap.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, pd, pd, pd, pd]
            L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(OracleParams),
                                     ctypes.POINTER(vp)]
            L.orc_destroy.argtypes = [vp]
            L.orc_init.argtypes = [vp, pd, pd, pd, pd]
            L.orc_step.argtypes = [vp, ctypes.c_int]
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_set_threads.restype = ctypes.c_int
            L.orc_get_fields.argtypes = [vp, pd, pd, pd, pd, pd, pd]
            L.orc_get_state.argtypes = [vp, pd]
            L.orc_set_state.argtypes = [vp, pd]
            L.orc_sum_phi.argtypes = [vp]
            L.orc_sum_phi.restype = d
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def lattice_constants():
    """(cx, cy, w, opp) of the D2Q9 lattice as the oracle holds them (Eq. 10)."""
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    opp = (ctypes.c_int * 9)()
    lib().orc_lattice_constants(cx, cy, w, opp)
    return np.array(cx[:]), np.array(cy[:]), np.array(w[:]), np.array(opp[:])


def feq(phi, ux, uy):
    """Allen-Cahn equilibrium, Eq. 9."""
    out = np.zeros(9)
    lib().orc_feq(phi, ux, uy, _ptr(out))
    return out


def geq(p, rho, ux, uy):
    """Navier-Stokes equilibrium, Eqs. 16-17."""
    out = np.zeros(9)
    lib().orc_geq(p, rho, ux, uy, _ptr(out))
    return out


def source_f(tau_f, lam, nx, ny, dtx, dty):
    """Allen-Cahn source term F_i, Eq. 11."""
    out = np.zeros(9)
    lib().orc_source_f(tau_f, lam, nx, ny, dtx, dty, _ptr(out))
    return out


def force_g(tau_g, drho, ux, uy, gpx, gpy, Fx, Fy):
    """Navier-Stokes forcing distribution G_i, Eq. 20."""
    out = np.zeros(9)
    lib().orc_force_g(tau_g, drho, ux, uy, gpx, gpy, Fx, Fy, _ptr(out))
    return out


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops; returns the count now in use."""
    return lib().orc_set_threads(int(n))


def grad_lap(phi, bc_y=0):
    """Isotropic gradient (Eq. 27) and Laplacian (Eq. 28) of a [ny, nx] field."""
    phi = _f64(phi)
    ny, nx = phi.shape
    gx = np.zeros_like(phi)
    gy = np.zeros_like(phi)
    lap = np.zeros_like(phi)
    lib().orc_grad_lap(nx, ny, bc_y, _ptr(phi), _ptr(gx), _ptr(gy), _ptr(lap))
    return gx, gy, lap


def make_params(**kw) -> OracleParams:
    """Parameters with the library's field names; unspecified fields take the
    static-droplet defaults (rho ratio 1000, nu = 0.1, sigma = 0.01, W = 4,
    tau_h = 0.8, periodic)."""
    d = dict(rho_l=1.0, rho_g=1e-3, nu_l=0.1, nu_g=0.1, visc_mode=0, sigma=0.01,
             W=4.0, tau_h=0.8, Gx=0.0, Gy=0.0, bc_y=0, normal_scheme=0)
    d.update(kw)
    return OracleParams(**d)


def viscosity(params: OracleParams, phi: float) -> float:
    """nu(phi) by Eq. 24, 25 or 26 (visc_mode 0, 1, 2)."""
    return lib().orc_viscosity(ctypes.byref(params), phi)


class Lattice:
    """One FP64 oracle lattice: ``Lattice(nx, ny, **params)``."""

    def __init__(self, nx: int, ny: int, **params):
        self.nx, self.ny = nx, ny
        self.params = make_params(**params)
        h = ctypes.c_void_p()
        rc = lib().orc_create(nx, ny, ctypes.byref(self.params), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"orc_create failed ({rc})")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi0, ux0=None, uy0=None, p0=None):
        """Initial state from [ny, nx] fields: f = f^eq(phi0, u0) (Eq. 9),
        g = g^eq(p0, rho(phi0), u0) (Eqs. 13, 16, 17), and the (phi u) history
        phi0 u0, so d_t(phi u) starts at 0; u0 and p0 default to 0."""
        self._keep = [_f64(a) for a in (phi0, ux0, uy0, p0)]
        a = self._keep
        for x in a:
            if x is not None and x.size != self.nx * self.ny:
                raise ValueError("field size mismatch")
        lib().orc_init(self._h, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(a[3]))
        return self

    def step(self, nsteps: int = 1):
        """nsteps time steps of Eqs. 8 and 15 with everything they use
        (Sec. II), streaming with the lattice's boundary rule."""
        lib().orc_step(self._h, int(nsteps))
        return self

    def fields(self):
        """dict of phi, rho, ux, uy, p, mu as [ny, nx] float64 arrays."""
        shape = (self.ny, self.nx)
        out = {k: np.zeros(shape) for k in ("phi", "rho", "ux", "uy", "p", "mu")}
        lib().orc_get_fields(self._h, *(_ptr(out[k]) for k in ("phi", "rho", "ux", "uy", "p", "mu")))
        return out

    def get_state(self):
        """(f[9,ny,nx], g[9,ny,nx], phiu[2,ny,nx]) pre-collision state, float64."""
        N = self.nx * self.ny
        buf = np.zeros(20 * N)
        lib().orc_get_state(self._h, _ptr(buf))
        s = (self.ny, self.nx)
        return (buf[:9 * N].reshape(9, *s), buf[9 * N:18 * N].reshape(9, *s),
                buf[18 * N:].reshape(2, *s))

    def set_state(self, f, g, phiu):
        """Load a pre-collision state in the layout get_state returns."""
        buf = np.concatenate([np.ravel(f), np.ravel(g), np.ravel(phiu)]).astype(np.float64)
        if buf.size != 20 * self.nx * self.ny:
            raise ValueError("state size mismatch")
        lib().orc_set_state(self._h, _ptr(buf))
        return self

    def sum_phi(self) -> float:
        """Sum of phi (Eq. 12) over the grid, a plain running sum."""
        return lib().orc_sum_phi(self._h)
