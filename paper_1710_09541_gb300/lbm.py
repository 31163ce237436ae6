"""ctypes binding of the C ABI in include/lbm_pf.h (argument marshalling only;
every step of the lattice update runs in the CUDA library).

The library must have been built (``python -m paper_1710_09541_gb300.build``
or ``__graft_entry__.build()``); importing this module without it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "liblbm_pf.so")

LBM_OK = 0
LBM_ERR_INVALID = -1
LBM_ERR_CUDA = -2
LBM_ERR_STATE = -3
LBM_ERR_NONFINITE = -4
LBM_ERR_OOM = -5
_STATUS = {0: "LBM_OK", -1: "LBM_ERR_INVALID", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_STATE",
           -4: "LBM_ERR_NONFINITE", -5: "LBM_ERR_OOM"}

LBM_VISC_LINEAR_NU, LBM_VISC_INVERSE_NU, LBM_VISC_STEP_MU = 0, 1, 2
LBM_BC_PERIODIC, LBM_BC_WALLS, LBM_BC_WALL_OPEN = 0, 1, 2
LBM_NORMAL_CENTRAL, LBM_NORMAL_LOCAL = 0, 1
LBM_STORE_FP32, LBM_STORE_FP16_SHIFTED, LBM_STORE_BF16_SHIFTED, LBM_STORE_BF16_SHIFTED_SR = 0, 1, 2, 3
LBM_KERNEL_AUTO, LBM_KERNEL_GENERIC = 0, 1

# every entry point include/lbm_pf.h declares
EXPORTS = ("lbm_create", "lbm_init", "lbm_step", "lbm_get_fields", "lbm_state_bytes",
           "lbm_get_state", "lbm_set_state", "lbm_diag", "lbm_synchronize", "lbm_destroy",
           "lbm_last_error", "lbm_diag_fields_noalloc", "lbm_batch_create", "lbm_batch_step",
           "lbm_batch_info", "lbm_batch_destroy", "lbm_batch_last_error",
           "lbm_spreading_radius", "lbm_probe", "lbm_workspace_bytes", "lbm_create_in",
           "lbm_laplace_jump")


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("nu_l", ctypes.c_double), ("nu_g", ctypes.c_double),
        ("visc_mode", ctypes.c_int),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double),
        ("tau_h", ctypes.c_double),
        ("Gx", ctypes.c_double), ("Gy", ctypes.c_double),
        ("bc_y", ctypes.c_int), ("normal_scheme", ctypes.c_int),
        ("storage", ctypes.c_int), ("check_every", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("kernel", ctypes.c_int),
    ]


_lib = None


def load() -> ctypes.CDLL:
    """Load liblbm_pf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"CUDA library not built: {_LIB_PATH} is missing "
                          "(run python -m paper_1710_09541_gb300.build)")
    L = ctypes.CDLL(_LIB_PATH)
    vp, pd, i, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_size_t
    L.lbm_create.argtypes = [i, i, ctypes.POINTER(lbm_params), ctypes.POINTER(vp)]
    L.lbm_init.argtypes = [vp, pd, pd, pd, pd]
    L.lbm_step.argtypes = [vp, i]
    L.lbm_get_fields.argtypes = [vp, pd, pd, pd, pd, pd]
    L.lbm_state_bytes.argtypes = [vp]
    L.lbm_state_bytes.restype = sz
    L.lbm_get_state.argtypes = [vp, vp, sz]
    L.lbm_set_state.argtypes = [vp, vp, sz]
    L.lbm_diag.argtypes = [vp, pd, pd, pd, pd]
    L.lbm_synchronize.argtypes = [vp]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_diag_fields_noalloc.argtypes = [vp, sz, vp, vp, ctypes.c_char_p, sz]
    L.lbm_spreading_radius.argtypes = [vp, i, i, pd, pd]
    L.lbm_laplace_jump.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, pd]
    L.lbm_workspace_bytes.argtypes = [i, i, ctypes.POINTER(lbm_params), ctypes.POINTER(sz)]
    L.lbm_create_in.argtypes = [i, i, ctypes.POINTER(lbm_params), vp, sz, ctypes.POINTER(vp)]
    pi = ctypes.POINTER(ctypes.c_int)
    L.lbm_probe.argtypes = [vp, i, pi, pi, pd, pd, pd, pd, pd]
    L.lbm_diag_fields_noalloc.restype = ctypes.c_int
    L.lbm_batch_create.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.lbm_batch_create.restype = ctypes.c_int
    L.lbm_batch_step.argtypes = [vp, i]
    L.lbm_batch_step.restype = ctypes.c_int
    L.lbm_batch_info.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), pd,
                                  ctypes.POINTER(i)]
    L.lbm_batch_info.restype = ctypes.c_int
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    L.lbm_batch_last_error.argtypes = [vp]
    L.lbm_batch_last_error.restype = ctypes.c_char_p
    for name in ("lbm_create", "lbm_init", "lbm_step", "lbm_get_fields", "lbm_get_state",
                 "lbm_set_state", "lbm_diag", "lbm_synchronize"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def make_params(stream=None, **kw) -> lbm_params:
    """lbm_params from keyword arguments (names as in the C struct).  stream:
    an integer cudaStream_t, an object with ``cuda_stream`` (torch.cuda.Stream)
    or None for the default stream."""
    d = dict(rho_l=1.0, rho_g=1e-3, nu_l=0.1, nu_g=0.1, visc_mode=0, sigma=0.01, W=4.0,
             tau_h=0.8, Gx=0.0, Gy=0.0, bc_y=0, normal_scheme=0, storage=0, check_every=0,
             kernel=0)
    unknown = set(kw) - set(d)
    if unknown:
        raise TypeError(f"unknown parameters: {sorted(unknown)}")
    d.update(kw)
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    return lbm_params(stream=stream or None, **d)


def diag_fields_noalloc(d_fields: int, n: int, d_out: int, stream=None) -> None:
    """lbm_diag_fields_noalloc: reduce caller-owned device fields (5*n doubles,
    planes phi, rho, ux, uy, p) into 4 device doubles at d_out without any
    allocation.  d_fields/d_out are device addresses (e.g. tensor.data_ptr())."""
    L = load()
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    err = ctypes.create_string_buffer(256)
    rc = L.lbm_diag_fields_noalloc(d_fields, n, d_out, stream or None, err, len(err))
    if rc != LBM_OK:
        raise LbmError(rc, err.value.decode())


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def workspace_bytes(nx: int, ny: int, **params) -> int:
    """lbm_workspace_bytes: device bytes an nx x ny lattice needs."""
    L = load()
    p = make_params(**params)
    n = ctypes.c_size_t()
    rc = L.lbm_workspace_bytes(int(nx), int(ny), ctypes.byref(p), ctypes.byref(n))
    if rc != LBM_OK:
        raise LbmError(rc, "lbm_workspace_bytes failed (see stderr)")
    return n.value


class Lattice:
    """One lattice on the current CUDA device: ``Lattice(nx, ny, **params)``.

    With ``workspace`` (a contiguous CUDA tensor of at least
    ``workspace_bytes(nx, ny, **params)`` bytes) the device state lives in that
    tensor (lbm_create_in); the lattice keeps a reference to it."""

    def __init__(self, nx: int, ny: int, stream=None, workspace=None, **params):
        self._L = load()
        self.nx, self.ny = int(nx), int(ny)
        self.params = make_params(stream=stream, **params)
        h = ctypes.c_void_p()
        if workspace is None:
            rc = self._L.lbm_create(self.nx, self.ny, ctypes.byref(self.params), ctypes.byref(h))
        else:
            if not workspace.is_contiguous():
                raise ValueError("workspace must be contiguous")
            nbytes = workspace.numel() * workspace.element_size()
            rc = self._L.lbm_create_in(self.nx, self.ny, ctypes.byref(self.params),
                                       workspace.data_ptr(), nbytes, ctypes.byref(h))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_create failed (see stderr)")
        self._workspace = workspace
        self._h = h

    # -- helpers -------------------------------------------------------------
    def _check(self, rc):
        if rc != LBM_OK:
            raise LbmError(rc, self._L.lbm_last_error(self._h).decode())

    def _in(self, a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.size != self.nx * self.ny:
            raise ValueError(f"expected {self.nx * self.ny} values, got {a.size}")
        return a

    # -- API -----------------------------------------------------------------
    def init(self, phi0, ux0=None, uy0=None, p0=None):
        a = [self._in(x) for x in (phi0, ux0, uy0, p0)]
        self._check(self._L.lbm_init(self._h, *(_dptr(x) for x in a)))
        return self

    def step(self, nsteps: int = 1):
        self._check(self._L.lbm_step(self._h, int(nsteps)))
        return self

    def fields(self, out=None):
        """dict phi, rho, ux, uy, p of shape [ny, nx] (float64).  ``out`` may
        supply preallocated (e.g. pinned) arrays for some or all keys."""
        out = dict(out or {})
        for k in ("phi", "rho", "ux", "uy", "p"):
            if k not in out:
                out[k] = np.empty((self.ny, self.nx))
        self._check(self._L.lbm_get_fields(self._h, *(_dptr(out[k]) for k in
                                                      ("phi", "rho", "ux", "uy", "p"))))
        return out

    def state_bytes(self) -> int:
        return int(self._L.lbm_state_bytes(self._h))

    def get_state(self):
        """(f[9,ny,nx], g[9,ny,nx], phiu[2,ny,nx]) as float32, pre-collision."""
        N = self.nx * self.ny
        buf = np.empty(20 * N, dtype=np.float32)
        self._check(self._L.lbm_get_state(self._h, buf.ctypes.data, buf.nbytes))
        s = (self.ny, self.nx)
        return buf[:9 * N].reshape(9, *s), buf[9 * N:18 * N].reshape(9, *s), buf[18 * N:].reshape(2, *s)

    def set_state(self, f, g, phiu):
        buf = np.ascontiguousarray(np.concatenate([np.ravel(f), np.ravel(g), np.ravel(phiu)]),
                                   dtype=np.float32)
        self._check(self._L.lbm_set_state(self._h, buf.ctypes.data, buf.nbytes))
        return self

    def diag(self):
        """(sum phi, max |u|, min p, max p) of the current state."""
        r = [ctypes.c_double() for _ in range(4)]
        self._check(self._L.lbm_diag(self._h, *(ctypes.byref(x) for x in r)))
        return tuple(x.value for x in r)

    def spreading_radius(self, y: int, xc: int | None = None):
        """(r, r_interp) on row y around column xc (default nx // 2)."""
        r, ri = ctypes.c_double(), ctypes.c_double()
        xc = self.nx // 2 if xc is None else int(xc)
        self._check(self._L.lbm_spreading_radius(self._h, int(y), xc, ctypes.byref(r),
                                                 ctypes.byref(ri)))
        return r.value, ri.value

    def laplace_jump(self, xc: float, yc: float, r_in: float, r_out: float) -> float:
        """Mean p inside r_in of (xc, yc) minus mean p outside r_out (lbm_laplace_jump)."""
        dp = ctypes.c_double()
        self._check(self._L.lbm_laplace_jump(self._h, float(xc), float(yc), float(r_in),
                                             float(r_out), ctypes.byref(dp)))
        return dp.value

    def probe(self, x, y):
        """Fields at nodes (x[j], y[j]): dict of float64 arrays phi, rho, ux, uy, p."""
        x = np.ascontiguousarray(x, dtype=np.int32).ravel()
        y = np.ascontiguousarray(y, dtype=np.int32).ravel()
        if x.shape != y.shape:
            raise ValueError("x and y need the same length")
        out = {k: np.empty(x.size, dtype=np.float64) for k in ("phi", "rho", "ux", "uy", "p")}
        pi = ctypes.POINTER(ctypes.c_int)
        self._check(self._L.lbm_probe(self._h, x.size, x.ctypes.data_as(pi), y.ctypes.data_as(pi),
                                      *(_dptr(out[k]) for k in ("phi", "rho", "ux", "uy", "p"))))
        return out

    def synchronize(self):
        self._check(self._L.lbm_synchronize(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbm_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many Lattice cases stepped together (lbm_batch_*).  The lattices stay
    owned by the caller and must outlive the batch."""

    def __init__(self, lattices):
        self._L = load()
        self.lattices = list(lattices)
        arr = (ctypes.c_void_p * len(self.lattices))(*(lat._h.value for lat in self.lattices))
        h = ctypes.c_void_p()
        rc = self._L.lbm_batch_create(len(self.lattices), arr, ctypes.byref(h))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_batch_create failed (see stderr)")
        self._h = h

    def step(self, nsteps: int = 1):
        rc = self._L.lbm_batch_step(self._h, int(nsteps))
        if rc != LBM_OK:
            raise LbmError(rc, self._L.lbm_batch_last_error(self._h).decode())
        return self

    def info(self):
        """{"periodic": {...}, "walls": {...}, "tuned": bool}; per class the
        number of cases, the tile shape (width, height) in use and its
        microseconds per step at tuning."""
        out = {}
        for cls, name in ((0, "periodic"), (1, "walls")):
            n, tx, ty, tuned = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            us = ctypes.c_double()
            rc = self._L.lbm_batch_info(self._h, cls, ctypes.byref(n), ctypes.byref(tx),
                                        ctypes.byref(ty), ctypes.byref(us), ctypes.byref(tuned))
            if rc != LBM_OK:
                raise LbmError(rc, "lbm_batch_info failed")
            out[name] = {"cases": n.value, "tile": (tx.value, ty.value), "us": us.value}
            out["tuned"] = bool(tuned.value)
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbm_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
