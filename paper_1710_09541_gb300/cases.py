"""Seeded synthetic inputs: initial order-parameter and velocity fields and the
parameter sets of the benchmark problems of arXiv:1710.09541 (Sec. III).

This module holds no lattice Boltzmann arithmetic: it only builds the initial
conditions (Eqs. 30, 33-37 with the readings stated below) and parameter
dictionaries, so the CUDA library and the FP64 oracle start from identical
inputs.  Arrays are float64, shape [ny, nx], x fastest.

Readings:
  * Eqs. 30 and 36 print tanh(2[R - (x-x0)^2 - (y-y0)^2]/W), which mixes a
    length with squared lengths; the radial distance is used:
    tanh(2[R - sqrt((x-x0)^2 + (y-y0)^2)]/W).
  * Node centres: periodic directions use x_i = i; a walled y direction puts
    node j at y_j = j + 1/2 so that the half-way walls sit at y = 0 and y = ny.
  * Spinodal noise: phi0 = mean + amp * (2 u - 1) with u in [0, 1) the top 53
    bits of SplitMix64 (Steele, Lea & Flood 2014) applied to seed + node index.
  * Droplet impact: phi0 = max(film, drop); u0 = (0, -phi_drop U) above the
    film surface, zero at and below it (Eqs. 35-37).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each 64-bit state value in ``x`` (one step)."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): top 53 bits of SplitMix64(seed + index)."""
    idx = np.arange(n, dtype=np.uint64) + np.uint64(seed)
    return (splitmix64(idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _coords(nx, ny, walls_y):
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None] + (0.5 if walls_y else 0.0)
    return x, y


def drop(nx, ny, R, W, x0=None, y0=None, walls_y=False):
    """Circular drop (phi = 1 inside), Eq. 30 with the radial distance."""
    x, y = _coords(nx, ny, walls_y)
    x0 = nx / 2.0 if x0 is None else x0
    y0 = ny / 2.0 if y0 is None else y0
    r = np.sqrt((x - x0) ** 2 + (y - y0) ** 2)
    return 0.5 + 0.5 * np.tanh(2.0 * (R - r) / W)


def layer(nx, ny, W, y_if=None, walls_y=True):
    """Planar interface, liquid (phi = 1) below y_if, Eq. 33."""
    x, y = _coords(nx, ny, walls_y)
    y_if = ny / 2.0 if y_if is None else y_if
    return np.broadcast_to(0.5 + 0.5 * np.tanh(2.0 * (y_if - y) / W), (ny, nx)).copy()


def spinodal(nx, ny, mean=0.5, amp=0.01, seed=12345):
    """Homogeneous mixture plus seeded uniform noise, Eq. 34."""
    u = uniform01(seed, nx * ny).reshape(ny, nx)
    return mean + amp * (2.0 * u - 1.0)


def impact(nx, ny, D, film, U, W):
    """Drop of diameter D resting on a film of thickness ``film`` and moving
    down at speed U (Eqs. 35-37).  Returns (phi0, ux0, uy0)."""
    x, y = _coords(nx, ny, True)
    R = D / 2.0
    phi_film = 0.5 + 0.5 * np.tanh(2.0 * (film - y) / W)
    r = np.sqrt((x - nx / 2.0) ** 2 + (y - R - film) ** 2)
    phi_drop = 0.5 + 0.5 * np.tanh(2.0 * (R - r) / W)
    phi_film = np.broadcast_to(phi_film, (ny, nx))
    phi0 = np.maximum(phi_film, phi_drop)
    above = np.broadcast_to(y > film, (ny, nx))
    uy0 = np.where(above, -phi_drop * U, 0.0)
    ux0 = np.zeros_like(phi0)
    return phi0, ux0, uy0


# ---- parameter sets ----------------------------------------------------------
# Keys follow the C struct ``lbm_params`` (and the oracle's mirror of it).

def params_static_drop(sigma=0.01, W=4.0, tau=0.8, ratio=1000.0):
    """Static droplet: rho_H = 1, rho_L = 1/ratio, tau_h = tau_g = tau."""
    nu = (tau - 0.5) / 3.0
    return dict(rho_l=1.0, rho_g=1.0 / ratio, nu_l=nu, nu_g=nu, visc_mode=0,
                sigma=sigma, W=W, tau_h=tau, Gx=0.0, Gy=0.0, bc_y=0)


def params_poiseuille(ny, nu_l=0.1, ratio=1000.0, mu_ratio=100.0, Gx=1e-7,
                      W=4.0, sigma=1e-3, tau_h=0.8):
    """Layered Poiseuille flow with the step viscosity (Eq. 26).
    mu_ratio = mu_l / mu_g; walls in y."""
    rho_l, rho_g = 1.0, 1.0 / ratio
    mu_l = rho_l * nu_l
    mu_g = mu_l / mu_ratio
    return dict(rho_l=rho_l, rho_g=rho_g, nu_l=nu_l, nu_g=mu_g / rho_g, visc_mode=2,
                sigma=sigma, W=W, tau_h=tau_h, Gx=Gx, Gy=0.0, bc_y=1)


def params_spinodal(ratio=1000.0, sigma=1e-3, W=4.0, nu=0.1, tau_h=0.8):
    return dict(rho_l=1.0, rho_g=1.0 / ratio, nu_l=nu, nu_g=nu, visc_mode=0,
                sigma=sigma, W=W, tau_h=tau_h, Gx=0.0, Gy=0.0, bc_y=0)


def params_impact(D=200.0, U=0.04, Re=100.0, We=8000.0, ratio=1000.0,
                  mu_ratio=40.0, W=5.0, tau_h=0.8):
    """Droplet impact: mu_l = rho_l U D / Re (Eq. 38), sigma = rho_l D U^2 / We
    (Eq. 39), mu_g = mu_l / mu_ratio."""
    rho_l, rho_g = 1.0, 1.0 / ratio
    mu_l = rho_l * U * D / Re
    mu_g = mu_l / mu_ratio
    return dict(rho_l=rho_l, rho_g=rho_g, nu_l=mu_l / rho_l, nu_g=mu_g / rho_g,
                visc_mode=0, sigma=rho_l * D * U * U / We, W=W, tau_h=tau_h,
                Gx=0.0, Gy=0.0, bc_y=1)


# The single-case throughput workload: a 2048 x 2048 periodic grid holding a
# spinodal-like mixture (dense interfaces everywhere) at density ratio 1000.
PERF_NX = 2048
PERF_NY = 2048


def perf_case(nx=PERF_NX, ny=PERF_NY, seed=1):
    params = dict(rho_l=1.0, rho_g=1e-3, nu_l=0.1, nu_g=0.1, visc_mode=0,
                  sigma=1e-3, W=4.0, tau_h=0.8, Gx=0.0, Gy=0.0, bc_y=0)
    return spinodal(nx, ny, 0.5, 0.01, seed), params


def perf_drop_case(nx=PERF_NX, ny=PERF_NY, R=512.0):
    """The 2048 x 2048 grid holding one static drop of radius R (W = 4, the
    static-drop parameters): mostly bulk, against the perf case's interfaces
    everywhere, so that the two together show whether the step's speed
    depends on the data."""
    return drop(nx, ny, R, 4.0), params_static_drop()


def batch_cases(n=64, seed=7):
    """The batched sweep: n independent cases, half static drops (periodic) and
    half droplet impacts (walls), on uneven grids from 256 x 256 to
    1024 x 512 (multiples of 64), drop diameter D in [64, 160], film 0.1 D,
    impact speed 0.04, Re log-uniform in [20, 500], density ratio in
    {10, 100, 1000}.  Returns a list of dicts with nx, ny, kind, params,
    phi0, ux0, uy0 (arrays float64 [ny, nx])."""
    u = uniform01(seed, 6 * n).reshape(n, 6)
    out = []
    for c in range(n):
        nx = 256 + 64 * int(u[c, 0] * 13)            # 256 .. 1024
        ny = 256 + 64 * int(u[c, 1] * 5)             # 256 .. 512
        D = float(min(64 + int(u[c, 2] * 97), 0.6 * min(nx, ny)))
        ratio = (10.0, 100.0, 1000.0)[int(u[c, 3] * 3)]
        Re = float(20.0 * (500.0 / 20.0) ** u[c, 4])
        if c % 2 == 0:
            params = params_static_drop(ratio=ratio)
            phi0 = drop(nx, ny, D / 2, params["W"])
            ux0 = uy0 = np.zeros_like(phi0)
            kind = "static_drop"
        else:
            params = params_impact(D=D, U=0.04, Re=Re, We=8000.0, ratio=ratio, mu_ratio=40.0)
            phi0, ux0, uy0 = impact(nx, ny, D, 0.1 * D, 0.04, params["W"])
            kind = "impact"
        out.append(dict(nx=nx, ny=ny, kind=kind, params=params, phi0=phi0, ux0=ux0, uy0=uy0,
                        D=D, Re=Re, ratio=ratio))
    return out


def capillary_velocity(params):
    """sigma / mu_l: the velocity scale used to normalise velocity errors."""
    return params["sigma"] / (params["rho_l"] * params["nu_l"])


__all__ = [
    "splitmix64", "uniform01", "drop", "layer", "spinodal", "impact",
    "params_static_drop", "params_poiseuille",
    "params_spinodal", "params_impact", "perf_case", "batch_cases", "capillary_velocity",
    "PERF_NX", "PERF_NY", "perf_drop_case",
]
