"""Second, independent transcription of one time step of the phase-field LB
model of arXiv:1710.09541, written with whole-array NumPy operations (np.roll
for streaming) instead of the oracle's node loops.  Used only to cross-check
the C oracle on tiny grids; it shares no code with it.

State: f, g of shape [9, ny, nx] (pre-collision), phiu of shape [2, ny, nx].
"""
import numpy as np

# Eq. 10, built from the paper's trigonometric definition of c_i
_ang = np.array([0.0] + [(i - 1) * np.pi / 2 for i in range(1, 5)]
                + [(i - 5) * np.pi / 2 + np.pi / 4 for i in range(5, 9)])
_len = np.array([0.0] + [1.0] * 4 + [np.sqrt(2.0)] * 4)
CX = np.rint(_len * np.cos(_ang)).astype(int)
CY = np.rint(_len * np.sin(_ang)).astype(int)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = np.array([int(np.where((CX == -CX[i]) & (CY == -CY[i]))[0][0]) for i in range(9)])


def _shift(a, dx, dy, walls):
    """a(x + dx, y + dy) on the grid; periodic in x, and in y periodic or
    mirrored (ghost row equals the first/last row) when walls is set."""
    out = np.roll(a, shift=(-dy, -dx), axis=(0, 1))
    if walls and dy != 0:
        rolled_x = np.roll(a, shift=-dx, axis=1)
        if dy > 0:
            out[-1, :] = rolled_x[-1, :]
        else:
            out[0, :] = rolled_x[0, :]
    return out


def moments(f, g, p, walls):
    phi = f.sum(axis=0)
    gx = sum(3.0 * W[i] * CX[i] * _shift(phi, CX[i], CY[i], walls) for i in range(1, 9))
    gy = sum(3.0 * W[i] * CY[i] * _shift(phi, CX[i], CY[i], walls) for i in range(1, 9))
    lap = sum(6.0 * W[i] * (_shift(phi, CX[i], CY[i], walls) - phi) for i in range(1, 9))
    drho = p["rho_l"] - p["rho_g"]
    rho = phi * drho + p["rho_g"]
    sig, Wd = p["sigma"], p["W"]
    mu = 4 * (12 * sig / Wd) * phi * (phi - 1) * (phi - 0.5) - 1.5 * sig * Wd * lap
    Fx = mu * gx + p["Gx"]
    Fy = mu * gy + p["Gy"]
    ux = ((CX[:, None, None] * g).sum(0) + Fx / 2) / rho
    uy = ((CY[:, None, None] * g).sum(0) + Fy / 2) / rho
    s0 = W[0] * (-1.5) * (ux ** 2 + uy ** 2)
    pr = 0.6 * (g[1:].sum(0) + 0.5 * drho * (ux * gx + uy * gy) + rho * s0)
    return dict(phi=phi, gx=gx, gy=gy, lap=lap, rho=rho, mu=mu, Fx=Fx, Fy=Fy, ux=ux, uy=uy, p=pr)


def nu_of(phi, p):
    if p["visc_mode"] == 1:
        return 1.0 / (phi * (1 / p["nu_l"] - 1 / p["nu_g"]) + 1 / p["nu_g"])
    if p["visc_mode"] == 2:
        rho = phi * (p["rho_l"] - p["rho_g"]) + p["rho_g"]
        return np.where(phi >= 0.5, p["rho_l"] * p["nu_l"], p["rho_g"] * p["nu_g"]) / rho
    return phi * (p["nu_l"] - p["nu_g"]) + p["nu_g"]


def _open_top(f, g):
    """Open top (bc_y = 2): the top row's incoming populations (c_y = -1)
    repeat the row below's (zero normal gradient)."""
    down = np.where(CY == -1)[0]
    f[down, -1, :] = f[down, -2, :]
    g[down, -1, :] = g[down, -2, :]


def init(phi0, ux0, uy0, p0, p):
    rho = phi0 * (p["rho_l"] - p["rho_g"]) + p["rho_g"]
    cu = CX[:, None, None] * ux0 + CY[:, None, None] * uy0
    usq = ux0 ** 2 + uy0 ** 2
    f = W[:, None, None] * phi0 * (1 + 3 * cu)
    s = W[:, None, None] * (3 * cu + 4.5 * cu ** 2 - 1.5 * usq)
    g = 3 * p0 * W[:, None, None] + rho * s
    g[0] -= 3 * p0
    if p.get("bc_y", 0) == 2:
        _open_top(f, g)
    return f, g, np.stack([phi0 * ux0, phi0 * uy0])


def step(f, g, phiu, p):
    walls = p["bc_y"] in (1, 2)
    m = moments(f, g, p, walls)
    phi, ux, uy, rho = m["phi"], m["ux"], m["uy"], m["rho"]
    tau_f = p["tau_h"]
    tau_g = 3 * nu_of(phi, p) + 0.5
    drho = p["rho_l"] - p["rho_g"]
    lam = 4 * phi * (1 - phi) / p["W"]
    Dx = phi * ux - phiu[0]
    Dy = phi * uy - phiu[1]
    if p.get("normal_scheme", 0) == 1:
        # Eq. 29: n along -C, C = first moment of the non-equilibrium part plus
        # half the time derivative of phi u
        neq = [f[i] - W[i] * phi * (1 + 3 * (CX[i] * ux + CY[i] * uy)) for i in range(9)]
        vx = sum(CX[i] * neq[i] for i in range(9)) + 0.5 * Dx
        vy = sum(CY[i] * neq[i] for i in range(9)) + 0.5 * Dy
        vx, vy = -vx, -vy
    else:
        vx, vy = m["gx"], m["gy"]
    mag = np.hypot(vx, vy)
    safe = np.where(mag > 1e-6, mag, 1.0)
    nxv = np.where(mag > 1e-6, vx / safe, 0.0)
    nyv = np.where(mag > 1e-6, vy / safe, 0.0)
    fo = np.empty_like(f)
    go = np.empty_like(g)
    usq = ux ** 2 + uy ** 2
    for i in range(9):
        cu = CX[i] * ux + CY[i] * uy
        fe = W[i] * phi * (1 + 3 * cu)
        Fi = (1 - 0.5 / tau_f) * W[i] * 3 * (CX[i] * (Dx + lam * nxv / 3) + CY[i] * (Dy + lam * nyv / 3))
        ge = 3 * m["p"] * W[i] + rho * W[i] * (3 * cu + 4.5 * cu ** 2 - 1.5 * usq)
        if i == 0:
            ge = ge - 3 * m["p"]
        cF = CX[i] * m["Fx"] + CY[i] * m["Fy"]
        cg = CX[i] * m["gx"] + CY[i] * m["gy"]
        Gi = (1 - 0.5 / tau_g) * W[i] * (3 * cF + 3 * drho * cu * cg)
        fo[i] = f[i] - (f[i] - fe) / tau_f + Fi
        go[i] = g[i] - (g[i] - ge) / tau_g + Gi
    fn = np.empty_like(f)
    gn = np.empty_like(g)
    for i in range(9):
        fn[i] = np.roll(fo[i], shift=(CY[i], CX[i]), axis=(0, 1))
        gn[i] = np.roll(go[i], shift=(CY[i], CX[i]), axis=(0, 1))
    if walls:
        for i in range(9):
            if CY[i] == 1 and p["bc_y"] == 1:   # leaves through the top wall from the last row
                fn[OPP[i], -1, :] = fo[i, -1, :]
                gn[OPP[i], -1, :] = go[i, -1, :]
            if CY[i] == -1:  # leaves through the bottom wall from row 0
                fn[OPP[i], 0, :] = fo[i, 0, :]
                gn[OPP[i], 0, :] = go[i, 0, :]
    if p["bc_y"] == 2:
        _open_top(fn, gn)
    return fn, gn, np.stack([phi * ux, phi * uy])
