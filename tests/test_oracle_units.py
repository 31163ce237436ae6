"""Pins of the oracle's per-node terms against what the paper fixes exactly:
the D2Q9 lattice (Eq. 10), the moment identities of the equilibria and forcing
(Eqs. 9, 11, Appendix Eqs. A1-A2), the equivalence of the two forms of G_i
(Eqs. 18 and 20), the finite-difference stencils (Eqs. 27-28) on functions with
closed-form discrete derivatives, and the interface invariant of Eqs. 3, 6, 7."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0


def _golden_lattice():
    rows = np.loadtxt(os.path.join(GOLDEN, "d2q9_eq10.txt"))
    return rows[:, 1].astype(int), rows[:, 2].astype(int), rows[:, 3] / rows[:, 4]


def test_lattice_matches_eq10():
    cx, cy, w, opp = oracle.lattice_constants()
    gcx, gcy, gw = _golden_lattice()
    assert np.array_equal(cx, gcx) and np.array_equal(cy, gcy)
    assert np.allclose(w, gw, rtol=0, atol=1e-16)
    # the trigonometric definition of Eq. 10 itself
    for i in range(1, 5):
        a = (i - 1) * np.pi / 2
        assert (cx[i], cy[i]) == (round(np.cos(a)), round(np.sin(a)))
    for i in range(5, 9):
        a = (i - 5) * np.pi / 2 + np.pi / 4
        assert (cx[i], cy[i]) == (round(np.sqrt(2) * np.cos(a)), round(np.sqrt(2) * np.sin(a)))
    for i in range(9):
        assert cx[opp[i]] == -cx[i] and cy[opp[i]] == -cy[i]


def test_lattice_isotropy():
    cx, cy, w, _ = oracle.lattice_constants()
    c = np.stack([cx, cy], 1).astype(float)
    d = np.eye(2)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * d, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    four = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    delta4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
              + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(four, CS2 ** 2 * delta4, atol=1e-16)


def _c():
    cx, cy, _, _ = oracle.lattice_constants()
    return np.stack([cx, cy], 1).astype(float)


@pytest.mark.parametrize("seed", range(5))
def test_feq_moments(seed):
    r = np.random.default_rng(seed)
    phi, ux, uy = r.uniform(0, 1), r.uniform(-0.1, 0.1), r.uniform(-0.1, 0.1)
    f = oracle.feq(phi, ux, uy)
    c = _c()
    assert abs(f.sum() - phi) < 1e-15
    assert np.allclose(c.T @ f, [phi * ux, phi * uy], atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", f, c, c), phi * CS2 * np.eye(2), atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_geq_moments_A1(seed):
    r = np.random.default_rng(100 + seed)
    p, rho = r.uniform(-1e-3, 1e-3), r.uniform(1e-3, 1)
    u = r.uniform(-0.1, 0.1, 2)
    g = oracle.geq(p, rho, *u)
    c = _c()
    d = np.eye(2)
    assert abs(g.sum()) < 1e-16
    assert np.allclose(c.T @ g, rho * u, atol=1e-17)
    assert np.allclose(np.einsum("i,ia,ib->ab", g, c, c), rho * np.outer(u, u) + p * d, atol=1e-17)
    third = np.einsum("i,ia,ib,ic->abc", g, c, c, c)
    delta4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
              + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(third, rho * CS2 * np.einsum("abcd,d->abc", delta4, u), atol=1e-17)


@pytest.mark.parametrize("seed", range(5))
def test_source_f_moments(seed):
    r = np.random.default_rng(200 + seed)
    tau = r.uniform(0.55, 2)
    lam = r.uniform(0, 1)
    th = r.uniform(0, 2 * np.pi)
    n = np.array([np.cos(th), np.sin(th)])
    D = r.uniform(-1e-3, 1e-3, 2)
    F = oracle.source_f(tau, lam, n[0], n[1], D[0], D[1])
    c = _c()
    assert abs(F.sum()) < 1e-17
    assert np.allclose(c.T @ F, (1 - 0.5 / tau) * (D + CS2 * lam * n), atol=1e-17)


@pytest.mark.parametrize("seed", range(5))
def test_force_g_moments_A2_and_eq18(seed):
    r = np.random.default_rng(300 + seed)
    tau = r.uniform(0.51, 5)
    drho = r.uniform(0.5, 1)
    u = r.uniform(-0.05, 0.05, 2)
    gphi = r.uniform(-0.3, 0.3, 2)
    Fv = r.uniform(-1e-4, 1e-4, 2)
    G = oracle.force_g(tau, drho, u[0], u[1], gphi[0], gphi[1], Fv[0], Fv[1])
    c = _c()
    _, _, w, _ = oracle.lattice_constants()
    k = 1 - 0.5 / tau
    grho = drho * gphi
    # Appendix Eq. A2
    assert abs(G.sum() - k * u @ grho) < 1e-16
    assert np.allclose(c.T @ G, k * Fv, atol=1e-17)
    Lam = k * CS2 * (np.outer(u, grho) + np.outer(grho, u) + (u @ grho) * np.eye(2))
    assert np.allclose(np.einsum("i,ia,ib->ab", G, c, c), Lam, atol=1e-16)
    # Eq. 18 (general form with grad rho) equals Eq. 20
    G18 = np.array([k * w[i] * (u @ grho + c[i] @ Fv / CS2
                                + (u @ (np.outer(c[i], c[i]) - CS2 * np.eye(2)) @ grho) / CS2)
                    for i in range(9)])
    assert np.allclose(G, G18, rtol=0, atol=1e-17)


def test_viscosity_modes_end_points():
    P = oracle.make_params(rho_l=1.0, rho_g=0.01, nu_l=0.05, nu_g=0.4)
    for mode in (0, 1):
        P.visc_mode = mode
        assert abs(oracle.viscosity(P, 1.0) - 0.05) < 1e-15
        assert abs(oracle.viscosity(P, 0.0) - 0.4) < 1e-15
    P.visc_mode = 0
    assert abs(oracle.viscosity(P, 0.5) - 0.225) < 1e-15      # arithmetic mean (Eq. 24)
    P.visc_mode = 1
    assert abs(1 / oracle.viscosity(P, 0.5) - 0.5 * (20 + 2.5)) < 1e-12  # harmonic (Eq. 25)
    P.visc_mode = 2
    rho = lambda ph: ph * 0.99 + 0.01
    assert abs(oracle.viscosity(P, 0.5) - 0.05 / rho(0.5)) < 1e-15     # mu_l at phi >= 0.5 (Eq. 26)
    assert abs(oracle.viscosity(P, 0.49) - 0.004 / rho(0.49)) < 1e-15  # mu_g below
    assert abs(oracle.viscosity(P, 1.0) - 0.05) < 1e-15
    assert abs(oracle.viscosity(P, 0.0) - 0.4) < 1e-15


def test_stencils_exact_on_quadratics():
    ny, nx = 12, 14
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    a, b, cc, d, e = 0.3, -0.7, 0.45, 1.1, -0.2
    phi = a * x * x + b * x * y + cc * y * y + d * x + e * y
    gx, gy, lap = oracle.grad_lap(phi, bc_y=1)
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    assert np.allclose(gx[inner], (2 * a * x + b * y + d)[inner], atol=1e-12)
    assert np.allclose(gy[inner], (b * x + 2 * cc * y + e)[inner], atol=1e-12)
    assert np.allclose(lap[inner], 2 * a + 2 * cc, atol=1e-12)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_stencils_closed_form_on_periodic_waves(axis):
    n = 32
    k = 2 * np.pi * 3 / n
    idx = np.arange(n, dtype=float)
    if axis == "x":
        phi = np.tile(np.cos(k * idx), (n, 1))
    else:
        phi = np.tile(np.cos(k * idx)[:, None], (1, n))
    gx, gy, lap = oracle.grad_lap(phi, bc_y=0)
    # central isotropic gradient of cos(k s): -sin(k s) sin(k); Laplacian: 2 cos(k s)(cos k - 1)
    g_exact = -np.sin(k * idx) * np.sin(k)
    g_exact = np.tile(g_exact, (n, 1)) if axis == "x" else np.tile(g_exact[:, None], (1, n))
    along, across = (gx, gy) if axis == "x" else (gy, gx)
    assert np.allclose(along, g_exact, atol=1e-14)
    assert np.allclose(across, 0, atol=1e-14)
    assert np.allclose(lap, 2 * phi * (np.cos(k) - 1), atol=1e-14)


def test_planar_profile_invariant_eqs_3_6_7():
    """For phi = 1/2 + 1/2 tanh(2 s / W), Eq. 7's k and beta make the chemical
    potential of Eq. 6 vanish and |grad phi| equal lambda of Eq. 3 in the
    continuum; the lattice values approach that as W grows."""
    sigma = 0.01
    mu_err, grad_err = [], []
    for W in (4.0, 8.0, 16.0):
        ny, nx = int(12 * W), 4
        s = np.arange(ny)[:, None] - ny / 2 + 0.5
        phi = np.broadcast_to(0.5 + 0.5 * np.tanh(2 * s / W), (ny, nx)).copy()
        lat = oracle.Lattice(nx, ny, rho_l=1, rho_g=1, sigma=sigma, W=W, bc_y=1)
        lat.init(phi)
        mu = lat.fields()["mu"]
        bulk = 4 * (12 * sigma / W) * np.abs(phi * (phi - 1) * (phi - 0.5)).max()
        mu_err.append(np.abs(mu).max() / bulk)
        gx, gy, _ = oracle.grad_lap(phi, bc_y=1)
        lam = 4 * phi * (1 - phi) / W
        inner = slice(2, ny - 2)
        grad_err.append(np.abs(np.abs(gy[inner]) - lam[inner]).max() / lam.max())
        assert np.abs(gx).max() < 1e-15
    # the two terms of Eq. 6 cancel to within the stencils' truncation error,
    # which falls at second order (x4 per doubling of W, >2.8 asymptotically here)
    for e in (mu_err, grad_err):
        assert e[0] < 0.1
        assert e[0] / e[1] > 2.8 and e[1] / e[2] > 2.8
