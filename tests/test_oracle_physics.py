"""Pins of the oracle's whole time step against results the paper or the
mathematics fixes: fixed points, closed-form transients, conservation, the
Laplace law, the layered-Poiseuille solution (Eq. 31, Table 1), checkpoint
resume, and brute force against an independent NumPy transcription.

Each test names the mistake it would catch."""
import os

import numpy as np
import pytest

import oracle
from paper_1710_09541_gb300 import cases
from tests import brute_numpy as bn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lattice(nx, ny, **kw):
    return oracle.Lattice(nx, ny, **kw)


def test_uniform_state_is_a_fixed_point():
    """Uniform phi, u, p with no gradients is stationary; u and p read back
    exactly (catches a dropped rho*s_0 in Eq. 22b or a wrong g_0^eq)."""
    nx, ny = 9, 7
    phi = np.full((ny, nx), 0.3)
    ux, uy, p = np.full_like(phi, 0.01), np.full_like(phi, -0.02), np.full_like(phi, 1e-3)
    lat = _lattice(nx, ny, sigma=0.01).init(phi, ux, uy, p)
    lat.step(50)
    F = lat.fields()
    assert np.allclose(F["phi"], 0.3, rtol=1e-14, atol=0)
    assert np.allclose(F["ux"], 0.01, rtol=1e-12, atol=0)
    assert np.allclose(F["uy"], -0.02, rtol=1e-12, atol=0)
    assert np.allclose(F["p"], 1e-3, rtol=1e-11, atol=0)


def test_uniform_body_force_closed_form():
    """Uniform fluid under a constant body force G (Eq. 4b): the half-force
    velocity of Eq. 22a and the first moment of G_i (Eq. A2) give
    rho u(t) = G (t + 1/2) exactly (catches a missing F/2 or a wrong force
    moment)."""
    nx, ny = 6, 5
    G = np.array([1e-6, -2e-6])
    lat = _lattice(nx, ny, rho_l=1.0, rho_g=1.0, Gx=G[0], Gy=G[1]).init(np.ones((ny, nx)))
    for t in range(0, 60, 7):
        F = lat.fields()
        assert np.allclose(F["rho"] * F["ux"], G[0] * (t + 0.5), rtol=1e-10, atol=0)
        assert np.allclose(F["rho"] * F["uy"], G[1] * (t + 0.5), rtol=1e-10, atol=0)
        lat.step(7)


def _shear_wave_rate(mode, phi_val):
    nx, ny = 4, 64
    # sigma = 0 removes the chemical potential; a very wide W makes lambda of
    # Eq. 3 vanish, so the uniform mixed phi is not driven apart by Eq. 1's
    # sharpening flux and the flow sees one constant viscosity
    P = dict(rho_l=1.0, rho_g=0.05, nu_l=0.08, nu_g=0.2, visc_mode=mode, sigma=0.0, W=1e12)
    k = 2 * np.pi / ny
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    u0 = 1e-4 * np.sin(k * y)
    lat = _lattice(nx, ny, **P).init(np.full((ny, nx), phi_val), u0)
    lat.step(100)
    a1 = (lat.fields()["ux"][:, 0] * np.sin(k * np.arange(ny))).sum()
    lat.step(400)
    F = lat.fields()
    assert np.abs(F["phi"] - phi_val).max() < 1e-8  # O(u^2) with u = 1e-4
    a2 = (F["ux"][:, 0] * np.sin(k * np.arange(ny))).sum()
    rate = np.log(a1 / a2) / 400
    return rate, k, oracle.viscosity(oracle.make_params(**P), phi_val)


@pytest.mark.parametrize("mode,phi_val", [(0, 0.3), (1, 0.3), (2, 0.3), (2, 0.7)])
def test_shear_wave_decay_matches_viscosity(mode, phi_val):
    """A shear wave decays as exp(-nu k_d^2 t) with k_d^2 = 2(1 - cos k), the
    lattice Laplacian's eigenvalue; nu = c_s^2 (tau_g - 1/2) (Eq. 23) with nu
    from Eq. 24, 25 or 26 (catches a wrong tau_g or viscosity rule)."""
    rate, k, nu = _shear_wave_rate(mode, phi_val)
    assert abs(rate / (nu * 2 * (1 - np.cos(k))) - 1) < 0.01


def test_drop_translates_with_uniform_flow():
    """Without surface tension and with equal densities, u stays uniform and
    the conservative Allen-Cahn equation (Eq. 1) carries the drop's centroid at
    exactly u (catches a reversed streaming direction, a wrong sign in Eq. 9 or
    a transposed axis)."""
    nx = ny = 48
    U = np.array([0.02, 0.01])
    phi0 = cases.drop(nx, ny, 8, 4.0, x0=16.0, y0=16.0)
    lat = _lattice(nx, ny, rho_l=1.0, rho_g=1.0, sigma=0.0, W=4.0).init(
        phi0, np.full_like(phi0, U[0]), np.full_like(phi0, U[1]))
    T = 400
    lat.step(T)
    phi = lat.fields()["phi"]
    y, x = np.mgrid[0:ny, 0:nx]
    c0 = np.array([(x * phi0).sum(), (y * phi0).sum()]) / phi0.sum()
    c1 = np.array([(x * phi).sum(), (y * phi).sum()]) / phi.sum()
    assert np.allclose(c1 - c0, U * T, atol=0.05)
    # the drop keeps its shape: the interface stays sharp (Eqs. 1-3)
    assert phi.max() > 0.99 and phi.min() > -0.01


@pytest.mark.parametrize("bc_y", [0, 1])
def test_phi_is_conserved(bc_y):
    """Collision conserves sum f_i (sum F_i = 0), streaming and half-way
    bounce-back permute: sum phi is constant to round-off (catches a lost or
    duplicated population at a wall)."""
    nx, ny = 40, 36
    phi0 = cases.drop(nx, ny, 10, 4.0, x0=20.0, y0=11.0, walls_y=bool(bc_y))
    u0 = 1e-3 * np.sin(np.arange(nx) / 5.0)[None, :] * np.ones((ny, 1))
    lat = _lattice(nx, ny, rho_g=0.01, bc_y=bc_y, Gx=1e-6, Gy=-1e-6).init(phi0, u0, -u0)
    s0 = lat.sum_phi()
    lat.step(2000)
    assert abs(lat.sum_phi() - s0) / s0 < 1e-12


@pytest.mark.parametrize("normal_scheme", [0, 1])
def test_laplace_law_resolved_interface(normal_scheme):
    """Static drops of R = 14, 20, 26 in a 96 x 96 periodic box (ratio 1000,
    sigma = 0.01) with a resolved interface, W = 8: the pressure jump,
    averaged over the inner half of the drop against the far gas and over
    the decaying acoustic oscillation, is sigma/R within 3% for each R, and
    the fit of the jump against 1/R has slope sigma within 3% (Laplace law;
    catches wrong k, beta of Eq. 7 or a wrong sign in Eq. 6).

    W = 8 because the jump converges to sigma/R as the interface is resolved:
    at R = 16 the ratio is 0.93, 0.98, 1.00 for W = 4, 6, 8.  The inner-half
    average, not the centre node, because with the central normal (Eq. 2 with
    Eq. 27) phi dips at the centre of larger drops (to 0.86 at R = 24, W = 4),
    where the normal of a maximum points outward on every side, and the
    pressure spikes there."""
    n = 96
    yy, xx = np.mgrid[0:n, 0:n]
    r = np.hypot(xx - n / 2, yy - n / 2)
    jumps = []
    for R in (14, 20, 26):
        P = dict(cases.params_static_drop(), W=8.0, normal_scheme=normal_scheme)
        lat = _lattice(n, n, **P).init(cases.drop(n, n, R, 8.0))
        lat.step(8000)
        acc = []
        for _ in range(16):
            lat.step(125)
            F = lat.fields()
            acc.append(F["p"][r < R / 2].mean() - F["p"][r > R + 12].mean())
        jumps.append(np.mean(acc))
        assert abs(jumps[-1] * R / 0.01 - 1) < 0.03, (R, jumps[-1] * R / 0.01)
    slope, _ = np.polyfit(1 / np.array([14.0, 20.0, 26.0]), jumps, 1)
    assert abs(slope / 0.01 - 1) < 0.03


def interface_height(col):
    """Height of the phi = 1/2 crossing in a column with liquid below, by
    linear interpolation between node centres y_j = j + 1/2."""
    j = int(np.nonzero((col[:-1] >= 0.5) & (col[1:] < 0.5))[0][0])
    return j + 0.5 + (col[j] - 0.5) / (col[j] - col[j + 1])


@pytest.mark.parametrize("ny,ratio", [(64, 1000.0), (63, 1000.0), (64, 10.0)])
def test_planar_interface_at_rest_stays_put(ny, ratio):
    """A flat layer between walls (the Eq. 33 geometry without the body
    force) has zero curvature, so nothing drives it.  Over 1e4 steps:
    - the phi = 1/2 crossing moves by less than 1e-4 node (measured at most
      1.5e-5; the interface sits on a node for odd ny, between nodes for even);
    - the pressure jump across it stays below 1e-7, the Laplace law at
      R -> inf (sigma / W = 2.5e-4; measured 4e-8);
    - phi stays within 1e-2 of Eq. 33's tanh (the W = 4 lattice profile of
      Eqs. 3, 6 and 7 differs from it by 6e-3);
    - the spurious speed stays below 5e-6 (measured 1.5e-6 at ratio 10, the
      slowest to settle).
    Catches a wrong lambda (Eq. 3) or sharpening direction (the profile
    widens or moves), a wrong k, beta or sign in Eqs. 6-7 (a chemical-
    potential force on the flat layer: a jump of 2e-7 to 1e-6 and flow), and
    a wrong sign of the interface term of Eq. 22b (flow)."""
    P = cases.params_poiseuille(ny, ratio=ratio, Gx=0.0, W=4.0)
    phi0 = cases.layer(4, ny, 4.0)
    lat = _lattice(4, ny, **P).init(phi0)
    h0 = interface_height(lat.fields()["phi"][:, 0])
    lat.step(10000)
    F = lat.fields()
    assert abs(interface_height(F["phi"][:, 0]) - h0) < 1e-4
    p = F["p"][:, 0]
    assert abs(p[4:12].mean() - p[-12:-4].mean()) < 1e-7
    assert np.abs(F["phi"] - phi0).max() < 1e-2
    assert np.hypot(F["ux"], F["uy"]).max() < 5e-6


def _poiseuille(ny, nx, params, steps, u_start):
    lat = _lattice(nx, ny, **params).init(cases.layer(nx, ny, params["W"]),
                                          np.broadcast_to(u_start[:, None], (ny, nx)))
    lat.step(steps)
    return lat.fields()["ux"][:, nx // 2]


def _two_layer_profile(ny, P):
    """Eq. 31 at node centres y_j = j + 1/2 - ny/2, h = ny/2, liquid below."""
    h = ny / 2.0
    s = (np.arange(ny) + 0.5 - h) / h
    mu_l, mu_g, G = P["rho_l"] * P["nu_l"], P["rho_g"] * P["nu_g"], P["Gx"]
    a = (mu_g - mu_l) / (mu_g + mu_l)
    up = G * h * h / (2 * mu_g) * (-s ** 2 - s * a + 2 * mu_g / (mu_g + mu_l))
    lo = G * h * h / (2 * mu_l) * (-s ** 2 - s * a + 2 * mu_l / (mu_g + mu_l))
    return np.where(s > 0, up, lo)


def test_single_phase_poiseuille():
    """Equal phases between half-way bounce-back walls: the steady profile is
    the parabola G y (H - y) / (2 mu) (catches a wrong wall rule or viscosity)."""
    ny, nx = 32, 4
    P = dict(rho_l=1.0, rho_g=1.0, nu_l=0.1, nu_g=0.1, sigma=0.0, W=4.0, Gx=1e-6, bc_y=1)
    y = np.arange(ny) + 0.5
    exact = 1e-6 * y * (ny - y) / (2 * 0.1)
    u = _poiseuille(ny, nx, P, 20000, np.zeros(ny))
    # measured 7.0e-4 (L2): the half-way wall's O(1/ny^2) placement error
    assert np.sqrt(((u - exact) ** 2).sum() / (exact ** 2).sum()) < 1e-3


def test_open_top_half_poiseuille_first_order():
    """Bottom wall and open top (bc_y = 2, the impact case's boundaries):
    under a body force a single-phase layer tends to the lower half of a
    channel of height 2 ny, u = G (2 H s - s^2) / (2 mu) with s = y + 1/2 and
    H = ny, because the zero-gradient copy makes the top a symmetry line.
    The copy is a first-order closure, so the L2 error halves as ny doubles
    (measured 2.0% and 1.0% at ny = 16 and 32; a closed top is 79% off).
    Catches copying the wrong directions or rows, or bouncing back at the top."""
    errs = []
    for ny in (16, 32):
        P = dict(rho_l=1.0, rho_g=1.0, nu_l=0.1, nu_g=0.1, sigma=0.0, W=4.0, Gx=1e-6, bc_y=2)
        lat = _lattice(4, ny, **P).init(np.ones((ny, 4)))
        lat.step(int(4 * ny * ny / 0.1))
        u = lat.fields()["ux"][:, 0]
        s = np.arange(ny) + 0.5
        exact = 1e-6 * (2 * ny * s - s * s) / (2 * 0.1)
        errs.append(np.sqrt(((u - exact) ** 2).sum() / (exact ** 2).sum()))
        assert abs(u[-1] / exact[-1] - 1) < 0.04      # no slip or reflection at the top
    assert errs[0] < 0.025 and errs[1] < 0.0125
    assert 1.8 < errs[0] / errs[1] < 2.2


def test_open_top_needs_two_rows_and_known_bc():
    for bc, ny in ((2, 1), (3, 8), (-1, 8)):
        with pytest.raises(Exception):
            _lattice(4, ny, bc_y=bc)


def test_layered_poiseuille_table1_ratio10():
    """Layered Poiseuille flow at the paper's setup (100 x 10 -> 100 x 4, the
    flow is x-uniform), density ratio 10, step viscosity (Eq. 26).  Table 1
    prints E_u = 8.9e-3; this oracle (central-gradient normal, node centres
    half a cell from the walls) reaches 1.5e-2.  The bound 2.5x the printed
    value still fails for a missing Lambda term of Eq. 20 (E_u ~ 2), a wrong
    interface side or a wrong viscosity rule."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_poiseuille_Eu.txt"))
    ratio, nu_ratio, Eu_paper = rows[0]
    ny, nx = 100, 4
    rho_l, nu_l, uc, h = 1.0, 0.1, 1e-4, 50.0
    rho_g = rho_l / ratio
    nu_g = nu_ratio * nu_l
    G = uc * (rho_l * nu_l + rho_g * nu_g) / h ** 2
    P = dict(rho_l=rho_l, rho_g=rho_g, nu_l=nu_l, nu_g=nu_g, visc_mode=2, sigma=1e-3, W=5.0,
             tau_h=0.8, Gx=G, bc_y=1)
    ua = _two_layer_profile(ny, P)
    u = _poiseuille(ny, nx, P, 60000, ua)
    Eu = np.abs(u - ua).sum() / np.abs(ua).sum()   # Eq. 32
    assert Eu < 2.5 * Eu_paper
    assert u[:ny // 2].max() < u[ny // 2:].max()   # the gas layer (upper) moves faster


def _layered_Eu(ratio, nu_ratio, ny, W, steps, visc_mode=2):
    """E_u (Eq. 32) of the layered Poiseuille flow of Sec. III B on a 4 x ny
    channel, started from Eq. 31 itself."""
    rho_l, nu_l, uc, h = 1.0, 0.1, 1e-4, ny / 2
    P = dict(rho_l=rho_l, rho_g=rho_l / ratio, nu_l=nu_l, nu_g=nu_ratio * nu_l, visc_mode=visc_mode,
             sigma=1e-3, W=W, tau_h=0.8, bc_y=1)
    P["Gx"] = uc * (rho_l * nu_l + P["rho_g"] * P["nu_g"]) / h ** 2
    ua = _two_layer_profile(ny, P)
    u = _poiseuille(ny, 4, P, steps, ua)
    return np.abs(u - ua).sum() / np.abs(ua).sum()


def test_layered_poiseuille_linear_viscosity_matches_table1_comparison_column():
    """Table 1's setup with the viscosity interpolated linearly (Eq. 24; with
    nu_g = nu_l this is a uniform nu, so mu follows rho): E_u reproduces the
    paper's column for the model of Fakhari et al. within 5% at density
    ratios 100 and 1000 (measured 2.71e-1 and 3.84e-1 against 2.7e-1 and
    3.9e-1).  At this setup E_u is set by the smooth viscosity across the
    interface rather than by the LB scheme, so the printed numbers pin the
    setup the two models share: the grid, W, the node placement and the
    interface position against the half-way walls (the placement as printed,
    phi0 and Eq. 31 at y = j, gives 2.93e-1 at ratio 100, 8.5% off).  E_u
    does not depend on G_x: the steady profile and Eq. 31 both scale with it."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_poiseuille_Eu_comparison.txt"))
    for ratio, nu_ratio, Eu_paper in rows[[1, 3]]:
        Eu = _layered_Eu(ratio, nu_ratio, 100, 5.0, 60000, visc_mode=0)
        assert abs(Eu / Eu_paper - 1) < 0.05, (ratio, Eu, Eu_paper)


@pytest.mark.parametrize("ratio,nu_ratio", [(100.0, 1.0), (1000.0, 10.0)])
def test_layered_poiseuille_converges_at_second_order(ratio, nu_ratio):
    """Table 1's setup (ny = 100, W = 5, step viscosity of Eq. 26) and the
    same flow on a grid twice as fine (ny = 200, W = 10, four times the
    steps): E_u against Eq. 31 falls by a factor 4 (measured 4.06 and 3.95;
    also 3.95 at ratio 10).  The scheme converges to the two-layer solution
    at second order, so the gap to the paper's E_u is a discretisation
    constant, not a wrong term (a dropped Lambda term of Eq. 20 leaves E_u
    near 2 on both grids)."""
    coarse = _layered_Eu(ratio, nu_ratio, 100, 5.0, 60000)
    fine = _layered_Eu(ratio, nu_ratio, 200, 10.0, 240000)
    assert 3.5 < coarse / fine < 4.5, (coarse, fine)
    assert fine < 3e-2


@pytest.mark.parametrize("bc_y,normal_scheme", [(0, 0), (1, 0), (2, 0), (0, 1), (1, 1)])
def test_brute_force_numpy_transcription(bc_y, normal_scheme):
    """8 x 8 grids, 10 steps, against the independent whole-array NumPy
    transcription, with the central (Eq. 2 with Eq. 27) or the local (Eq. 29)
    normal (catches index and sign slips in either)."""
    nx = ny = 8
    r = np.random.default_rng(7 + bc_y + 3 * normal_scheme)
    phi0 = cases.drop(nx, ny, 2.5, 3.0, x0=3.7, y0=4.2, walls_y=bool(bc_y)) + 0.01 * r.random((ny, nx))
    ux0 = 0.01 * r.standard_normal((ny, nx))
    uy0 = 0.01 * r.standard_normal((ny, nx))
    p0 = 1e-4 * r.standard_normal((ny, nx))
    P = dict(rho_l=1.0, rho_g=0.01, nu_l=0.05, nu_g=0.2, visc_mode={0: 0, 1: 2, 2: 1}[bc_y],
             sigma=0.02, W=3.0, tau_h=0.9, Gx=1e-5, Gy=-2e-5, bc_y=bc_y, normal_scheme=normal_scheme)
    lat = _lattice(nx, ny, **P).init(phi0, ux0, uy0, p0)
    f, g, phiu = bn.init(phi0, ux0, uy0, p0, P)
    of, og, ophiu = lat.get_state()
    assert np.allclose(of, f, atol=1e-16) and np.allclose(og, g, atol=1e-17)
    for _ in range(10):
        f, g, phiu = bn.step(f, g, phiu, P)
    lat.step(10)
    of, og, ophiu = lat.get_state()
    assert np.abs(of - f).max() < 1e-13
    assert np.abs(og - g).max() < 1e-15
    assert np.abs(ophiu - phiu).max() < 1e-15
    m = bn.moments(f, g, P, bc_y in (1, 2))
    F = lat.fields()
    for k in ("phi", "ux", "uy", "p", "mu"):
        assert np.abs(F[k] - m[k]).max() <= 1e-12 * max(1.0, np.abs(m[k]).max()), k


def test_checkpoint_resume_is_exact():
    nx, ny = 20, 16
    P = cases.params_static_drop()
    phi0 = cases.drop(nx, ny, 5, 4.0)
    a = _lattice(nx, ny, **P).init(phi0)
    a.step(30)
    b = _lattice(nx, ny, **P).init(phi0)
    b.step(12)
    c = _lattice(nx, ny, **P).set_state(*b.get_state())
    c.step(18)
    for x, y in zip(a.get_state(), c.get_state()):
        assert np.array_equal(x, y)
