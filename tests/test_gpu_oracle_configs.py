"""The CUDA path against the FP64 oracle on the workload configurations, over
the horizons each is quoted on (Sec. III A, C, D setups), and the batched
kernel against the oracle.

Where the flow amplifies perturbations (an extremum of phi with lambda != 0,
Eq. 3, turns the normal of Eq. 2 by eps / |grad phi|, and the cut-off of n
switches branch under perturbations of 1e-7), a pointwise bound is measured
against the oracle's own spread: the same FP64 oracle started from phi0
rounded to FP32, or from phi0 plus 1e-7 noise, moves by as much.  The FP32
run on the GPU is one more perturbed member of that family, so it is held to
a stated multiple of the spread.

Field error = max |gpu - oracle| / max(max |oracle|, s_ref); s_ref = 1 for
phi, rho_l for rho, sigma/mu_l for u, sigma/R (drop) or sigma/W for p."""
import numpy as np
import pytest

import oracle
from paper_1710_09541_gb300 import cases
from tests.test_gpu_parity import (TOL, TOL_P, _assert_fields, _field_errors, _one_step_check,
                                   _one_step_setup, _scales, _spreading_radius)

pytestmark = pytest.mark.gpu

# a GPU run may part from the exact-input oracle by this multiple of the
# largest deviation of the perturbed oracle runs (same field, same time)
SPREAD_FACTOR = 2.0


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09541_gb300 import build as lbm_build
    from paper_1710_09541_gb300 import lbm as _lbm

    lbm_build.build()
    _lbm.load()
    return _lbm


def _round32(a):
    return None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)


def _fmt(d):
    return {k: f"{v:.2e}" for k, v in d.items()}


# ------------------------------------------------------------ config 1 ----

def test_static_drop_64_after_100_steps(lbm):
    """Static droplet, 64 x 64 periodic, R = 16, W = 4, ratio 1000,
    sigma = 0.01, tau = 0.8 (Sec. III A setup): fields after 100 FP32 steps
    against the oracle started from phi0 rounded to FP32.  The bound is 1e-5
    (3e-5 for p) or twice the oracle's own change under that rounding
    (rounded-input oracle against exact-input oracle), whichever is larger."""
    nx = ny = 64
    P = cases.params_static_drop()
    phi0 = cases.drop(nx, ny, 16, 4.0)
    sc = _scales(P, R=16)
    exact = oracle.Lattice(nx, ny, **P).init(phi0).step(100).fields()
    rounded = oracle.Lattice(nx, ny, **P).init(_round32(phi0)).step(100).fields()
    gap = _field_errors(rounded, exact, sc)
    with lbm.Lattice(nx, ny, **P) as g:
        got = g.init(phi0).step(100).fields()
    err = _field_errors(got, rounded, sc)
    print("config 1, 100 steps: gpu vs rounded-input oracle", _fmt(err),
          "| oracle rounded vs exact", _fmt(gap))
    for k, v in err.items():
        tol = TOL_P if k == "p" else TOL
        assert np.isfinite(v) and v <= max(tol, SPREAD_FACTOR * gap[k]), (k, err, gap)


# ------------------------------------------------------------ config 3 ----

def _spread_members(phi0):
    """Inputs of the perturbed oracle runs: phi0 rounded to FP32, and phi0
    plus normal noise of 1e-7 (two seeds)."""
    out = [_round32(phi0)]
    for seed in (1, 2):
        out.append(phi0 + 1e-7 * np.random.default_rng(seed).standard_normal(phi0.shape))
    return out


@pytest.mark.parametrize("ratio", [3.0, 1000.0])
def test_spinodal_1024_pointwise_first_200_steps(lbm, ratio):
    """Spinodal decomposition at full size (1024 x 1024 periodic, phi0 =
    0.5 +- 0.01 from seed 12345, sigma = 1e-3, W = 4), density ratios 3 and
    1000: every node at steps 50, 100 and 200, against the exact-input oracle,
    within SPREAD_FACTOR times the largest deviation of three perturbed oracle
    runs (rounded to FP32, and two 1e-7 noise draws)."""
    n = 1024
    P = cases.params_spinodal(ratio=ratio)
    phi0 = cases.spinodal(n, n, 0.5, 0.01, seed=12345)
    sc = _scales(P)
    times = (50, 100, 200)
    exact = oracle.Lattice(n, n, **P).init(phi0)
    members = [oracle.Lattice(n, n, **P).init(p) for p in _spread_members(phi0)]
    with lbm.Lattice(n, n, **P) as g:
        g.init(phi0)
        done = 0
        for T in times:
            exact.step(T - done)
            g.step(T - done)
            for m in members:
                m.step(T - done)
            done = T
            ref = exact.fields()
            got = g.fields()
            spread = {k: 0.0 for k in sc}
            for m in members:
                for k, v in _field_errors(m.fields(), ref, sc).items():
                    spread[k] = max(spread[k], v)
            err = _field_errors(got, ref, sc)
            corr = np.corrcoef((got["phi"] - 0.5).ravel(), (ref["phi"] - 0.5).ravel())[0, 1]
            print(f"spinodal ratio {ratio:g}, step {T}: gpu vs oracle", _fmt(err),
                  "| oracle spread", _fmt(spread), f"| corr {corr:.6f}")
            for k, v in err.items():
                assert np.isfinite(v) and v <= SPREAD_FACTOR * spread[k], (T, k, err, spread)
            assert corr > 0.999


# ------------------------------------------------------------ config 4 ----

def _radius_interp(phi, film, W):
    """Spreading radius with the ends at the phi = 1/2 crossings (linear
    interpolation between the run's end nodes and their gas neighbours)."""
    row = phi[int(round(film + W)), :]
    c = phi.shape[1] // 2
    if not row[c] >= 0.5:
        return 0.0
    l = c
    while l > 0 and row[l - 1] >= 0.5:
        l -= 1
    r = c
    while r < len(row) - 1 and row[r + 1] >= 0.5:
        r += 1
    L = l - 0.5 if l == 0 else (l - 1) + (0.5 - row[l - 1]) / (row[l] - row[l - 1])
    R = r + 0.5 if r == len(row) - 1 else r + (row[r] - 0.5) / (row[r] - row[r + 1])
    return 0.5 * (R - L)


def test_impact_2400x600_pointwise_first_quarter(lbm):
    """Droplet impact at full size (the setup below): every node after 200 and
    1250 steps (t* = 0.25, the horizon over which pointwise agreement is
    expected for this flow), against the exact-input oracle, within
    SPREAD_FACTOR times the largest deviation of three perturbed oracle runs.
    From the first contact of drop and film the flow amplifies round-off:
    rounding the inputs to FP32 moves the FP64 oracle by 1e-2 in phi after
    200 steps and 8e-2 after 1250, where the film meets the drop."""
    nx, ny, D, film, U = 2400, 600, 200.0, 20.0, 0.04
    P = cases.params_impact(Re=100.0)
    phi0, u0, v0 = cases.impact(nx, ny, D, film, U, P["W"])
    sc = _scales(P, R=D / 2)
    exact = oracle.Lattice(nx, ny, **P).init(phi0, u0, v0)
    members = [oracle.Lattice(nx, ny, **P).init(p, _round32(u0), _round32(v0)) for p in _spread_members(phi0)]
    with lbm.Lattice(nx, ny, **P) as g:
        g.init(phi0, u0, v0)
        done = 0
        for T in (200, 1250):
            exact.step(T - done)
            g.step(T - done)
            for m in members:
                m.step(T - done)
            done = T
            ref = exact.fields()
            spread = {k: 0.0 for k in sc}
            for m in members:
                for k, v in _field_errors(m.fields(), ref, sc).items():
                    spread[k] = max(spread[k], v)
            err = _field_errors(g.fields(), ref, sc)
            print(f"impact, step {T}: gpu vs oracle", _fmt(err), "| oracle spread", _fmt(spread))
            for k, v in err.items():
                assert np.isfinite(v) and v <= SPREAD_FACTOR * spread[k], (T, k, err, spread)


def test_impact_2400x600_spreading_radius_to_t1(lbm):
    """Droplet impact at full size (2400 x 600, walls, D = 200, film 20,
    U = 0.04, Re = 100, We = 8000, ratio 1000, mu ratio 40, W = 5): the
    spreading radius every t* = t U / D = 0.25 up to t* = 1 (5000 steps)
    within 1% of the oracle's (interpolated ends; the node-counted radius
    within 1% or one node)."""
    nx, ny, D, film, U = 2400, 600, 200.0, 20.0, 0.04
    P = cases.params_impact(Re=100.0)
    phi0, u0, v0 = cases.impact(nx, ny, D, film, U, P["W"])
    every = int(round(0.25 * D / U))
    o = oracle.Lattice(nx, ny, **P).init(phi0, u0, v0)
    with lbm.Lattice(nx, ny, **P) as g:
        g.init(phi0, u0, v0)
        for k in range(1, 5):
            g.step(every)
            o.step(every)
            fg, fo = g.fields(), o.fields()
            ri_g, ri_o = _radius_interp(fg["phi"], film, P["W"]), _radius_interp(fo["phi"], film, P["W"])
            r_g, r_o = _spreading_radius(fg["phi"], film, P["W"]), _spreading_radius(fo["phi"], film, P["W"])
            err = _field_errors(fg, fo, _scales(P, R=D / 2))
            print(f"impact t* = {0.25 * k:.2f}: radius gpu {ri_g:.3f} oracle {ri_o:.3f} "
                  f"(nodes {r_g} / {r_o}); fields", _fmt(err))
            assert abs(ri_g - ri_o) <= 0.01 * ri_o, (k, ri_g, ri_o)
            assert abs(r_g - r_o) <= max(0.01 * r_o, 1.0), (k, r_g, r_o)


# --------------------------------------------------------------- batch ----

def _batch_cases():
    """Uneven cases of all three boundary kinds, FP32 storage, whose flows keep
    phi without interior extrema over 100 steps (the free-run tier)."""
    out = []
    nx, ny = 100, 70   # a drop carried by a uniform flow, ragged periodic grid
    P = dict(rho_l=1.0, rho_g=1e-3, nu_l=0.1, nu_g=0.1, sigma=0.0, W=4.0)
    phi0 = cases.drop(nx, ny, 12, 4.0, x0=40, y0=30)
    out.append((nx, ny, P, (phi0, np.full_like(phi0, 0.01), np.full_like(phi0, -0.004)),
                {"phi": 1.0, "rho": 1.0, "ux": 0.01, "uy": 0.01, "p": 1e-8}))
    for bc in (1, 2):  # a drop resting on the lower wall, closed or open top
        nx, ny = 77, 45
        P = dict(rho_l=1.0, rho_g=0.01, nu_l=0.1, nu_g=0.3, visc_mode=0, sigma=0.01, W=4.0,
                 tau_h=0.8, Gx=1e-6, Gy=0.0, bc_y=bc)
        out.append((nx, ny, P, (cases.drop(nx, ny, 12, 4.0, x0=38, y0=8, walls_y=True),),
                    _scales(P, R=12)))
    P = cases.params_poiseuille(256, Gx=1e-7, mu_ratio=100.0)   # the layered Poiseuille config
    out.append((8, 256, P, (cases.layer(8, 256, P["W"]),), _scales(P)))
    return out


def test_batch_free_run_vs_oracle(lbm):
    """Four uneven cases (periodic, walls, wall with open top, the 8 x 256
    layered Poiseuille) advanced 100 steps together by lbm_batch_step (graph
    replays and a remainder), FP32 storage: each case's fields within 1e-5
    (p 3e-5) of the oracle's."""
    specs = _batch_cases()
    lats = [lbm.Lattice(nx, ny, **P).init(*init) for nx, ny, P, init, _ in specs]
    try:
        with lbm.Batch(lats) as b:
            b.step(100)
        for lat, (nx, ny, P, init, sc) in zip(lats, specs):
            ref = oracle.Lattice(nx, ny, **P).init(*init).step(100).fields()
            errs = _assert_fields(lat.fields(), ref, sc)
            print(f"batch free run {nx}x{ny} bc {P.get('bc_y', 0)}:", _fmt(errs))
    finally:
        for lat in lats:
            lat.close()


def test_batch_one_step_parity_from_oracle_states(lbm):
    """The oracle's state after 60 steps of each case, loaded into the batch's
    cases with lbm_set_state, then one lbm_batch_step: every population of
    every case against one oracle step (the one-step bounds)."""
    specs = _batch_cases()
    setups, lats = [], []
    try:
        for nx, ny, P, init, _ in specs:
            state = oracle.Lattice(nx, ny, **P).init(*init).step(60).get_state()
            S = _one_step_setup(nx, ny, P, state)
            setups.append(S)
            lats.append(lbm.Lattice(nx, ny, **P).set_state(*S["st32"]))
        with lbm.Batch(lats) as b:
            b.step(1)
        for S, lat in zip(setups, lats):
            _one_step_check(S, lat.get_state(), lat.fields())
    finally:
        for lat in lats:
            lat.close()
