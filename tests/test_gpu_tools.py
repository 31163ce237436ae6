"""Impact-case tooling on the device (lbm_spreading_radius, lbm_probe):
values equal those derived from lbm_get_fields bit for bit, and the
spreading radius follows its definition (half the x-extent of the phi >= 1/2
run through the centre column) and the oracle's within 1%."""
import numpy as np
import pytest

import oracle
from paper_1710_09541_gb300 import cases
from tests.test_gpu_parity import _spreading_radius

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_probe_equals_fields(lbm, storage, bc):
    nx, ny = 70, 45
    P = dict(cases.params_static_drop(ratio=100.0), bc_y=bc)
    phi0 = cases.drop(nx, ny, 11, 4.0, x0=20.0, y0=14.0, walls_y=bc > 0)
    r = np.random.default_rng(storage * 3 + bc)
    xs = np.concatenate([[0, nx - 1, 0, nx - 1, 20], r.integers(0, nx, 200)])
    ys = np.concatenate([[0, 0, ny - 1, ny - 1, 14], r.integers(0, ny, 200)])
    with lbm.Lattice(nx, ny, storage=storage, **P) as g:
        g.init(phi0, np.full_like(phi0, 0.003), np.full_like(phi0, -0.002)).step(37)
        F = g.fields()
        got = g.probe(xs, ys)
    for k in ("phi", "rho", "ux", "uy", "p"):
        assert np.all(np.isfinite(F[k])), k
        assert np.array_equal(got[k], F[k][ys, xs]), k


def test_probe_rejects_points_outside(lbm):
    with lbm.Lattice(16, 12, **cases.params_static_drop()) as g:
        g.init(cases.drop(16, 12, 4, 4.0))
        for x, y in (([16], [0]), ([0], [12]), ([-1], [3])):
            with pytest.raises(lbm.LbmError) as e:
                g.probe(x, y)
            assert e.value.status == lbm.LBM_ERR_INVALID
        assert g.probe([], [])["p"].size == 0


@pytest.mark.parametrize("bc", [1, 2])
@pytest.mark.parametrize("storage", [0, 1])
def test_spreading_radius_definition_and_oracle(lbm, bc, storage):
    """Impact scaled to D = 40 on 480 x 120 (film 4, U = 0.04, Re = 100): at
    t* = 0.25 ... 1 the device radius equals the definition applied to the
    GPU's own phi; r_interp lies within half a node of it; against the FP64
    oracle within 1% (or one node) for FP32 storage."""
    nx, ny, D, film = 480, 120, 40.0, 4.0
    P = dict(cases.params_impact(D=D, Re=100.0), bc_y=bc)
    phi0, u0, v0 = cases.impact(nx, ny, D, film, 0.04, P["W"])
    row = int(round(film + P["W"]))
    o = oracle.Lattice(nx, ny, **P).init(phi0, u0, v0) if storage == 0 else None
    with lbm.Lattice(nx, ny, storage=storage, **P) as g:
        g.init(phi0, u0, v0)
        for _ in range(4):
            g.step(250)
            r, ri = g.spreading_radius(row)
            assert r == _spreading_radius(g.fields()["phi"], film, P["W"])
            assert r > 0 and r - 0.5 <= ri <= r + 0.5
            if o is not None:
                o.step(250)
                ro = _spreading_radius(o.fields()["phi"], film, P["W"])
                assert abs(r - ro) <= max(0.01 * ro, 1.0)
        # inside the film the run spans the whole row; above the drop, no liquid
        assert g.spreading_radius(1) == (nx / 2, nx / 2)
        assert g.spreading_radius(ny - 2) == (0.0, 0.0)
        with pytest.raises(lbm.LbmError):
            g.spreading_radius(ny)


def _jump_host(p, xc, yc, r_in, r_out, periodic_y):
    ny, nx = p.shape
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    dx = xx - xc
    dx -= nx * np.rint(dx / nx)
    dy = yy - yc
    if periodic_y:
        dy -= ny * np.rint(dy / ny)
    r2 = dx * dx + dy * dy
    return p[r2 < r_in * r_in].mean() - p[r2 > r_out * r_out].mean()


@pytest.mark.parametrize("bc", [0, 1])
def test_laplace_jump_matches_fields(lbm, bc):
    """The device reduction equals the same averages taken on the read-back p
    (FP64 sums in a different order), including a centre near the periodic
    seam."""
    nx, ny = 70, 45
    P = dict(cases.params_static_drop(ratio=100.0), bc_y=bc)
    # the drop straddles the periodic seam: union of its two images in x
    phi0 = np.maximum(cases.drop(nx, ny, 11, 4.0, x0=3.0, y0=22.0, walls_y=bc > 0),
                      cases.drop(nx, ny, 11, 4.0, x0=3.0 + nx, y0=22.0, walls_y=bc > 0))
    with lbm.Lattice(nx, ny, **P) as g:
        g.init(phi0).step(300)
        assert np.isfinite(g.diag()[0])
        p = g.fields()["p"]
        for xc, yc, ri, ro in ((3.0, 22.0, 5.5, 20.0), (35.0, 22.0, 3.0, 25.0)):
            got = g.laplace_jump(xc, yc, ri, ro)
            ref = _jump_host(p, xc, yc, ri, ro, bc == 0)
            assert abs(got - ref) <= 1e-12 * max(abs(ref), 1e-12), (got, ref)
        for bad in ((3.0, 22.0, 0.0, 5.0), (3.0, 22.0, 6.0, 5.0), (3.3, 22.3, 0.2, 5.0)):
            with pytest.raises(lbm.LbmError) as e:
                g.laplace_jump(*bad)
            assert e.value.status == lbm.LBM_ERR_INVALID


def test_laplace_jump_resolved_drop_vs_oracle(lbm):
    """A resolved drop (W = 8, R = 20, 96 x 96, ratio 1000, sigma = 0.01):
    the time-averaged device jump follows the FP64 oracle's within 1% and the
    Laplace law sigma/R within 3%."""
    n, R = 96, 20
    P = dict(cases.params_static_drop(), W=8.0)
    phi0 = cases.drop(n, n, R, 8.0)
    o = oracle.Lattice(n, n, **P).init(phi0).step(8000)
    got, ref = [], []
    with lbm.Lattice(n, n, **P) as g:
        g.init(phi0).step(8000)
        for _ in range(16):
            g.step(125)
            o.step(125)
            got.append(g.laplace_jump(n / 2, n / 2, R / 2, R + 12))
            ref.append(_jump_host(o.fields()["p"], n / 2, n / 2, R / 2, R + 12, True))
    assert abs(np.mean(got) / np.mean(ref) - 1) < 0.01
    assert abs(np.mean(got) * R / 0.01 - 1) < 0.03
