"""A stand-in for a sanitizer (compute-sanitizer is not available on the GPUs
these tests run on): the debug build of the library (liblbm_pf_debug.so)
checks every neighbour row and column and every shared-memory slot the step
computes, records an out-of-range one instead of touching memory, and
poisons each tile's phi slots with NaN before filling them, so a halo slot
left unwritten surfaces as a non-finite error.  Grids smaller than a tile,
one node wide, ragged in both directions, walled and open-topped, in all three
storage formats, and a batch, run through it: every call succeeds, and the
states equal the release library's bit for bit (the checks change no
arithmetic)."""
import numpy as np
import pytest

from paper_1710_09541_gb300 import cases

pytestmark = pytest.mark.gpu

GRIDS = [(1, 1, 0), (3, 5, 0), (5, 2, 1), (8, 8, 2), (31, 16, 1), (33, 17, 0), (100, 70, 0),
         (77, 45, 2)]


@pytest.fixture(scope="module")
def libs():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09541_gb300 import build as lbm_build
    from paper_1710_09541_gb300 import lbm

    release, debug = lbm_build.build(), lbm_build.build(debug=True)
    saved = (lbm._LIB_PATH, lbm._lib)
    yield lbm, release, debug
    lbm._LIB_PATH, lbm._lib = saved


def _use(lbm, path):
    lbm._LIB_PATH, lbm._lib = path, None
    lbm.load()


def _states(lbm, nx, ny, bc, storage):
    P = dict(rho_l=1.0, rho_g=0.1, nu_l=0.1, nu_g=0.1, visc_mode=0, sigma=0.01, W=3.0,
             tau_h=0.8, Gx=1e-5, Gy=2e-5, bc_y=bc, check_every=1)
    r = np.random.default_rng(nx * 100 + ny)
    phi0 = 0.5 + 0.3 * r.random((ny, nx))
    ux0 = 1e-3 * r.standard_normal((ny, nx))
    with lbm.Lattice(nx, ny, storage=storage, **P) as g:
        g.init(phi0, ux0).step(20)
        F = g.fields()
        return g.get_state(), F


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_debug_build_single_case_grids(libs, storage):
    lbm, release, debug = libs
    out = {}
    for path in (debug, release):
        _use(lbm, path)
        out[path] = [_states(lbm, nx, ny, bc, storage) for nx, ny, bc in GRIDS]
    for (sd, Fd), (sr, Fr) in zip(out[debug], out[release]):
        for a, b in zip(sd, sr):
            assert np.array_equal(a, b)
        for k in Fd:
            assert np.array_equal(Fd[k], Fr[k]), k


def test_debug_build_batch(libs):
    lbm, release, debug = libs
    specs = cases.batch_cases(n=6, seed=11)
    specs[3]["params"] = dict(specs[3]["params"], bc_y=2)
    for sp in specs:
        sp["params"] = dict(sp["params"], check_every=1)
    out = {}
    for path in (debug, release):
        _use(lbm, path)
        lats = [lbm.Lattice(sp["nx"], sp["ny"], storage=1, **sp["params"])
                .init(sp["phi0"], sp["ux0"], sp["uy0"]) for sp in specs]
        try:
            with lbm.Batch(lats) as bt:
                bt.step(37)
            out[path] = [lat.get_state() for lat in lats]
        finally:
            for lat in lats:
                lat.close()
    for sd, sr in zip(out[debug], out[release]):
        for a, b in zip(sd, sr):
            assert np.array_equal(a, b)
