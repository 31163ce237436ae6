"""Batched stepping (lbm_batch_*): many independent cases of uneven sizes and
parameters advanced by one kernel launch per step, replayed as a CUDA graph,
with the tile height chosen by timing.  A case advanced in a batch must give
the same bits as the same case advanced alone with lbm_step."""
import numpy as np
import pytest

from paper_1710_09541_gb300 import cases

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


def _lattices(lbm, specs, storage):
    out = []
    for s in specs:
        lat = lbm.Lattice(s["nx"], s["ny"], storage=storage, **s["params"])
        lat.init(s["phi0"], s["ux0"], s["uy0"])
        out.append(lat)
    return out


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_batch_equals_individual_steps(lbm, storage):
    """Six cases (drops periodic, impacts walled, sizes 256..1024 x 256..512):
    7 batch steps (no graph), one case stepped alone, then 150 batch steps
    (tuning, graph replays and a remainder) against each case stepped alone."""
    specs = cases.batch_cases(n=6, seed=11)
    specs[3]["params"] = dict(specs[3]["params"], bc_y=2)   # one impact with the open top
    A = _lattices(lbm, specs, storage)
    B = _lattices(lbm, specs, storage)
    try:
        with lbm.Batch(A) as bt:
            bt.step(7)
            A[2].step(3)
            bt.step(150)
            info = bt.info()
            assert info["tuned"]
            assert info["periodic"]["cases"] == 3 and info["walls"]["cases"] == 3
            # tile shapes in nodes: the thread blocks 32x4, 32x8, 32x16, 64x2, 64x4, whose
            # threads take one node each with FP32 storage and two (stacked in y) with 16 bits
            k = 1 if storage == 0 else 2
            shapes = tuple((tx, k * ty) for tx, ty in ((32, 4), (32, 8), (32, 16), (64, 2), (64, 4)))
            for cls in ("periodic", "walls"):
                assert info[cls]["tile"] in shapes
                assert info[cls]["us"] > 0
        for k, lat in enumerate(B):
            lat.step(157 + (3 if k == 2 else 0))
        for a, b in zip(A, B):
            for x, y in zip(a.get_state(), b.get_state()):
                assert np.array_equal(x, y)
    finally:
        for lat in A + B:
            lat.close()


@pytest.mark.parametrize("odd", [False, True])
def test_large_batch_with_prefetch_equals_individual_steps(lbm, odd):
    """The 64-case sweep with FP16 storage (16.5 M nodes, 1.5 GB per step,
    so the batched kernel prefetches the tile two per SM ahead), 10 steps,
    against four of its cases stepped alone, bit for bit.  Every case of the
    sweep has nx % 8 == 0, and the prefetch goes through the cases' tensor
    maps; with one more case of nx = 1004 the whole batch falls back to
    per-thread prefetch requests.  Small batches, as in the other tests, run
    without the prefetch."""
    specs = cases.batch_cases()
    pick = [0, 1, 36, 63]
    if odd:
        P = cases.params_static_drop(ratio=100.0)
        phi0 = cases.drop(1004, 300, 40.0, P["W"])
        specs = specs + [dict(nx=1004, ny=300, kind="static_drop", params=P, phi0=phi0,
                              ux0=np.zeros_like(phi0), uy0=np.zeros_like(phi0))]
        pick.append(64)
    A = _lattices(lbm, specs, 1)
    B = _lattices(lbm, [specs[k] for k in pick], 1)
    try:
        with lbm.Batch(A) as bt:
            bt.step(10)
        for lat in B:
            lat.step(10)
        for k, b in zip(pick, B):
            for x, y in zip(A[k].get_state(), b.get_state()):
                assert np.array_equal(x, y), k
    finally:
        for lat in A + B:
            lat.close()


@pytest.mark.parametrize("kinds", ["static_drop", "impact"])
def test_batch_of_one_class(lbm, kinds):
    """All cases in one boundary class (the other class empty), an odd step
    count so the graph is re-captured on the next call."""
    specs = [sp for sp in cases.batch_cases(n=8, seed=5) if sp["kind"] == kinds][:3]
    A = _lattices(lbm, specs, 1)
    B = _lattices(lbm, specs, 1)
    try:
        with lbm.Batch(A) as bt:
            bt.step(101)
            bt.step(65)
            info = bt.info()
            empty = "walls" if kinds == "static_drop" else "periodic"
            assert info[empty]["cases"] == 0 and info[empty]["us"] == 0
        for lat in B:
            lat.step(166)
        for a, b in zip(A, B):
            for x, y in zip(a.get_state(), b.get_state()):
                assert np.array_equal(x, y)
    finally:
        for lat in A + B:
            lat.close()


def test_batch_rejects_mixed_storage_and_repeats(lbm):
    specs = cases.batch_cases(n=2, seed=3)
    a = _lattices(lbm, specs[:1], 0)[0]
    b = _lattices(lbm, specs[1:], 1)[0]
    try:
        with pytest.raises(lbm.LbmError):
            lbm.Batch([a, b])
        with pytest.raises(lbm.LbmError):
            lbm.Batch([a, a])
    finally:
        a.close()
        b.close()


def test_batch_rejects_stochastic_rounding(lbm):
    """A batch replays fixed launches, which have no per-step seed for the
    dithers: BF16_SHIFTED_SR cases are stepped one by one."""
    specs = cases.batch_cases(n=2, seed=3)
    lats = _lattices(lbm, specs, 3)
    try:
        with pytest.raises(lbm.LbmError):
            lbm.Batch(lats)
    finally:
        for lat in lats:
            lat.close()


def test_batch_at_the_case_limit(lbm):
    """200 small cases (the kernel-parameter table's capacity) of mixed
    boundary kinds and sizes; a 201st is rejected."""
    specs = []
    r = np.random.default_rng(4)
    for k in range(201):
        nx, ny = int(r.integers(8, 40)), int(r.integers(4, 24))
        P = dict(cases.params_static_drop(ratio=10.0), bc_y=k % 3)
        phi0 = cases.drop(nx, ny, min(nx, ny) / 3, 3.0, walls_y=k % 3 > 0)
        specs.append(dict(nx=nx, ny=ny, params=P, phi0=phi0, ux0=None, uy0=None))
    A = _lattices(lbm, specs[:200], 1)
    B = _lattices(lbm, specs[:200], 1)
    extra = _lattices(lbm, specs[200:], 1)
    try:
        with pytest.raises(lbm.LbmError):
            lbm.Batch(A + extra)
        with lbm.Batch(A) as bt:
            bt.step(133)
        for lat in B:
            lat.step(133)
        for a, b in zip(A, B):
            for x, y in zip(a.get_state(), b.get_state()):
                assert np.array_equal(x, y)
    finally:
        for lat in A + B + extra:
            lat.close()


def test_batch_reports_nonfinite_case(lbm):
    """A NaN planted in one case's state (host side, through lbm_set_state)
    makes a batch step with check_every > 0 fail with LBM_ERR_NONFINITE naming
    that case; the flags are cleared afterwards."""
    specs = cases.batch_cases(n=4, seed=21)
    for sp in specs:
        sp["params"] = dict(sp["params"], check_every=1)
    A = _lattices(lbm, specs, 0)
    try:
        with lbm.Batch(A) as bt:
            bt.step(3)
            f, g, phiu = A[2].get_state()
            f = f.copy()
            f[3, 10, 10] = np.nan
            A[2].set_state(f, g, phiu)
            with pytest.raises(lbm.LbmError) as e:
                bt.step(4)
            assert e.value.status == lbm.LBM_ERR_NONFINITE
            assert "case 2" in str(e.value)
            for k in (0, 1, 3):
                assert np.isfinite(A[k].diag()[0])
    finally:
        for lat in A:
            lat.close()
