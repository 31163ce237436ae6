"""Lattices whose device state lives in a caller's buffer (lbm_create_in with
a PyTorch tensor): the same bits as a library-allocated lattice, the buffer
left alive after the lattice is destroyed, and host or undersized buffers
rejected before any kernel could touch them."""
import numpy as np
import pytest

from paper_1710_09541_gb300 import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09541_gb300 import build as lbm_build
    from paper_1710_09541_gb300 import lbm as _lbm

    lbm_build.build()
    _lbm.load()
    return _lbm, torch


@pytest.mark.parametrize("storage,bc", [(0, 0), (1, 2), (2, 1)])
def test_workspace_lattice_equals_allocated_one(env, storage, bc):
    lbm, torch = env
    nx, ny = 96, 64
    P = dict(cases.params_impact(D=24.0, Re=100.0), bc_y=bc) if bc else cases.params_static_drop(ratio=100.0)
    if bc:
        phi0, u0, v0 = cases.impact(nx, ny, 24.0, 2.4, 0.04, P["W"])
    else:
        phi0, u0, v0 = cases.drop(nx, ny, 14, 4.0), None, None
    n = lbm.workspace_bytes(nx, ny, storage=storage, **P)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    with lbm.Lattice(nx, ny, storage=storage, workspace=ws, **P) as a, \
            lbm.Lattice(nx, ny, storage=storage, **P) as b:
        a.init(phi0, u0, v0).step(77)
        b.init(phi0, u0, v0).step(77)
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(x, y)
        Fa, Fb = a.fields(), b.fields()
        for k in Fa:
            assert np.array_equal(Fa[k], Fb[k]), k
        assert a.diag() == b.diag()
    # the library did not free the caller's buffer
    ws.fill_(7)
    torch.cuda.synchronize()
    assert int(ws[:16].sum()) == 7 * 16


def test_workspace_rejects_host_and_small_buffers(env):
    lbm, torch = env
    P = cases.params_static_drop()
    n = lbm.workspace_bytes(32, 32, **P)
    for bad in (torch.empty(n, dtype=torch.uint8),                      # pageable host memory
                torch.empty(n, dtype=torch.uint8).pin_memory(),         # pinned host memory
                torch.empty(n - 256, dtype=torch.uint8, device="cuda")):  # too small
        with pytest.raises(lbm.LbmError) as e:
            lbm.Lattice(32, 32, workspace=bad, **P)
        assert e.value.status == lbm.LBM_ERR_INVALID
