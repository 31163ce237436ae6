"""lbm_diag_fields_noalloc: the grid reductions for callers that cannot
allocate device memory when they ask for them (a process whose device memory
is owned by its own pool, or a stepping loop that must not synchronise the
device, which cudaMalloc/cudaFree may do).  The entry point keeps its block
partials in a fixed array inside the library instead of allocating.

Checked against lbm_diag, the handle-based entry point, on two calls in a row
with different sizes (so stale partials left by the first call would show up
in the second), plus the empty case and the size limit.  Collected last so a
failure here cannot hide the other tests; it also passes alone in a fresh
process, where its first call performs the per-device set-up."""
import numpy as np
import pytest

from paper_1710_09541_gb300 import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09541_gb300 import build as lbm_build
    from paper_1710_09541_gb300 import lbm

    lbm_build.build()
    lbm.load()
    return torch, lbm


def _lattice_fields_and_diag(lbm, nx, ny, steps, seed):
    P = cases.params_static_drop()
    phi0 = np.maximum(cases.drop(nx, ny, min(nx, ny) / 4, 4.0), 0.01 * cases.spinodal(nx, ny, seed=seed))
    with lbm.Lattice(nx, ny, **P) as g:
        g.init(phi0).step(steps)
        F = g.fields()
        ref = g.diag()
    return np.stack([F[k] for k in ("phi", "rho", "ux", "uy", "p")]), ref


def _noalloc(torch, lbm, fields):
    n = fields.shape[1] * fields.shape[2]
    d_fields = torch.tensor(fields.reshape(5, n), dtype=torch.float64, device="cuda")
    d_out = torch.full((4,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    lbm.diag_fields_noalloc(d_fields.data_ptr(), n, d_out.data_ptr(), stream=stream)
    torch.cuda.synchronize()
    return d_out.cpu().numpy()


def _same(got, ref):
    s, umax, pmin, pmax = ref
    assert abs(got[0] - s) <= 1e-12 * abs(s)
    assert got[1] == umax and got[2] == pmin and got[3] == pmax


def test_noalloc_matches_lbm_diag_on_two_calls(env):
    torch, lbm = env
    big, ref_big = _lattice_fields_and_diag(lbm, 1024, 512, 20, seed=3)     # 128 partial slots
    small, ref_small = _lattice_fields_and_diag(lbm, 100, 70, 30, seed=4)   # 2 partial slots
    _same(_noalloc(torch, lbm, big), ref_big)
    _same(_noalloc(torch, lbm, small), ref_small)


def test_noalloc_empty_and_limits(env):
    torch, lbm = env
    d_out = torch.zeros(4, dtype=torch.float64, device="cuda")
    lbm.diag_fields_noalloc(0, 0, d_out.data_ptr())
    torch.cuda.synchronize()
    out = d_out.cpu().numpy()
    assert out[0] == 0 and out[1] == 0 and out[2] == np.inf and out[3] == -np.inf
    with pytest.raises(lbm.LbmError) as e:
        lbm.diag_fields_noalloc(d_out.data_ptr(), 4096 * 4096 + 1, d_out.data_ptr())
    assert e.value.status == lbm.LBM_ERR_INVALID and "maximum" in str(e.value)
    with pytest.raises(lbm.LbmError):
        lbm.diag_fields_noalloc(d_out.data_ptr(), 10, 0)
