"""The C ABI used from C: tests/c_client.c is compiled against include/lbm_pf.h
and linked with liblbm_pf.so, with no Python in between.

* CPU: the calls that need no GPU return their documented status.
* GPU: a 64 x 64 static drop stepped by the C client gives the same bits as
  the Python binding on the same input (the binding marshals arguments and
  nothing else), and its sum of phi matches the FP64 oracle's."""
import os
import subprocess

import numpy as np
import pytest

from paper_1710_09541_gb300 import build as lbm_build
from paper_1710_09541_gb300 import cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    lib = lbm_build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("c_client") / "c_client")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(ROOT, "tests", "c_client.c"), "-L", libdir, "-llbm_pf",
                    "-Wl,-rpath," + libdir], check=True)
    return exe


def test_c_client_host_calls(client):
    r = subprocess.run([client, "host"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.gpu
@pytest.mark.parametrize("storage", [0, 1])
def test_c_client_run_matches_the_binding(client, tmp_path, storage):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1710_09541_gb300 import lbm

    nx = ny = 64
    phi0 = cases.drop(nx, ny, 16, 4.0)
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(src, "wb") as fh:
        np.array([nx, ny], dtype=np.int32).tofile(fh)
        phi0.astype(np.float64).tofile(fh)
    r = subprocess.run([client, "run", str(storage), str(src), str(dst)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(dst, dtype=np.float64)
    fields = out[:5 * nx * ny].reshape(5, ny, nx)
    diag = out[5 * nx * ny:]
    lbm.load()
    with lbm.Lattice(nx, ny, storage=storage, **cases.params_static_drop()) as g:
        ref = g.init(phi0).step(50).fields()
        ref_diag = g.diag()
    for k, name in enumerate(("phi", "rho", "ux", "uy", "p")):
        assert np.array_equal(fields[k], ref[name]), name
    assert np.array_equal(diag, np.array(ref_diag))
    s64 = oracle.Lattice(nx, ny, **cases.params_static_drop()).init(phi0).step(50).sum_phi()
    assert abs(diag[0] / s64 - 1) < 1e-6
