"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/lbm_pf.h declares, and rejects bad parameters
before touching the device."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

from paper_1710_09541_gb300 import build as lbm_build
from paper_1710_09541_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    lbm_build.build()
    return lbm.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src))
    return names


def test_header_declares_the_binding_names():
    assert _declared() == set(lbm.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_params_struct_layout_matches_header(tmp_path):
    """Compile a C probe against include/lbm_pf.h and compare the size and
    every field offset of lbm_params with the ctypes mirror."""
    fields = [f[0] for f in lbm.lbm_params._fields_]
    src = tmp_path / "probe.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm_pf.h"\n'
                   "int main(void){printf(\"%zu\\n\", sizeof(lbm_params));"
                   + "".join(f'printf("%zu\\n", offsetof(lbm_params, {f}));' for f in fields)
                   + "return 0;}\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                           text=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(lbm.lbm_params)
    assert vals[1:] == [getattr(lbm.lbm_params, f).offset for f in fields]


@pytest.mark.parametrize("bad", [
    dict(rho_g=0.0), dict(nu_l=-1.0), dict(visc_mode=3), dict(W=0.0), dict(tau_h=0.5),
    dict(sigma=-1.0), dict(bc_y=3), dict(bc_y=-1), dict(bc_y=2, kernel=2), dict(normal_scheme=5), dict(storage=7), dict(check_every=-1),
    dict(Gx=float("inf")),
])
def test_create_rejects_bad_parameters(L, bad):
    p = lbm.make_params(**bad)
    h = ctypes.c_void_p()
    assert L.lbm_create(16, 16, ctypes.byref(p), ctypes.byref(h)) == lbm.LBM_ERR_INVALID
    assert not h.value


# nx * ny must stay below floor(2^31 / 20) = 107374182 so that every 32-bit
# index of the 20-plane state permutation fits; one node past the limit fails
@pytest.mark.parametrize("nx,ny", [(0, 4), (4, 0), (-3, 5), (1 << 20, 1 << 20), (1, 107374182),
                                   (107374182, 1), (16384, 6554)])
def test_create_rejects_bad_sizes(L, nx, ny):
    p = lbm.make_params()
    h = ctypes.c_void_p()
    assert L.lbm_create(nx, ny, ctypes.byref(p), ctypes.byref(h)) == lbm.LBM_ERR_INVALID


def test_workspace_bytes_and_create_in_checks(L):
    """No CUDA call is needed to size a workspace or to reject a bad one."""
    p = lbm.make_params(storage=lbm.LBM_STORE_FP16_SHIFTED)
    n = ctypes.c_size_t()
    assert L.lbm_workspace_bytes(64, 32, ctypes.byref(p), ctypes.byref(n)) == lbm.LBM_OK
    N = 64 * 32
    assert n.value >= 2 * 38 * N + 8 * N + 80 * N and n.value % 256 == 0
    p32 = lbm.make_params()
    n32 = ctypes.c_size_t()
    assert L.lbm_workspace_bytes(64, 32, ctypes.byref(p32), ctypes.byref(n32)) == lbm.LBM_OK
    assert n32.value > n.value                        # FP32 populations take 160 B/node
    bad = lbm.make_params(tau_h=0.4)
    assert L.lbm_workspace_bytes(64, 32, ctypes.byref(bad), ctypes.byref(n)) == lbm.LBM_ERR_INVALID
    h = ctypes.c_void_p()
    # NULL, too small, misaligned: rejected before the pointer is ever used
    assert L.lbm_create_in(64, 32, ctypes.byref(p32), None, n32.value, ctypes.byref(h)) == lbm.LBM_ERR_INVALID
    assert L.lbm_create_in(64, 32, ctypes.byref(p32), 1 << 20, n32.value - 1,
                           ctypes.byref(h)) == lbm.LBM_ERR_INVALID
    assert L.lbm_create_in(64, 32, ctypes.byref(p32), (1 << 20) + 16, n32.value,
                           ctypes.byref(h)) == lbm.LBM_ERR_INVALID
    assert not h.value


def test_storage_formats_and_their_sizes(L):
    """The stochastically rounded BF16 format keeps BF16's layout; an unknown
    format is rejected."""
    sizes = []
    for st in (lbm.LBM_STORE_FP16_SHIFTED, lbm.LBM_STORE_BF16_SHIFTED, lbm.LBM_STORE_BF16_SHIFTED_SR):
        p = lbm.make_params(storage=st)
        n = ctypes.c_size_t()
        assert L.lbm_workspace_bytes(64, 32, ctypes.byref(p), ctypes.byref(n)) == lbm.LBM_OK
        sizes.append(n.value)
    assert sizes[0] == sizes[1] == sizes[2]
    n = ctypes.c_size_t()
    for st in (-1, 4):
        p = lbm.make_params(storage=st)
        assert L.lbm_workspace_bytes(64, 32, ctypes.byref(p), ctypes.byref(n)) == lbm.LBM_ERR_INVALID


def test_open_top_needs_two_rows(L):
    p = lbm.make_params(bc_y=lbm.LBM_BC_WALL_OPEN)
    h = ctypes.c_void_p()
    assert L.lbm_create(16, 1, ctypes.byref(p), ctypes.byref(h)) == lbm.LBM_ERR_INVALID
    assert not h.value


def test_header_enum_values_match_the_binding():
    import re
    text = open(os.path.join(ROOT, "include", "lbm_pf.h")).read()
    for name in ("LBM_BC_PERIODIC", "LBM_BC_WALLS", "LBM_BC_WALL_OPEN", "LBM_STORE_FP32",
                 "LBM_STORE_FP16_SHIFTED", "LBM_STORE_BF16_SHIFTED", "LBM_STORE_BF16_SHIFTED_SR",
                 "LBM_KERNEL_AUTO",
                 "LBM_KERNEL_GENERIC"):
        m = re.search(name + r"\s*=\s*(\d+)", text)
        assert m and int(m.group(1)) == getattr(lbm, name), name


def test_null_handle_calls_are_rejected(L):
    assert L.lbm_step(None, 1) == lbm.LBM_ERR_INVALID
    assert L.lbm_get_fields(None, None, None, None, None, None) == lbm.LBM_ERR_INVALID
    assert L.lbm_diag(None, None, None, None, None) == lbm.LBM_ERR_INVALID
    assert L.lbm_state_bytes(None) == 0
    assert L.lbm_spreading_radius(None, 0, 0, None, None) == lbm.LBM_ERR_INVALID
    assert L.lbm_laplace_jump(None, 0.0, 0.0, 1.0, 2.0, None) == lbm.LBM_ERR_INVALID
    assert L.lbm_probe(None, 0, None, None, None, None, None, None, None) == lbm.LBM_ERR_INVALID
    L.lbm_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    """Without the CUDA library the binding raises ImportError; there is no
    CPU fallback, and nothing in the package imports the oracle."""
    code = (
        "import sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_1710_09541_gb300 import cases, lbm\n"
        f"lbm._LIB_PATH, lbm._lib = {str(tmp_path / 'absent.so')!r}, None\n"
        "try:\n"
        "    lbm.Lattice(8, 8)\n"
        "except ImportError:\n"
        "    pass\n"
        "else:\n"
        "    sys.exit(1)\n"
        "sys.exit(2 if 'oracle' in sys.modules else 0)\n")
    assert subprocess.run([sys.executable, "-c", code], cwd=str(tmp_path)).returncode == 0


def test_batch_calls_check_their_arguments_on_the_host(L):
    """lbm_batch_create rejects a missing output, a case count outside
    1..200, a missing case array and a NULL case before any device work; the
    other batch calls reject a NULL batch."""
    out = ctypes.c_void_p(1)
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.lbm_batch_create(1, arr, None) == lbm.LBM_ERR_INVALID
    for n, cases_ in ((0, arr), (201, arr), (1, None), (2, arr)):
        out.value = 1
        assert L.lbm_batch_create(n, cases_, ctypes.byref(out)) == lbm.LBM_ERR_INVALID, n
        assert not out.value
    n = ctypes.c_int()
    assert L.lbm_batch_step(None, 1) == lbm.LBM_ERR_INVALID
    assert L.lbm_batch_info(None, 0, ctypes.byref(n), None, None, None, None) == lbm.LBM_ERR_INVALID
    assert L.lbm_batch_last_error(None)
    L.lbm_batch_destroy(None)
