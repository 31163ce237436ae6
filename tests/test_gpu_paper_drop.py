"""The static droplet of Sec. III A on the GPU against the FP64 oracle's
equilibrium: 200 x 200 periodic, R = 50, density ratio 1000, nu = 0.1,
sigma = 0.001, W = 5, tau_h = 0.8, 200 000 steps.  The expected values come
from tests/golden/paper_drop_equilibrium.txt, written from the oracle alone
by make_paper_drop_equilibrium.py.

* FP32 storage, both normals: the maximum spurious speed within 5% and the
  pressure jump within 0.2% of the oracle's (measured on GB300: 1.10e-6
  against 1.09e-6, and 0.9526 against 0.9526 in units of sigma / R).
* FP16-shifted storage, Eq. 29 normal: the jump within 1% (measured 0.953).
  The spurious speed sits at the storage's floor (1.5e-5 to 2.3e-5 between
  1e5 and 1e6 steps), and is bounded by 5e-5.

The paper prints a maximum spurious speed of about 1.6e-9 for this setup.
Neither the oracle nor the GPU reproduces it: both settle near 1.1e-6, on the
gas side of the interface."""
import os

import numpy as np
import pytest

from paper_1710_09541_gb300 import cases

pytestmark = pytest.mark.gpu

N, R, STEPS = 200, 50.0, 200000
PARAMS = dict(rho_l=1.0, rho_g=1e-3, nu_l=0.1, nu_g=0.1, visc_mode=0, sigma=0.001, W=5.0, tau_h=0.8)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_drop_equilibrium.txt")


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


def _equilibrium(lbm, normal_scheme, storage):
    with lbm.Lattice(N, N, storage=storage, normal_scheme=normal_scheme, **PARAMS) as g:
        g.init(cases.drop(N, N, R, 5.0)).step(STEPS)
        F = g.fields()
    yy, xx = np.mgrid[0:N, 0:N]
    r = np.hypot(xx - N / 2, yy - N / 2)
    dp = F["p"][r < R / 2].mean() - F["p"][r > 1.5 * R].mean()
    return np.hypot(F["ux"], F["uy"]).max(), dp * R / PARAMS["sigma"]


def _golden():
    return {int(row[0]): (row[1], row[2]) for row in np.loadtxt(GOLDEN, ndmin=2)}


@pytest.mark.parametrize("normal_scheme", [0, 1])
def test_paper_drop_equilibrium_fp32(lbm, normal_scheme):
    umax_o, jump_o = _golden()[normal_scheme]
    umax, jump = _equilibrium(lbm, normal_scheme, 0)
    assert abs(umax / umax_o - 1) < 0.05, (umax, umax_o)
    assert abs(jump / jump_o - 1) < 0.002, (jump, jump_o)


def test_paper_drop_equilibrium_fp16(lbm):
    umax_o, jump_o = _golden()[1]
    umax, jump = _equilibrium(lbm, 1, 1)
    assert abs(jump / jump_o - 1) < 0.01, (jump, jump_o)
    assert umax < 5e-5, umax
