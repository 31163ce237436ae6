"""The spinodal and impact workloads at full size, each storage format
against FP32 on the GPU (the FP32 path itself is checked against the FP64
oracle in test_gpu_parity.py).

Both flows amplify small perturbations, so a single FP32 run is not the
measure of what 16-bit storage may change.  Each test also runs FP32 from
the same input plus a 1e-6 perturbation (seeded normal noise on phi0) and
holds the 16-bit run to what such round-off-level perturbations do:

* spinodal decomposition, 1024 x 1024 periodic, density ratios 3 and 1000,
  FP32 vs FP16-shifted storage: the same pattern over the first 200 steps
  (the correlation of phi - 1/2), the liquid fraction, and the domain length
  up to 20 000 steps within 2% of the envelope of three FP32 runs (two of
  them perturbed).  Measured: the perturbed FP32 runs part by up to 4.9% in
  domain length at ratio 1000 (0.7% at ratio 3) by 20 000 steps; FP16 runs lie
  inside the envelope or at most 1.3% outside it.
* droplet impact, 2400 x 600 (D = 200, film 20, U = 0.04, We = 8000, ratio
  1000, mu ratio 40, W = 5, walls), Re = 20, 100, 500, FP32 vs BF16- and
  FP16-shifted storage, the spreading radius every t* = 0.5 up to t* = 4.  FP32 is robust:
  a perturbed run moves no sample by more than 0.3%.  BF16 is not, at single
  samples: where the lamella tip pinches off, the contiguous radius jumps, and
  over six BF16 runs (three inputs, two builds) single samples part from FP32
  by up to 19% at Re = 100 and 500.  The final radius agrees within 1.7%.
  At Re = 20 (deposition, no lamella) BF16 spreads 5-7% less (at worst 10.6%
  at t* = 1.5; 11.7% at t* = 4 in one run, after a rim pinch-off).
  FP16-shifted storage stays within 0.63% of FP32 at every sample for all
  three Reynolds numbers (bound 2%): its 11 significant bits resolve the
  per-step viscous change of the g codes that BF16's 8 bits round away.
  BF16 with the g codes rounded stochastically (BF16_SHIFTED_SR) keeps that
  change on average: at Re = 20 it stays within 0.6% of FP32 at every sample
  (four runs).  At Re = 100 and 500 the rounding noise decides when the lamella
  pinches off: in one of four Re = 100 runs a pinch-off at t* = 0.5 (+17.5%)
  left the radius 8-10% behind FP32 to t* = 4; the other three ended within
  2.9%.  At Re = 500 the final radius agreed within 0.3%.
  The power law r/D = C sqrt(t*) of Sec. III D (C = 1.35 at its own U = 0.05)
  holds with C in [0.9, 1.5] once the lamella has formed."""
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


def _domain_length(phi):
    a = phi > 0.5
    links = (a != np.roll(a, 1, 0)).sum() + (a != np.roll(a, 1, 1)).sum()
    return phi.size / max(links, 1)


def _perturbed(phi0, k):
    """phi0 itself (k = 0) or phi0 plus seeded normal noise of size 1e-6."""
    return phi0 if k == 0 else phi0 + 1e-6 * np.random.default_rng(k).standard_normal(phi0.shape)


@pytest.mark.parametrize("ratio", [3.0, 1000.0])
def test_spinodal_1024_fp32_vs_fp16(lbm, ratio):
    n = 1024
    P = cases.params_spinodal(ratio=ratio)
    phi0 = cases.spinodal(n, n, 0.5, 0.01, seed=12345)
    runs = [(0, 0), (0, 1), (0, 2), (1, 0)]               # (storage, perturbation)
    snaps, stats = {}, {}
    for st, k in runs:
        with lbm.Lattice(n, n, storage=st, **P) as g:
            g.init(_perturbed(phi0, k)).step(200)
            snaps[st, k] = g.fields()["phi"] - 0.5
            done, s = 200, []
            for t in (2000, 5000, 10000, 20000):
                g.step(t - done)
                done = t
                phi = g.fields()["phi"]
                s.append((_domain_length(phi), (phi > 0.5).mean()))
            drift = g.diag()[0] / phi0.sum() - 1
        stats[st, k] = np.array(s)
        assert abs(drift) < 5e-6, drift
    a, b = snaps[0, 0].ravel(), snaps[1, 0].ravel()
    corr = float(a @ b / np.sqrt((a @ a) * (b @ b)))
    assert corr > 0.999                                     # measured 0.99998 for both ratios
    ens = np.array([stats[0, k][:, 0] for k in range(3)])
    l16, f16, f32 = stats[1, 0][:, 0], stats[1, 0][:, 1], stats[0, 0][:, 1]
    assert np.all(l16 >= 0.98 * ens.min(0)) and np.all(l16 <= 1.02 * ens.max(0)), (ens, l16)
    assert np.all(np.abs(f16 / f32 - 1) < 0.005), (f32, f16)


@pytest.mark.parametrize("Re", [20.0, 100.0, 500.0])
def test_impact_2400x600_fp32_vs_16bit(lbm, Re):
    P = cases.params_impact(Re=Re)
    phi0, u0, v0 = cases.impact(2400, 600, 200.0, 20.0, 0.04, P["W"])
    row = int(round(20 + P["W"]))
    radii = {}
    for st, k in ((0, 0), (0, 1), (2, 0), (1, 0), (3, 0)):
        with lbm.Lattice(2400, 600, storage=st, **P) as g:
            g.init(_perturbed(phi0, k), u0, v0)
            r = []
            for _ in range(8):
                g.step(2500)                                  # t* += 0.5 (D / U = 5000 steps)
                r.append(g.spreading_radius(row)[1])
            assert np.isfinite(g.diag()[0])
        radii[st, k] = np.array(r)
    r32 = radii[0, 0]
    # FP32 does not amplify a 1e-6 perturbation on this measure (measured 0.3%)
    assert np.all(np.abs(radii[0, 1] / r32 - 1) < 0.01), (r32, radii[0, 1])
    # FP16-shifted storage follows FP32 at every sample (measured within 0.63%
    # at Re = 20, 100 and 500), the target config 4 sets for the radius
    assert np.all(np.abs(radii[1, 0] / r32 - 1) < 0.02), (r32, radii[1, 0])
    dev = np.abs(radii[2, 0] / r32 - 1)
    dsr = np.abs(radii[3, 0] / r32 - 1)
    if Re == 20.0:
        assert np.all(dev < 0.15) and dev[-1] < 0.12, (r32, radii[2, 0])
        # stochastic rounding removes the deposition's bias (measured 0.6%)
        assert np.all(dsr < 0.015), (r32, radii[3, 0])
    else:
        assert np.all(dev < 0.25) and dev[-1] < 0.03, (r32, radii[2, 0])
        # the noise can move a pinch-off, after which the radius trails (8.6% measured)
        assert np.all(dsr < 0.25) and dsr[-1] < 0.15, (r32, radii[3, 0])
        t = np.arange(1, 9) * 0.5
        C = r32 / 200.0 / np.sqrt(t)
        assert np.all((C[1:] > 0.9) & (C[1:] < 1.5)), C
