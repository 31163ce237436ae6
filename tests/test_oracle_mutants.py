"""The oracle's pins are strong enough: each of 39 plausible mistakes, planted
in a temporary copy of the oracle's C source, makes a named pin fail.

A mistake is one textual change (a dropped term, a wrong sign, factor, index
or direction, a swapped phase) in one part of the step: the lattice (Eq. 10),
the equilibria (Eqs. 9, 16, 17), the source terms (Eqs. 11, 20), the
closures (Eqs. 13, 23-26), the stencils (Eqs. 27, 28), the chemical
potential (Eqs. 6, 7), the recovery of u and p (Eq. 22), the collision
(Eqs. 2, 3, 8, 15), the normal of Eq. 29, the d_t(phi u) history, streaming
and the boundaries.  The pin named for it is the fastest of those that catch
it; the unit and physics pins are named wherever one catches the mistake,
the independent NumPy transcription only where none does.

Each mutant is compiled and run in its own process (one thread each); the
oracle's own source is never modified."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")

U = "tests.test_oracle_units"
PH = "tests.test_oracle_physics"

# (name, original text, planted text, (pin module, pin function, arguments))
MUTANTS = [
    ("diagonal weight 1/18", "1.0 / 36.0, 1.0 / 36.0};", "1.0 / 36.0, 1.0 / 18.0};",
     (U, "test_lattice_isotropy", ())),
    ("c_2 and c_4 swapped", "static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};",
     "static const int CY[9] = {0, 0, -1, 0, 1, 1, 1, -1, -1};", (U, "test_lattice_matches_eq10", ())),
    ("opposite map ignores c_y", "if (CX[j] == -CX[i] && CY[j] == -CY[i]) return j;",
     "if (CX[j] == -CX[i] && CY[j] == CY[i]) return j;", (PH, "test_phi_is_conserved", (1,))),
    ("f^eq without 1/c_s^2", "feq[i] = WGT[i] * phi * (1.0 + cu / CS2);",
     "feq[i] = WGT[i] * phi * (1.0 + cu);", (U, "test_feq_moments", (0,))),
    ("s_i: sign of u.u", "- uu / (2.0 * CS2));", "+ uu / (2.0 * CS2));", (U, "test_geq_moments_A1", (0,))),
    ("g_0^eq without -1", "(p / CS2) * (WGT[0] - 1.0)", "(p / CS2) * WGT[0]",
     (U, "test_geq_moments_A1", (0,))),
    ("F_i prefactor 1 - 1/tau", "Fi[i] = (1.0 - 1.0 / (2.0 * tau_f))", "Fi[i] = (1.0 - 1.0 / tau_f)",
     (U, "test_source_f_moments", (0,))),
    ("F_i: lambda n without c_s^2", "double ax = dtx + CS2 * lambda * nx;", "double ax = dtx + lambda * nx;",
     (U, "test_source_f_moments", (0,))),
    ("G_i without the Lambda term", "(cF / CS2 + drho * cu * cg / CS2)", "(cF / CS2)",
     (U, "test_force_g_moments_A2_and_eq18", (0,))),
    ("G_i without its prefactor", "Gi[i] = (1.0 - 1.0 / (2.0 * tau_g))", "Gi[i] = (1.0)",
     (U, "test_force_g_moments_A2_and_eq18", (0,))),
    ("Eq. 25 phases swapped",
     "return 1.0 / (phi * (1.0 / P->nu_l - 1.0 / P->nu_g) + 1.0 / P->nu_g);",
     "return 1.0 / (phi * (1.0 / P->nu_g - 1.0 / P->nu_l) + 1.0 / P->nu_l);",
     (U, "test_viscosity_modes_end_points", ())),
    ("Eq. 26 tie at phi = 1/2 to the gas", "double mu = (phi >= 0.5)", "double mu = (phi > 0.5)",
     (U, "test_viscosity_modes_end_points", ())),
    ("Eq. 26 without nu = mu / rho", "        return mu / rho;", "        return mu;",
     (U, "test_viscosity_modes_end_points", ())),
    ("Eq. 24 phases swapped", "return phi * (P->nu_l - P->nu_g) + P->nu_g; /* Eq. 24 */",
     "return phi * (P->nu_g - P->nu_l) + P->nu_l; /* Eq. 24 */", (U, "test_viscosity_modes_end_points", ())),
    ("wall ghost row mirrors row 1", "if (y < 0) y = 0;", "if (y < 0) y = 1;",
     (PH, "test_brute_force_numpy_transcription", (1, 0))),
    ("gradient without 1/c_s^2", "sx += WGT[i] * CX[i] * nb / CS2;", "sx += WGT[i] * CX[i] * nb;",
     (U, "test_stencils_exact_on_quadratics", ())),
    ("Laplacian without its 2", "sl += 2.0 * WGT[i] * (nb - c) / CS2;", "sl += WGT[i] * (nb - c) / CS2;",
     (U, "test_stencils_exact_on_quadratics", ())),
    ("open top copies its own row", "below = (size_t)(ny - 2) * nx + x;", "below = (size_t)(ny - 1) * nx + x;",
     (PH, "test_open_top_half_poiseuille_first_order", ())),
    ("rho from rho_l, not the jump", "double rho = phi * drho + P->rho_g;",
     "double rho = phi * P->rho_l + P->rho_g;", (PH, "test_drop_translates_with_uniform_flow", ())),
    ("beta halved", "double beta = 12.0 * P->sigma", "double beta = 6.0 * P->sigma",
     (PH, "test_planar_interface_at_rest_stays_put", (64, 1000.0))),
    ("k = sigma W", "double k = 1.5 * P->sigma", "double k = 1.0 * P->sigma",
     (PH, "test_planar_interface_at_rest_stays_put", (64, 1000.0))),
    ("mu_phi: sign of k lap phi", "- k * L->lap[n]; /* Eq. 6 */", "+ k * L->lap[n]; /* Eq. 6 */",
     (PH, "test_planar_interface_at_rest_stays_put", (63, 1000.0))),
    ("u without F/2", "double ux = (mx + 0.5 * Fx) / rho;", "double ux = mx / rho;",
     (PH, "test_uniform_body_force_closed_form", ())),
    ("p without c_s^2 / (1 - w_0)", "double p = CS2 / (1.0 - WGT[0]) *", "double p = CS2 *",
     (PH, "test_uniform_state_is_a_fixed_point", ())),
    ("p: sign of the interface term", "sum_nz + 0.5 * drho", "sum_nz - 0.5 * drho",
     (PH, "test_planar_interface_at_rest_stays_put", (64, 10.0))),
    ("p without rho s_0", "+ rho * s0); /* Eq. 22b */", "+ s0); /* Eq. 22b */",
     (PH, "test_uniform_state_is_a_fixed_point", ())),
    ("tau_g = 3 nu + 0.6", "double tau_g = nu / CS2 + 0.5;", "double tau_g = nu / CS2 + 0.6;",
     (PH, "test_shear_wave_decay_matches_viscosity", (0, 0.3))),
    ("lambda = 2 phi (1 - phi) / W", "double lambda = 4.0 * phi", "double lambda = 2.0 * phi",
     (PH, "test_planar_interface_at_rest_stays_put", (64, 1000.0))),
    ("central normal reversed", "*nx_o = gx / mag;\n            *ny_o = gy / mag;",
     "*nx_o = -gx / mag;\n            *ny_o = -gy / mag;", (PH, "test_drop_translates_with_uniform_flow", ())),
    ("Eq. 29 normal reversed", "*nx_o = -Cx / mag;\n        *ny_o = -Cy / mag;",
     "*nx_o = Cx / mag;\n        *ny_o = Cy / mag;", (PH, "test_brute_force_numpy_transcription", (0, 1))),
    ("Eq. 29 without d_t(phi u) / 2", "double Cx = 0.5 * dtx, Cy = 0.5 * dty;",
     "double Cx = 0.0 * dtx, Cy = 0.0 * dty;", (PH, "test_brute_force_numpy_transcription", (0, 1))),
    ("d_t(phi u) dropped", "double dtx = phi * ux - L->phiu_x[n];", "double dtx = 0.0;",
     (PH, "test_brute_force_numpy_transcription", (0, 0))),
    ("phi u history never updated",
     "            L->phiu_x[n] = phi * ux;\n            L->phiu_y[n] = phi * uy;\n        }", "        }",
     (PH, "test_drop_translates_with_uniform_flow", ())),
    ("phi u history starts at 0",
     "        L->phiu_x[n] = phi * ux;\n        L->phiu_y[n] = phi * uy;\n    }\n"
     "    if (P->bc_y == 2) open_top_fill(L->f",
     "        L->phiu_x[n] = 0.0;\n        L->phiu_y[n] = phi * uy;\n    }\n"
     "    if (P->bc_y == 2) open_top_fill(L->f", (PH, "test_brute_force_numpy_transcription", (0, 0))),
    ("bounce-back keeps the direction", "                    id = opposite(i);", "                    id = i;",
     (PH, "test_phi_is_conserved", (1,))),
    ("streaming reversed in x", "int xd = ((x + CX[i]) % nx + nx) % nx;", "int xd = ((x - CX[i]) % nx + nx) % nx;",
     (PH, "test_drop_translates_with_uniform_flow", ())),
    ("phi without f_0", "for (int i = 0; i < 9; ++i) s += L->f[i * N + n];\n        L->phi[n] = s;",
     "for (int i = 1; i < 9; ++i) s += L->f[i * N + n];\n        L->phi[n] = s;",
     (PH, "test_phi_is_conserved", (0,))),
    ("open top reflects instead of losing", "continue; /* leaves through the open top */",
     "{ yd = ny - 1; } /* leaves through the open top */", (PH, "test_open_top_half_poiseuille_first_order", ())),
    ("f relaxes with tau_f + 0.1", "double fpost = fpre[i] - (fpre[i] - feq[i]) / tau_f + Fi[i];",
     "double fpost = fpre[i] - (fpre[i] - feq[i]) / (tau_f + 0.1) + Fi[i];",
     (PH, "test_planar_interface_at_rest_stays_put", (64, 1000.0))),
]

_CHILD = """
import sys
sys.path.insert(0, {root!r})
import oracle
oracle._SRC, oracle._BUILD, oracle._LIB_PATH = {src!r}, {d!r}, {lib!r}
oracle.set_threads(1)
import importlib
pin = getattr(importlib.import_module({mod!r}), {fn!r})
try:
    pin(*{args!r})
except AssertionError:
    sys.exit(3)
sys.exit(0)
"""


def _run(k, m, base, text):
    """Build the oracle with mistake m and call its pin in a fresh process;
    returns (name, exit code) -- 0 when the pin passed -- or (name, None)
    when the mutant does not build."""
    name, old, new, (mod, fn, args) = m
    d = os.path.join(base, f"m{k:02d}")
    os.makedirs(d)
    src = os.path.join(d, "lbm_oracle.c")
    with open(src, "w") as fh:
        fh.write(text.replace(old, new))
    lib = os.path.join(d, "liblbm_oracle.so")
    built = subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                            "-shared", "-o", lib, src, "-lm"], capture_output=True, text=True)
    if built.returncode:
        return name, None
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT, src=src, d=d, lib=lib, mod=mod,
                                                            fn=fn, args=args)],
                       capture_output=True, text=True, cwd=ROOT, timeout=300)
    return name, r.returncode


def test_every_planted_mistake_fails_its_pin(tmp_path):
    text = open(SRC).read()
    for m in MUTANTS:
        assert text.count(m[1]) == 1, f"{m[0]}: original text not found once"
    assert len({m[0] for m in MUTANTS}) == len(MUTANTS)
    # controls: the unmodified source through the same build-and-call path
    # must pass its pins, so a broken harness cannot pass for a caught mutant
    controls = [("control " + m[0], m[1], m[1], m[3]) for m in MUTANTS[:3]]
    jobs = list(enumerate(controls + MUTANTS))
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(lambda km: _run(km[0], km[1], str(tmp_path), text), jobs))
    ctl, mut = res[:len(controls)], res[len(controls):]
    assert all(rc == 0 for _, rc in ctl), ctl
    unbuilt = [name for name, rc in mut if rc is None]
    missed = [name for name, rc in mut if rc == 0]
    assert not unbuilt and not missed, {"do not build": unbuilt, "not caught": missed}
    # the pins fail by assertion (exit 3), not by crashing
    crashed = {name: rc for name, rc in mut if rc not in (0, 3, None)}
    assert not crashed, crashed


@pytest.mark.parametrize("mod,fn,args", sorted({m[3] for m in MUTANTS}))
def test_named_pins_pass_on_the_oracle(mod, fn, args):
    """The same pins, called the same way, pass on the unmodified oracle."""
    import importlib

    getattr(importlib.import_module(mod), fn)(*args)
