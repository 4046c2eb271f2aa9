"""Plants plausible mistakes in a scratch copy of the oracle (on the CPU)
and checks that the oracle pins catch every one of them."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "drop_delta_in_dm1": ("m[13 + 3 * a + g] += Vj * (x[a] * dW[g] + (a == g ? W : 0.0));",
                          "m[13 + 3 * a + g] += Vj * (x[a] * dW[g]);"),
    "drop_B_term_in_corrected_gradient": ("Ai * (dBx + Bi[g]) * W;", "Ai * (dBx) * W;"),
    "transposed_dB": ("double dBx = dBi[0 * 3 + g] * x[0] + dBi[1 * 3 + g] * x[1] + dBi[2 * 3 + g] * x[2];",
                      "double dBx = dBi[g * 3 + 0] * x[0] + dBi[g * 3 + 1] * x[1] + dBi[g * 3 + 2] * x[2];"),
    "dA_cross_term_factor": ("dA[3 * i + g] = -Ai * Ai * (dm0 + 2.0 * Bdm1 + BdmB);",
                             "dA[3 * i + g] = -Ai * Ai * (dm0 + 1.0 * Bdm1 + BdmB);"),
    "viscosity_of_j_uses_h_i": ("double Qj = orc_visc_Q(xji, vji, h[j], rho[j], c[j], p);",
                                "double Qj = orc_visc_Q(xji, vji, h[i], rho[j], c[j], p);"),
    "energy_rate_sign": ("du += -0.5 * (F[0]", "du += 0.5 * (F[0]"),
    "split_factor_sign": ("return erfc(t) + r / (sqrt(ORC_PI) * r_s) * exp(-t * t);",
                          "return erfc(t) - r / (sqrt(ORC_PI) * r_s) * exp(-t * t);"),
    "kernel_normalisation": ("double norm = 495.0 / (32.0 * ORC_PI * H * H * H);",
                             "double norm = 495.0 / (32.0 * ORC_PI * H * H * H) * 1.001;"),
    "non_strict_predicate": ("return r2 < H * H;", "return r2 <= H * H;"),
    "m2_packing_index": ("static const int ORC_SYM_B[6] = {0, 1, 2, 1, 2, 2};",
                         "static const int ORC_SYM_B[6] = {0, 1, 2, 1, 1, 2};"),
    "gravity_drops_softening": ("double s2 = r2 + e2;", "double s2 = r2;"),
    "viscosity_clamp_inverted": ("if (mu > 0.0) mu = 0.0;", "if (mu < 0.0) mu = 0.0;"),
    "viscosity_linear_term_sign": ("return rho * (-p->av_alpha * c * mu + p->av_beta * mu * mu);",
                                   "return rho * (p->av_alpha * c * mu + p->av_beta * mu * mu);"),
    # the friends-of-friends labels, caught by their own pins
    "fof_non_strict_link": ("if (!(orc_sep(pos, i, j, L, dx) < b2)) continue;",
                            "if (!(orc_sep(pos, i, j, L, dx) <= b2)) continue;", "tests/test_oracle_fof.py"),
    "fof_ignores_species_of_j": ("if (j <= i || !((species_mask >> species[j]) & 1)) continue;",
                                 "if (j <= i) continue;", "tests/test_oracle_fof.py"),
    "fof_labels_by_largest_root": ("if (ri < rj) par[rj] = ri;\n                else par[ri] = rj;",
                                   "if (ri < rj) par[ri] = rj;\n                else par[rj] = ri;",
                                   "tests/test_oracle_fof.py"),
    "kdk_half_drift": ("pos[i] = orc_wrap_pos(pos[i] + dt * vel[i], p->L);",
                       "pos[i] = orc_wrap_pos(pos[i] + hdt * vel[i], p->L);"),
    "kdk_predictor_drops_half_kick": ("for (int64_t i = 0; i < 3 * n; ++i) vp[i] = vel[i] + hdt * acc[i];",
                                      "for (int64_t i = 0; i < 3 * n; ++i) vp[i] = vel[i];"),
    "kdk_energy_predictor_drops_half_kick": ("for (int64_t i = 0; i < n; ++i) up[i] = u[i] + hdt * dudt[i];",
                                             "for (int64_t i = 0; i < n; ++i) up[i] = u[i];"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, name):
    before, after, *pins = MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "crk_oracle.c")).read()
    assert src.count(before) == 1, name
    work = tmp_path / "tree"
    shutil.copytree(os.path.join(ROOT, "oracle"), work / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), work / "tests",
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(work / "paper_2510_03557_gb300")
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_2510_03557_gb300", f), work / "paper_2510_03557_gb300" / f)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), work / "pytest.ini")
    (work / "oracle" / "crk_oracle.c").write_text(src.replace(before, after))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:randomly",
                        pins[0] if pins else "tests/test_oracle_pins.py"], cwd=work, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 1, f"mutation {name} survived:\n{r.stdout[-2000:]}"


# Mistakes planted in the numpy parts of the oracle, each caught by that
# module's own pins.
PY_MUTATIONS = {
    "pm_filter_half_width": ("pm.py", "np.exp(-k2 * r_s * r_s)", "np.exp(-0.5 * k2 * r_s * r_s)"),
    "pm_one_window_undone": ("pm.py", "/ (k2 * C * C)", "/ (k2 * C)"),
    "pm_cells_at_corners": ("pm.py", "s = pos / d - 0.5", "s = pos / d"),
    "pm_gradient_sign": ("pm.py", "-1j * kd * phi", "1j * kd * phi"),
    "bins_predictor_as_if_step_ended": ("bins.py", "tau = (2 * (s + 1 - s0) - Lb) * (0.5 * d)",
                                        "tau = Lb * (0.5 * d)"),
    "bins_ignore_sync": ("bins.py", "return np.maximum(b, b_sync)", "return b"),
    "bins_close_every_particle": ("bins.py", "vel = np.where(active[:, None], vel + hdt[:, None] * acc, vel)",
                                  "vel = vel + hdt[:, None] * acc"),
    "bins_courant_on_c_squared": ("bins.py", "dc = np.where(hot, (courant * h) / c, np.inf)",
                                  "dc = np.where(hot, (courant * h) / (c * c), np.inf)"),
    "bins_mesh_opening_full_kick": ("bins.py", "            vel = vel + (0.5 * dt_long) * mesh(pos)\n        for s",
                                    "            vel = vel + dt_long * mesh(pos)\n        for s"),
}
PY_PINS = {"pm.py": "tests/test_oracle_pm.py", "bins.py": "tests/test_oracle_bins.py"}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_pins_catch_planted_mistake_in_numpy_oracle(tmp_path, name):
    fname, before, after = PY_MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    assert src.count(before) == 1, name
    work = tmp_path / "tree"
    shutil.copytree(os.path.join(ROOT, "oracle"), work / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), work / "tests",
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(work / "paper_2510_03557_gb300")
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_2510_03557_gb300", f), work / "paper_2510_03557_gb300" / f)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), work / "pytest.ini")
    (work / "oracle" / fname).write_text(src.replace(before, after))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:randomly", PY_PINS[fname]],
                       cwd=work, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"mutation {name} survived:\n{r.stdout[-2000:]}"
