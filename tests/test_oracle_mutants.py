"""Each plausible mistake planted in a copy of the oracle must make some pin fail.

The copies are built on the CPU from textual edits of ``oracle/sf_oracle.c`` and the
pin suite is run against each one in a child process (``SF_ORACLE_LIB``).
"""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sf_oracle.c")

# name -> (original text, planted mistake)
MUTANTS = {
    "slack_sign_as_printed": ("double s = h - B->q[o];", "double s = -B->q[o] - h;"),
    "slack_not_clamped": ("s = s > 0.0 ? s : 0.0;", ";"),
    "obstacle_centre_dropped": ("double e = ev[ax] + (po ? po[ax] : 0.0);", "double e = ev[ax];"),
    "obstacle_radius_is_robot": ("double A = m >= 0 ? P->obs_ab[2 * m] : P->a;", "double A = P->a;"),
    "lambda_step_sign": ("lam[(size_t)ax * N + u] - P->rho * g[u]", "lam[(size_t)ax * N + u] + P->rho * g[u]"),
    "workspace_term_dropped_from_eta": ("GT_apply(P, C, hs, fe);", ";"),
    "alpha_arguments_swapped": ("double alpha = atan2(dy, dx);", "double alpha = atan2(dx, dy);"),
    "beta_arguments_swapped": ("double beta = atan2(u1, u2);", "double beta = atan2(u2, u1);"),
    "d_clamp_dropped": ("double d = t > 1.0 ? t : 1.0;", "double d = t;"),
    "pair_row_sign_in_FT": ("if (bj >= 0) out[bj * P->nxi + c] -= ", "if (bj >= 0) out[bj * P->nxi + c] += "),
    "basis_time_grid_off_by_one": ("double tau = (double)k / (double)(H - 1);", "double tau = (double)k / (double)H;"),
    "lower_box_row_sign": ("q[nH + i * P->H + k] = -s;", "q[nH + i * P->H + k] = s;"),
    "schur_correction_sign": ("x[v] -= s;", "x[v] += s;"),
    "adjoint_eta_not_in_lambda": ("lt[(size_t)ax * N + u] = lb[(size_t)ax * N + u] + etab[(size_t)ax * N + u];",
                                  "lt[(size_t)ax * N + u] = lb[(size_t)ax * N + u];"),
    "adjoint_jacobian_transposed": ("s += J[rr * nd + q] * eb[(size_t)rr * RF + r];",
                                    "s += J[q * nd + rr] * eb[(size_t)rr * RF + r];"),
    "adjoint_slack_gate_inverted": ("qbx[gq] = r2b - sb * act;", "qbx[gq] = r2b - sb * (1.0 - act);"),
    "smooth_eta_keeps_candidate": ("eta[u] = (P->cost == 0 ? P->xi[(size_t)ax * N + u] : 0.0) + lam_new",
                                   "eta[u] = P->xi[(size_t)ax * N + u] + lam_new"),
    "smooth_time_scale_not_squared": ("/ (T * T);", "/ T;"),
    "adjoint_smooth_candidate_gradient": ("if (P.cost == 0) gx[(size_t)ax * N + u] += etab", "gx[(size_t)ax * N + u] += etab"),
    "velocity_basis_difference_sign": ("double w = j == c - 1 ? 1.0 : -1.0;", "double w = j == c - 1 ? -1.0 : 1.0;"),
    "velocity_time_scale_dropped": ("Wd[k * nxi + c] = (double)deg * v / T;", "Wd[k * nxi + c] = (double)deg * v;"),
    "velocity_row_is_goal_derivative": ("memcpy(C->Wd0, Wd, sizeof(double) * nxi);",
                                        "memcpy(C->Wd0, Wd + (size_t)(H - 1) * nxi, sizeof(double) * nxi);"),
    "fp_seed_sign_on_later_iterate": ("xb[u] += 2.0 * g_fp", "xb[u] -= 2.0 * g_fp"),
    "fp_seed_lambda_dropped": ("lb[u] += 2.0 * g_fp * (Lm[NN * (it + 1) + u] - Lm[NN * it + u]);", ";"),
    "fp_seed_earlier_iterate_dropped": ("xb[u] -= 2.0 * g_fp * (X[NN * (it + 1) + u] - X[NN * it + u]);", ";"),
}


def _run(name, tmp):
    orig, bad = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(orig) == 1, name
    msrc = os.path.join(tmp, name + ".c")
    with open(msrc, "w") as f:
        f.write(src.replace(orig, bad))
    lib = os.path.join(tmp, name + ".so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-o", lib, msrc, "-lm"])
    env = dict(os.environ, SF_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], env=env, capture_output=True, text=True,
                       timeout=600)
    return r.returncode, r.stdout[-400:]


def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
            results = dict(zip(MUTANTS, ex.map(lambda n: _run(n, tmp), MUTANTS)))
    survivors = {k: v[1] for k, v in results.items() if v[0] == 0}
    assert not survivors, "mutants passed every pin: %s" % list(survivors)
