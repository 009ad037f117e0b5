"""Planted mistakes in the FP64 oracle must each fail at least one pin.

Each mutant below changes one expression of ``oracle/dscreen_oracle.c`` into a
plausible mistake (a flipped sign, a dropped term, a wrong index or constant).
The mutated copy is compiled into a temporary directory and the pins of
``test_oracle_pins.py`` run against it in a child process; the mutant counts
as caught only when a pin fails (pytest exit code 1), not when the harness
breaks.  The unmutated source runs through the same harness as a control.
The oracle itself is never modified.  CPU only.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dscreen_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# name -> (exact text in the oracle, replacement, the passage it breaks)
MUTANTS = {
    "dst3_centre_sign": ("cvec[n] -= psi / ns2 * sg * ds[n];", "cvec[n] += psi / ns2 * sg * ds[n];",
                         "Lemma 3 centre"),
    "dst3_radius_unsquared": ("R2 - c->delta * c->delta", "R2 - c->delta", "Lemma 3 radius"),
    "dome_dropped_psi_t": ("return dc0 - psi * t + sqrt(", "return dc0 + sqrt(", "Lemma 4 maximum"),
    "dome_branch_sign": ("if (t * R <= -psi) return dc0 + R;", "if (t * R <= psi) return dc0 + R;",
                         "Lemma 4 case split"),
    "dome_normal_unsigned": ("c->tdome[i] = sg * vec_dot(", "c->tdome[i] = vec_dot(", "Lemma 4 normal d_*"),
    "safe_norm_dropped": ("(1.0 - fabs(c->dtc[g])) / c->nrm[g] - rad", "(1.0 - fabs(c->dtc[g])) - rad",
                          "Lemma 2 for unnormalised atoms"),
    "gsafe_weight_dropped": ("(g_w(c->w, g) - c->dtc[g]) / c->nrm[g]", "(1.0 - c->dtc[g]) / c->nrm[g]",
                             "Lemma 5 weight"),
    "dgst3_offset_unsquared": ("/ lam - wg * wg;", "/ lam - wg;", "Lemma 6 hyperplane offset"),
    "dgst3_centre_sign": ("cvec[n] -= coef * nv[n] / nn;", "cvec[n] += coef * nv[n] / nn;", "Lemma 6 centre"),
    "mu_unclipped": ("if (m > 0.0) {", "if (0) {", "Lemma 8 clip"),
    "mu_lambda_dropped": ("vec_dot(theta, y, N) / (lambda * tt)", "vec_dot(theta, y, N) / tt",
                          "Lemma 8 scaling"),
    "fista_momentum": ("beta = (l - 1.0) / ln;", "beta = l / ln;", "Table 1 FISTA momentum"),
    "momentum_direction": ("u[i] = xi + beta * (xi - x[i]);", "u[i] = xi + beta * (x[i] - xi);",
                           "Table 1 extrapolation"),
    "soft_threshold_half": ("double a = fabs(v[lo]) - t;", "double a = fabs(v[lo]) - 0.5 * t;",
                            "eq. softTh"),
    "group_threshold_weight": ("(nv - t * g_w(c->w, g)) / nv", "(nv - t) / nv", "eq. gr_softTh weight"),
    "lambda_star_weight": ("double v = sqrt(s) / g_w(w, g);", "double v = sqrt(s);", "eq. gstar weight"),
    "power_method_sqrt": ("double rq_new = vec_dot(u, u, N);", "double rq_new = sqrt(vec_dot(u, u, N));",
                          "step constant ||D||^2"),
    "jacobi_rotation_sign": ("A[k * m + p] = c * akp - s * akq;", "A[k * m + p] = c * akp + s * akq;",
                             "||D_g||_2 for Lemmas 5-7"),
    "dual_lambda_unsquared": ("0.5 * yy - 0.5 * lambda * lambda * R * R", "0.5 * yy - 0.5 * lambda * R * R",
                              "dual objective of the gap"),
    "cp_dual_unaveraged": ("(theta[n] + sigma * r[n]) / (1.0 + sigma)", "(theta[n] + sigma * r[n])",
                           "Table 1 Chambolle-Pock dual step"),
    "dome_centre_norm_dropped": ("double dc0 = c->b[g] / (lam * ni);", "double dc0 = c->b[g] / lam;",
                                 "Lemma 4 for unnormalised atoms"),
    "dome_offset_norm_dropped": ("c->psi_dome = psi / sqrt(ns2);", "c->psi_dome = psi;",
                                 "Lemma 4 hyperplane distance"),
    "dome_cosine_norm_dropped": ("/ (ni * sqrt(ns2));", "/ sqrt(ns2);", "Lemma 4 angle to d_*"),
    "group_max_unweighted": ("            double val = sqrt(q) / g_w(w, g);\n            if (val > m) m = val;\n"
                             "            prox_group",
                             "            double val = sqrt(q);\n            if (val > m) m = val;\n            prox_group",
                             "Lemma 8 feasibility with weights"),
    "fista_gradient_step_from_x": ("v[i] = cp ? x[i] - tau * z[i] : u[i] - z[i] / L;",
                                   "v[i] = cp ? x[i] - tau * z[i] : x[i] - z[i] / L;", "Table 1 FISTA gradient point"),
    "fista_without_momentum": ("beta = (l - 1.0) / ln;", "beta = 0.0 * (l - 1.0) / ln;", "Table 1 FISTA momentum"),
    "step_constant_below_norm": ("* (1.0 + 1e-6);", "* (1.0 - 1e-3);", "L >= ||D||^2 behind Table 1"),
    "screened_atoms_rescreened": ("        if (!active_g[g]) continue;\n        double margin;", "        double margin;",
                                  "Algorithm 3 screens each atom once"),
    "warm_start_u_unset": ("{ x[i] = x0[i]; u[i] = x0[i]; }", "{ x[i] = x0[i]; }", "warm start x_0 = u_0"),
    "gap_at_extrapolated_point": ("            if (x[i] != 0.0)\n                for (int64_t n = 0; n < N; n++) r[n] += D[i * ld + n] * x[i];",
                                  "            if (u[i] != 0.0)\n                for (int64_t n = 0; n < N; n++) r[n] += D[i * ld + n] * u[i];",
                                  "the gap certifies the returned iterate"),
    "history_counts_groups": ("if (act[g]) nact += (int)(g_hi(goff, g) - g_lo(goff, g));", "if (act[g]) nact += 1;",
                              "|A_t| of the flops accounting counts atoms"),
    "history_nonzeros_of_u": ("record_iteration(goff, G, K, act, x, R, rad, gap, mu, hist ? hist +",
                              "record_iteration(goff, G, K, act, u, R, rad, gap, mu, hist ? hist +",
                              "||x_t||_0 of the flops accounting"),
    "cp_average_with_tau": ("(theta[n] + sigma * r[n]) / (1.0 + sigma)", "(theta[n] + sigma * r[n]) / (1.0 + tau)",
                            "Table 1 Chambolle-Pock dual step"),
    "cp_dual_step_tau": ("(theta[n] + sigma * r[n]) / (1.0 + sigma)", "(theta[n] + tau * r[n]) / (1.0 + sigma)",
                         "Table 1 Chambolle-Pock dual step"),
    "cp_primal_step_sigma": ("v[i] = cp ? x[i] - tau * z[i] : u[i] - z[i] / L;",
                             "v[i] = cp ? x[i] - sigma * z[i] : u[i] - z[i] / L;", "Table 1 Chambolle-Pock primal step"),
    "cp_threshold_sigma": ("cp ? lambda * tau : lambda / L", "cp ? lambda * sigma : lambda / L",
                           "Table 1 Chambolle-Pock proximal threshold"),
    "cp_extrapolation_dropped": ("            beta = phi;\n", "            beta = 0.0 * phi;\n",
                                 "Table 1 Chambolle-Pock extrapolation (Arrow-Hurwicz without it)"),
    "sparsa_bb_inverted": ("alpha = ds2 / dx2;", "alpha = dx2 / ds2;", "SpaRSA's Barzilai-Borwein step"),
    "sparsa_first_step_unit": ("    double alpha = L;\n", "    double alpha = 1.0;\n", "SpaRSA's first step (ISTA's)"),
    "sparsa_acceptance_loosened": ("ok = F <= Fmax - 0.5 * OR_SPARSA_SIGMA * Lt * dx2;",
                                   "ok = F <= Fmax + 0.5 * OR_SPARSA_SIGMA * Lt * dx2 + 1e-3 * Fmax;",
                                   "SpaRSA's nonmonotone acceptance"),
    "twist_b_formula": ("tb = 2.0 * ta / (1.0 + xi1);", "tb = ta / (1.0 + xi1);", "TwIST's beta"),
    "twist_monotone_reversed": ("ok = it == 1 || fallback || F <= Fprev;", "ok = it == 1 || fallback || F >= Fprev;",
                                "TwIST's monotone safeguard"),
    "twist_first_step_two_step": ("if (twist && it >= 2 && !fallback)", "if (twist && it >= 1 && !fallback)",
                                  "TwIST's first (shrinkage) step"),
    "backtracking_model_halved": ("ok = dq <= Lt * sq;", "ok = dq <= 2.0 * Lt * sq;", "Beck-Teboulle's upper model"),
    "backtracking_no_growth": ("            else Lt *= OR_ETA;\n", "            else Lt *= 1.0;\n",
                               "backtracking's growth of L"),
    "cp_tau_schedule_inverted": ("tau *= phi;", "tau /= phi;", "Table 1 Chambolle-Pock step schedule (gamma > 0)"),
    "cp_sigma_schedule_inverted": ("sigma /= phi;", "sigma *= phi;", "Table 1 Chambolle-Pock step schedule (gamma > 0)"),
    "fista_sequence_other_constant": ("sqrt(1.0 + 4.0 * l * l)", "sqrt(1.0 + 2.0 * l * l)", "Table 1 FISTA l_t"),
    "fista_sequence_linear": ("double ln = 0.5 * (1.0 + sqrt(1.0 + 4.0 * l * l));", "double ln = l + 1.0 / 3.0;",
                              "Table 1 FISTA l_t"),
    "cp_dual_start_minus_y": ("        for (int64_t n = 0; n < N; n++) theta[n] = 0.0;\n    res->status = 1;",
                              "        for (int64_t n = 0; n < N; n++) theta[n] = -y[n];\n    res->status = 1;",
                              "the reading theta_0 = 0 of Table 1 Chambolle-Pock"),
    "cp_extrapolation_halved": ("            beta = phi;\n", "            beta = 0.5 * phi;\n",
                                "Table 1 Chambolle-Pock extrapolation factor"),
    "cp_default_steps_smaller": ("double tau = opt->cp_tau > 0 ? opt->cp_tau : 0.99 / sqrt(L);",
                                 "double tau = opt->cp_tau > 0 ? opt->cp_tau : 0.5 / sqrt(L);",
                                 "the reading tau_0 = sigma_0 = 0.99 / sqrt(L)"),
    "margin_log_scaled_by_norm": ("if (marg) marg[g] = margin;", "if (marg) marg[g] = margin * c->nrm[g];",
                                  "logged test margins (Lemmas 2, 4 for unnormalised atoms)"),
    "dome_margin_smaller_maximum": ("margin = 1.0 / ni - (up > lo ? up : lo);", "margin = 1.0 / ni - (up < lo ? up : lo);",
                                    "Lemma 4: both signs of d_i^T theta"),
    "sequential_scaling_underestimated": ("                double z = col_dot(D, ld, i, theta, N);\n                q += z * z;",
                                          "                double z = col_dot(D, ld, i, theta, N);\n                q += 0.25 * z * z;",
                                          "Lemma 8 feasibility of the sequential dual point"),

}

# Mistakes that no pin catches, each with the reason; they run as strict xfails,
# so a pin that starts to catch one turns its entry into a failure to update.
KNOWN_SURVIVORS = {}

_CHILD = (
    "import sys\n"
    "sys.path.insert(0, {root!r})\n"
    "import oracle\n"
    "oracle._SRC, oracle._BUILD, oracle._LIB = {src!r}, {bdir!r}, {lib!r}\n"
    "import pytest\n"
    "sys.exit(pytest.main([{pins!r}, '-x', '-q', '-p', 'no:cacheprovider']))\n"
)


def _run_pins(name, text, workdir):
    """Compile ``text`` as the oracle and run the pins on it; returns (exit code, output tail)."""
    bdir = os.path.join(workdir, name)
    os.makedirs(bdir)
    src = os.path.join(bdir, "dscreen_oracle.c")
    lib = os.path.join(bdir, "liboracle.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", lib, src, "-lm"])
    code = _CHILD.format(root=ROOT, src=src, bdir=bdir, lib=lib, pins=PINS)
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    return p.returncode, (p.stdout + p.stderr)[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    with open(SRC) as f:
        base = f.read()
    jobs = {"unmutated": base}
    for name, (old, new, _) in {**MUTANTS, **KNOWN_SURVIVORS}.items():
        assert base.count(old) == 1, f"{name}: the mutated text must occur exactly once in the oracle"
        jobs[name] = base.replace(old, new)
    workdir = str(tmp_path_factory.mktemp("mutants"))
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_run_pins, name, text, workdir) for name, text in jobs.items()}
        return {name: f.result() for name, f in futs.items()}


def test_unmutated_oracle_passes_the_harness(outcomes):
    rc, tail = outcomes["unmutated"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, tail = outcomes[name]
    assert rc == 1, f"{name} ({MUTANTS[name][2]}): pins exit code {rc}, expected a failing pin\n{tail}"


@pytest.mark.parametrize("name", [pytest.param(n, marks=pytest.mark.xfail(strict=True, reason=KNOWN_SURVIVORS[n][2]))
                                  for n in sorted(KNOWN_SURVIVORS)])
def test_known_survivor_is_still_unpinned(outcomes, name):
    rc, tail = outcomes[name]
    assert rc == 1, f"{name}: pins exit code {rc}\n{tail}"
