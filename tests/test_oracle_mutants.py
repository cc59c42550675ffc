"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/oracle.c (a dropped term, a wrong sign, a wrong
index or operand), compiles the copy on the CPU and runs the whole pin suite
(test_oracle_build.py, test_oracle_solve.py, test_oracle_e.py, test_oracle_resume.py,
test_oracle_refresh.py) against it.
Every mutant must fail at least one pin.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    # loop node transit: wrong sign in out/(out - d)
    "loop_transit_sign": ("F[i] * (double)o / ((double)o - d)", "F[i] * (double)o / ((double)o + d)"),
    # loop node transit dropped (treated as a plain node)
    "loop_transit_dropped": ("double transit = loop[i] ?", "double transit = 0 ?"),
    # push also to the node itself
    "push_to_self": ("if (col_out[k] != i) F[col_out[k]] += sent;", "F[col_out[k]] += sent;"),
    # sent divided by out + 1
    "sent_divisor": ("double sent = transit * d / (double)o;", "double sent = transit * d / (double)(o + 1);"),
    # damping factor dropped from the push
    "sent_no_d": ("double sent = transit * d / (double)o;", "double sent = transit / (double)o;"),
    # fluid not cleared after the visit
    "fluid_kept": ("    F[i] = 0.0;\n    if (o == 0)", "    if (o == 0)"),
    # dangling mass e never accumulated
    "e_dropped": ("info->e += transit;", "info->e += 0.0;"),
    # DI-SOP threshold without the out-degree factor
    "sop_no_out": ("if (fabs(F[i]) > (r_cycle / (double)L) * out_i)", "if (fabs(F[i]) > (r_cycle / (double)L))"),
    # DI-SOP tie fallback missing (stalls, then stops on the cycle cap)
    "sop_no_fallback": ("if (info->visits == visits_before) {", "if (0) {"),
    # PI divides by the in-degree of the neighbour
    "pi_indeg": ("acc += d * X[j] / (double)outdeg[j];", "acc += d * X[j] / (double)(rp_in[j + 1] - rp_in[j]);"),
    # PI forgets B
    "pi_no_B": ("double acc = B[i];\n            for (int64_t k = rp_in[i]; k < rp_in[i + 1]; k++) {\n                int32_t j = col_in[k];\n                acc += d * X[j]",
                "double acc = 0.0;\n            for (int64_t k = rp_in[i]; k < rp_in[i + 1]; k++) {\n                int32_t j = col_in[k];\n                acc += d * X[j]"),
    # duplicates kept
    "no_dedupe": ("if (k > 0 && tmp[b + k] == tmp[b + k - 1]) continue;", ""),
    # in-CSR stores destinations instead of origins
    "in_csr_transposed": ("col_in[cur[col_out[k]]++] = (int32_t)v;", "col_in[cur[col_out[k]]++] = col_out[k];"),
    # loop flag never set
    "loop_flag_missing": ("if (col_out[k] == v) loop[v] = 1;", ""),
    # peeling level not 1 + max
    "level_off_by_one": ("if (level[u] + 1 > level[w] && !e_mask[w]) level[w] = level[u] + 1;",
                         "if (level[u] > level[w] && !e_mask[w]) level[w] = level[u];"),
    # peeling starts from in-degree <= 1
    "peel_start": ("if (indeg[v] == 0) { queue[tail++]", "if (indeg[v] <= 1) { queue[tail++]"),
    # residual with the wrong sign of H
    "residual_sign": ("Fstar[i] = acc - H[i];", "Fstar[i] = acc + H[i];"),
    # PI' skips the self-link (treats a loop like the D-iteration's closed form)
    "pi_push_skips_loop": ("for (int64_t k = rp_out[i]; k < rp_out[i + 1]; k++) Xn[col_out[k]] += transit;",
                           "for (int64_t k = rp_out[i]; k < rp_out[i + 1]; k++) if (col_out[k] != i) Xn[col_out[k]] += transit;"),
    # PI' divides by out + 1
    "pi_push_divisor": ("double transit = d * X[i] / (double)o;", "double transit = d * X[i] / (double)(o + 1);"),
    # resumed run ignores the given history
    "resume_drops_H0": ("for (int64_t i = 0; i < n; i++) { H[i] = H0[i]; F[i] = F0[i]; }",
                        "for (int64_t i = 0; i < n; i++) { H[i] = 0.0; F[i] = F0[i]; }"),
    # DI-CYC visits only positive fluid (a signed resumed state never drains)
    "cyc_positive_only": ("        } else {\n            for (int64_t i = 0; i < n; i++)\n                if (F[i] != 0.0)",
                          "        } else {\n            for (int64_t i = 0; i < n; i++)\n                if (F[i] > 0.0)"),
    # E pre-diffusion in id order, ignoring the levels
    "e_prepass_id_order": ("if (e_mask[i] && e_level[i] == l) {", "if (e_mask[i] && l == 0) {"),
    # E pre-diffusion skips the last level
    "e_prepass_short": ("for (int32_t l = 0; l < n_levels; l++)", "for (int32_t l = 0; l + 1 < n_levels; l++)"),
    # refreshed DI-SOP: r taken again one node late
    "refresh_late": ("if (r_every > 0 && i > 0 && i % r_every == 0) r_cycle = sum_fluid(n, F);",
                     "if (r_every > 0 && i > 1 && i % r_every == 1) r_cycle = sum_fluid(n, F);"),
    # refreshed DI-SOP: the refresh sums B instead of the current fluid (r never moves)
    "refresh_stale": ("if (r_every > 0 && i > 0 && i % r_every == 0) r_cycle = sum_fluid(n, F);",
                      "if (r_every > 0 && i > 0 && i % r_every == 0) r_cycle = r;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = text.replace(old, new)
    csrc = tmp_path / "oracle_mut.c"
    csrc.write_text(mutated)
    so = tmp_path / "oracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", str(so), str(csrc), "-lm"])
    env = dict(os.environ, DI_ORACLE_LIB=str(so))
    try:
        proc = subprocess.run(
            [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
             os.path.join(ROOT, "tests", "test_oracle_build.py"),
             os.path.join(ROOT, "tests", "test_oracle_solve.py"),
             os.path.join(ROOT, "tests", "test_oracle_e.py"),
             os.path.join(ROOT, "tests", "test_oracle_resume.py"),
             os.path.join(ROOT, "tests", "test_oracle_refresh.py")],
            cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    except subprocess.TimeoutExpired:
        return  # a mutant that no longer converges within the cycle cap is caught too
    assert proc.returncode != 0, f"mutant {name} passed every pin:\n{proc.stdout[-2000:]}"
