"""Each plausible mistake planted in a copy of the oracle must fail a pin.

A mutant is oracle.c with one line changed (a dropped term, a transposed
operand, a wrong index or scale).  The pin suite runs against the mutant
build in a subprocess (ORACLE_SO) and must fail.  The real oracle.c is never
modified.
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "power_drops_dangling_term": (
        "double gamma = c * dangling_mass + (1.0 - c) * total_mass;",
        "double gamma = (1.0 - c) * total_mass;"),
    "power_transposed_edge": (
        "next[out_dst[e]] += c * pi[i] / (double)deg;",
        "next[i] += c * pi[out_dst[e]] / (double)deg;"),
    "dense_transposed_operand": (
        "M[(size_t)out_dst[e] * N + (size_t)j] -= c / (double)deg;",
        "M[(size_t)j * N + (size_t)out_dst[e]] -= c / (double)deg;"),
    "dense_uniform_teleport_for_dangling": (
        "M[(size_t)i * N + (size_t)j] -= c * p[i];",
        "M[(size_t)i * N + (size_t)j] -= c / (double)n;"),
    "sequential_reserves_1_minus_c": (
        "pibar[i] += v;",
        "pibar[i] += (1.0 - c) * v;"),
    "sequential_phase2_drops_h": (
        "pibar[d] = h[d];",
        "pibar[d] = 0.0;"),
    "rounds_ifp2_keeps_invalid_edges": (
        "                if (algo == ORC_IFP2 && outdeg(out_off, j) == 0) continue;\n                r[j]",
        "                r[j]"),
    "rounds_ifp1_finalise_unscaled": (
        "pi[i] = x[i] + (1.0 - c) * r[i];",
        "pi[i] = x[i] + r[i];"),
    "rounds_phase2_missing_reserve_scale": (
        "s += c * x[u] / ((1.0 - c) * (double)outdeg(out_off, u));",
        "s += c * x[u] / (double)outdeg(out_off, u);"),
    "rounds_stop_counts_dangling": (
        "if (outdeg(out_off, i) > 0) R += fabs(r[i]);",
        "R += fabs(r[i]);"),
    "rounds_pushes_from_current_not_snapshot": (
        "r[j] += c * v[i] / (double)deg;",
        "r[j] += c * r[i] / (double)deg;"),
    "residual_wrong_sign": (
        "y[out_dst[e]] -= c * pi[i] / (double)deg;",
        "y[out_dst[e]] += c * pi[i] / (double)deg;"),
    "levels_scanned_in_reverse": (
        "for (int32_t l = 0; l <= L; l++) {",
        "for (int32_t l = L; l >= 0; l--) {"),
    "levels_push_into_dangling": (
        "if (outdeg(out_off, k) == 0) continue;",
        ";"),
    "levels_residual_without_pending": (
        "if (outdeg(out_off, i) > 0) R += fabs(r[i]) + fabs(pend[i]);",
        "if (outdeg(out_off, i) > 0) R += fabs(r[i]);"),
    "async_reserve_unscaled": (
        "x[i] += (1.0 - c) * v;",
        "x[i] += v;"),
    "async_residual_kept_after_push": (
        "r[i] -= v;       /* i hands all of it on: r_i becomes 0 */",
        "/* residual kept */"),
    "async_frontier_includes_dangling": (
        "in_f[i] = outdeg(out_off, i) > 0 && fabs(r[i]) > xi_act;",
        "in_f[i] = fabs(r[i]) > xi_act;"),
    "async_scans_in_reverse_id_order": (
        "        for (int32_t i = 0; i < n; i++) {\n            if (!in_f[i]) continue;",
        "        for (int32_t i = n - 1; i >= 0; i--) {\n            if (!in_f[i]) continue;"),
    "scan_in_reverse_id_order": (
        "        for (int32_t i = 0; i < n; i++) {\n            int64_t deg = outdeg(out_off, i);\n            if (deg == 0) continue;\n            if (!(fabs(r[i]) > xi_act))",
        "        for (int32_t i = n - 1; i >= 0; i--) {\n            int64_t deg = outdeg(out_off, i);\n            if (deg == 0) continue;\n            if (!(fabs(r[i]) > xi_act))"),
    "scan_keeps_the_pushed_residual": (
        "            r[i] = 0.0;\n            x[i] = x[i] + (1.0 - c) * v;",
        "            x[i] = x[i] + (1.0 - c) * v;"),
    "scan_bound_without_pushes": (
        "            Rub += c * fabs(v) * (double)valid / (double)deg; /* may land after its target's turn */",
        "            (void)valid;"),
    "scan_reserve_unscaled": (
        "            x[i] = x[i] + (1.0 - c) * v;",
        "            x[i] = x[i] + v;"),
    "power_off_by_one_degree": (
        "next[out_dst[e]] += c * pi[i] / (double)deg;",
        "next[out_dst[e]] += c * pi[i] / (double)(deg + 1);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    before, after = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(before) == 1, f"mutation site for {name} not unique in oracle.c"
    src = tmp_path / "oracle_mutant.c"
    src.write_text(text.replace(before, after))
    so = oracle.compile_c(str(src), str(tmp_path / "oracle_mutant.so"))
    env = dict(os.environ, ORACLE_SO=so)
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"mutant {name} passed every pin:\n{res.stdout[-2000:]}"
