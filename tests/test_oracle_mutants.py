"""The oracle's pins are strong enough to catch plausible mistakes: each case below plants
one (a dropped term, a wrong sign, a wrong index or bound, a transposed operand, a skipped
step, an off-by-one in a rule, a wrong constant) in
a copy of the oracle's source, builds it with the oracle's own flags, and runs the CPU
pins against that library (through MSP_ORACLE_LIB in a child process); at least one pin
must fail.  The product oracle is never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "msp_oracle.cpp")
PINS = ["tests/test_oracle_amg.py", "tests/test_oracle_colouring.py",
        "tests/test_oracle_krylov.py", "tests/test_oracle_smoothers.py",
        "tests/test_oracle_wells.py", "tests/test_batch_cpu.py"]

# name: (exact source text, planted mistake)
MUTANTS = {
    "gauss_jordan_elimination_sign": (
        "a[r * b + k] = a[r * b + k] - f * a[c * b + k];",
        "a[r * b + k] = a[r * b + k] + f * a[c * b + k];"),
    "colouring_second_circle_ignored": (
        "int vi = !Wh.empty() ? Wh.begin()->second : Vq.begin()->second;",
        "int vi = Vq.begin()->second;"),
    "strength_of_connection_sign": (
        "s[p - S.rp[i]] = -0.5 * t;", "s[p - S.rp[i]] = 0.5 * t;"),
    "galerkin_term_dropped": (
        "it->second = it->second + a.v[p];", "it->second = it->second;"),
    "gauss_seidel_sign": (
        "          acc -= a.v[p] * x[j];\n      }\n      x[i] = acc / d;",
        "          acc += a.v[p] * x[j];\n      }\n      x[i] = acc / d;"),
    "bilu_operands_transposed": (
        "blk_mul(b, &h.lu[(size_t)p * bb], &h.u_inv[(size_t)k * bb], L.data());",
        "blk_mul(b, &h.u_inv[(size_t)k * bb], &h.lu[(size_t)p * bb], L.data());"),
    "stage_n_reads_the_pressure_slot": (
        "for (int k = 0; k < bn; ++k) acc[k] = r[(size_t)i * b + k + 1];",
        "for (int k = 0; k < bn; ++k) acc[k] = r[(size_t)i * b + k];"),
    "decoupled_restriction_terms_dropped": (
        "for (int k = 0; k < b; ++k) s = s + h.omega[(size_t)i * b + k] * r[(size_t)i * b + k];",
        "for (int k = 0; k < 1; ++k) s = s + h.omega[(size_t)i * b + k] * r[(size_t)i * b + k];"),
    "givens_sign": (
        "s[j + 1] = -sn[j] * s[j];", "s[j + 1] = sn[j] * s[j];"),
    "gram_schmidt_sign": (
        "V[j + 1][k] -= hij * V[i][k];", "V[j + 1][k] += hij * V[i][k];"),
    "schur_complement_sign": (
        "out[r * b + c] -= acc;", "out[r * b + c] += acc;"),
    "well_recovery_sign": (
        "        r[i] -= acc;\n", "        r[i] += acc;\n"),
    "adaptive_setup_rule_off_by_one": (
        "if (!h->first_solve && h->prev_it > h->cfg.mu) {",
        "if (!h->first_solve && h->prev_it >= h->cfg.mu) {"),
    "restriction_not_summed": (
        "for (int i = 0; i < n; ++i) bc[L.agg[i]] += r[i];  // restriction P^T r",
        "for (int i = 0; i < n; ++i) bc[L.agg[i]] = r[i];  // restriction P^T r"),
    "prolongation_dropped": (
        "for (int i = 0; i < n; ++i) x[i] += xc[L.agg[i]];  // prolongation by injection",
        "for (int i = 0; i < n; ++i) x[i] += 0.0 * xc[L.agg[i]];"),
    "bilu_backward_skips_the_upper_part": (
        "if (pos[j] > t) blk_gemv_sub(b, &h.lu[(size_t)p * bb], &x[(size_t)j * b], acc.data());",
        "if (pos[j] > t + nb) blk_gemv_sub(b, &h.lu[(size_t)p * bb], &x[(size_t)j * b], acc.data());"),
    "jp_priority_reversed": (
        "order[v] = {-(S.rp[v + 1] - S.rp[v]), (uint32_t)(splitmix64((uint64_t)v ^ kJpSeed) >> 32),",
        "order[v] = {(S.rp[v + 1] - S.rp[v]), (uint32_t)(splitmix64((uint64_t)v ^ kJpSeed) >> 32),"),
    "matching_threshold_strict": (
        "if (s[p - S.rp[i]] >= thr) {", "if (s[p - S.rp[i]] > thr) {"),
    "matching_visit_order_reversed": (
        "std::sort(order.begin(), order.end());\n  std::vector<int> partner(n, -1);",
        "std::sort(order.rbegin(), order.rend());\n  std::vector<int> partner(n, -1);"),
    "matching_tie_to_larger_index": (
        "(cand_s[p] == sbest && j < best)", "(cand_s[p] == sbest && j > best)"),
    "matching_row_only_strength": (
        "double t = entry(a, i, j) + entry(a, j, i);", "double t = 2.0 * entry(a, i, j);"),
    "pgs_no_chunk_size": (
        "constexpr int kPgsNoChunk = 16;", "constexpr int kPgsNoChunk = 8;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "the oracle's source changed: update %s" % name
    mutant = tmp_path / "mutant.cpp"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-o", str(lib), str(mutant)], check=True)
    env = dict(os.environ, MSP_ORACLE_LIB=str(lib))
    try:
        out = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p",
                              "no:cacheprovider", "-m", "not gpu"] + PINS, cwd=ROOT, env=env,
                             capture_output=True, text=True, timeout=300)
    except subprocess.TimeoutExpired:
        return  # the mistake stopped a pin from finishing: caught
    assert out.returncode != 0, "mistake %s passed every pin:\n%s" % (name, out.stdout[-2000:])
