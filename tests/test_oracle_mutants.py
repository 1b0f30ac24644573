"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a temporary copy of the oracle's C source
(on the CPU, never on a GPU), builds it, and runs the pin suite against it
in a subprocess: the suite has to fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "plm_oracle.c")

MUTANTS = {
    "field dropped from the logits": ("double acc = h_r[s];", "double acc = 0.0;"),
    "gradient sign flipped": ("double d = -(w[b] / beff)", "double d = (w[b] / beff)"),
    "coupling read with transposed states":
        ("acc += J_r[((size_t)s * N + i) * q + seq[i]];",
         "acc += J_r[((size_t)seq[i] * N + i) * q + s];"),
    "lambda_J not halved": ("const double lambda_Jp = 0.5 * lambda_J; /* step 1 of the rundown */\n    const size_t Jr_len = (size_t)q * N * q;\n#pragma omp parallel for schedule(dynamic, 1)\n    for (int r = 0; r < N; ++r) {\n        f[r]",
                            "const double lambda_Jp = 1.0 * lambda_J;\n    const size_t Jr_len = (size_t)q * N * q;\n#pragma omp parallel for schedule(dynamic, 1)\n    for (int r = 0; r < N; ++r) {\n        f[r]"),
    "penalty gradient missing its factor 2": ("gJ_r[e] += 2.0 * lambda_Jp * J_r[e];", "gJ_r[e] += lambda_Jp * J_r[e];"),
    "mirror block not transposed":
        ("bj[k * q + l] = J[(size_t)j * Jr_len + ((size_t)l * N + i) * q + k];",
         "bj[k * q + l] = J[(size_t)j * Jr_len + ((size_t)k * N + i) * q + l];"),
    "gap-gap not counted as identity":
        ("if (S[(size_t)a * N + i] == S[(size_t)b * N + i]) matches++;",
         "if (S[(size_t)a * N + i] == S[(size_t)b * N + i] && S[(size_t)b * N + i] != 0) matches++;"),
    "strict similarity threshold": ("if (matches >= T) count++;", "if (matches > T) count++;"),
    "APC row mean includes the diagonal": ("row[i] = s / (N - 1);", "row[i] = s / N;"),
    "gauge grand mean with wrong sign": ("- colm[l] - rowm[k] + all;", "- colm[l] - rowm[k] - all;"),
    "diagonal block receives data gradient":
        ("if (i == r) continue;\n                        gJ_r[((size_t)s * N + i) * q + seq[i]] += d;",
         "gJ_r[((size_t)s * N + i) * q + seq[i]] += d;"),
    "weights not normalised by B_eff": ("return -loglik / beff + lambda_h", "return -loglik / B + lambda_h"),
    "min and max combiners swapped":
        ("if (combine == 1) v = gi[e] < gj[e] ? gi[e] : gj[e];",
         "if (combine == 1) v = gi[e] > gj[e] ? gi[e] : gj[e];"),
    "min combiner computed as the mean":
        ("if (combine == 1) v = gi[e] < gj[e] ? gi[e] : gj[e];",
         "if (combine == 1) v = 0.5 * (gi[e] + gj[e]);"),
    "max combiner of the score alternatives computed as the min":
        ("else if (combine == 2) v[e] = gi[e] > gj[e] ? gi[e] : gj[e];",
         "else if (combine == 2) v[e] = gi[e] < gj[e] ? gi[e] : gj[e];"),
    # symmetric plmDCA (caught by the symmetric pins)
    "symmetric mirror copy not transposed":
        ("J[(((size_t)j * q + l) * N + i) * q + k] = blk[k * q + l]; /* J_ji(l,k) */",
         "J[(((size_t)j * q + k) * N + i) * q + l] = blk[k * q + l];", "sym"),
    "symmetric block gradient of the second site not transposed":
        ("gJ[(((size_t)j * q + l) * N + i) * q + k];",
         "gJ[(((size_t)j * q + k) * N + i) * q + l];", "sym"),
    "symmetric block gradient from one site only":
        ("blk[k * q + l] = gJ[(((size_t)i * q + k) * N + j) * q + l] +",
         "blk[k * q + l] = gJ[(((size_t)i * q + k) * N + j) * q + l] + 0.0 *", "sym"),
    # score alternatives (caught by the score pins)
    "l_p norm without absolute values":
        ("double a = fabs(v[k * q + l]);", "double a = v[k * q + l];", "scores"),
    "gap exclusion on rows only":
        ("if (exclude_gap && (k == 0 || l == 0)) continue;",
         "if (exclude_gap && k == 0) continue;", "scores"),
    "Burkoff log ratio without the column frequency":
        ("if (P > 0.0) out += P * log(P / (fi[k] * fj[l]));",
         "if (P > 0.0) out += P * log(P / fi[k]);", "scores"),
    "average sum correction with the grand mean subtracted":
        ("fn[(size_t)i * N + j] - col[j] - row[i] + tot;",
         "fn[(size_t)i * N + j] - col[j] - row[i] - tot;", "scores"),
}

PIN_FILES = {"pins": "test_oracle_pins.py", "sym": "test_oracle_symmetric.py",
             "scores": "test_oracle_scores.py"}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name][:2]
    pins = PIN_FILES[MUTANTS[name][2] if len(MUTANTS[name]) > 2 else "pins"]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mutated = src.replace(old, new, 1)
    cfile = tmp_path / "mut.c"
    cfile.write_text(mutated)
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                    "-o", str(lib), str(cfile), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q",
                          os.path.join(ROOT, "tests", pins)],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"pins did not catch: {name}\n{res.stdout[-2000:]}"
