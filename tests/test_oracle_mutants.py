"""Planted mistakes in the oracle must fail at least one pin.

Each mutant is a plausible slip (a dropped term, a wrong sign or index, a transposed
operand, a strict inequality, a missing step of the proposed schedule, FP64 instead of
FP32 rounding...). It is planted in a copy of the oracle's C source on the CPU, compiled
to a temporary library and run against the full pin battery in a child process.
"""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cc_oracle.c")

MUTANTS = {
    "int_dropped_dz": ("dx * dx + dy * dy + dz * dz;\n    return d2 <= (int64_t)r2;",
                       "dx * dx + dy * dy;\n    return d2 <= (int64_t)r2;"),
    "int_sign": ("int64_t dx = (int64_t)xi - (int64_t)xj;", "int64_t dx = (int64_t)xi + (int64_t)xj;"),
    "int_transposed": ("int64_t dy = (int64_t)yi - (int64_t)yj;", "int64_t dy = (int64_t)yi - (int64_t)zj;"),
    "int_strict": ("return d2 <= (int64_t)r2;", "return d2 < (int64_t)r2;"),
    "int_r2_plus_one": ("return d2 <= (int64_t)r2;", "return d2 <= (int64_t)r2 + 1;"),
    "loop_j_from_i": ("for (int64_t j = i + 1; j < n; ++j)\n            c += (uint64_t)collide_i32",
                      "for (int64_t j = i; j < n; ++j)\n            c += (uint64_t)collide_i32"),
    "loop_j_stops_early": ("for (int64_t j = i + 1; j < n; ++j)\n            c += (uint64_t)collide_i32",
                           "for (int64_t j = i + 1; j < n - 1; ++j)\n            c += (uint64_t)collide_i32"),
    "f32_s_not_squared": ("float s2 = s * s;", "float s2 = s;"),
    "f32_radius_twice": ("float s = ra + rb;", "float s = ra + ra;"),
    "f32_dropped_dz": ("float d2 = (dx * dx + dy * dy) + dz * dz;", "float d2 = (dx * dx + dy * dy);"),
    "f32_strict": ("return d2 <= s2;", "return d2 < s2;"),
    "f32_in_fp64": ("float d2 = (dx * dx + dy * dy) + dz * dz;  /* five roundings, this order */\n"
                    "    float s = ra + rb;\n    float s2 = s * s;",
                    "double d2 = ((double)xa - xb) * ((double)xa - xb) + ((double)ya - yb) * ((double)ya - yb)"
                    " + ((double)za - zb) * ((double)za - zb);\n"
                    "    double s = (double)ra + rb;\n    double s2 = s * s;"),
    "f32_term_no_floor": ("return 1.0 / (d > 1e-6 ? d : 1e-6);", "return 1.0 / d;"),
    "f32_term_squared": ("return 1.0 / (d > 1e-6 ? d : 1e-6);", "return 1.0 / (d > 1e-6 ? d * d : 1e-6);"),
    "f32_j_from_i": ("for (int64_t j = i + 1; j < n; ++j) {\n            if (collide_f32",
                     "for (int64_t j = i; j < n; ++j) {\n            if (collide_f32"),
    "cyclic_no_even_step_schedule": ("            if (k < cap) { pi[k] = i; pj[k] = i + n / 2; }\n            ++k;",
                                     "            if (k < cap) { pi[k] = i; pj[k] = i + n / 2; }"),
    "cyclic_even_step_all": ("if (n % 2 == 0 && i < n / 2) {\n            if (k < cap)",
                             "if (n % 2 == 0) {\n            if (k < cap)"),
    "cyclic_steps_n_over_2": ("int64_t steps = (n - 1) / 2;\n    for (int64_t i = 0; i < n; ++i) {\n        for (int64_t s = 1; s <= steps; ++s) {\n            if (k < cap)",
                              "int64_t steps = n / 2;\n    for (int64_t i = 0; i < n; ++i) {\n        for (int64_t s = 1; s <= steps; ++s) {\n            if (k < cap)"),
    "cyclic_count_no_even_step": ("            int64_t j = i + n / 2;\n            c += (uint64_t)collide_i32",
                                  "            int64_t j = i + n / 2;\n            c += 0 * (uint64_t)collide_i32"),
    "cyclic_count_wrong_wrap": ("int64_t j = (i + s) % n;", "int64_t j = (i + s) % n == 0 ? 1 : (i + s) % n;"),
    "alg1_after_increment": ("collisions += space[s];   /* beads already at this site */\n        space[s] += 1;",
                             "space[s] += 1;\n        collisions += space[s];"),
    "alg2_missing_neighbour": ("contacts += space[SITE(x[b], y[b], z[b] - 1)];", ""),
    "alg2_no_halving": ("return contacts / 2;", "return contacts;"),
    "sets_all_ordered": ("for (int64_t j = i + 1; j < b; ++j)\n                c += (uint64_t)collide_i32",
                         "for (int64_t j = a; j < b; ++j)\n                c += (uint64_t)collide_i32"),
    "i32_sum_no_floor": ("s += 1.0 / (d > 1e-6 ? d : 1e-6);", "s += 1.0 / d;"),
    "i32_sum_d2_not_d": ("double d = sqrt((double)d2);", "double d = (double)d2;"),
    "i32_sum_strict": ("if (d2 <= (int64_t)r2) {\n                double d", "if (d2 < (int64_t)r2) {\n                double d"),
    "i32_sum_dropped_dy": ("int64_t d2 = dx * dx + dy * dy + dz * dz;\n            if (d2 <= (int64_t)r2) {\n                double d",
                           "int64_t d2 = dx * dx + dz * dz;\n            if (d2 <= (int64_t)r2) {\n                double d"),
    "sets_sum_halved": ("if (sums) sums[k] = s;", "if (sums) sums[k] = s / 2;"),
    "sets_sum_wrong_partner": ("                    s += term_f64(x[i], y[i], z[i], x[j], y[j], z[j]);\n                }\n        counts[k] = c;",
                               "                    s += term_f64(x[i], y[i], z[i], x[a], y[a], z[a]);\n                }\n        counts[k] = c;"),
    "sets_sum_not_reset": ("        uint64_t c = 0;\n        double s = 0.0;\n        for (int64_t i = a; i < b; ++i)",
                           "        uint64_t c = 0;\n        static double s = 0.0;\n        for (int64_t i = a; i < b; ++i)"),
    "work_formula": ("return (n - 1) / 2 + ((n % 2 == 0 && i < n / 2) ? 1 : 0);",
                     "return n / 2;"),
}

RUNNER = r"""
import sys, traceback
sys.path.insert(0, {root!r})
import oracle
from tests import pins
oracle.use_library({lib!r})
failed = []
for p in pins.ALL_PINS:
    try:
        p(oracle)
    except Exception as e:
        failed.append(p.__name__)
print("FAILED:" + ",".join(failed))
"""


def _run_mutant(name, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mut = src.replace(old, new, 1)
    csrc = os.path.join(tmp, f"{name}.c")
    lib = os.path.join(tmp, f"lib{name}.so")
    with open(csrc, "w") as f:
        f.write(mut)
    subprocess.run(["gcc", *oracle.CFLAGS, csrc, "-o", lib, "-lm"], check=True,
                   capture_output=True)
    r = subprocess.run([sys.executable, "-c", RUNNER.format(root=ROOT, lib=lib)],
                       capture_output=True, text=True, timeout=600,
                       env={**os.environ, "OMP_NUM_THREADS": "2"})
    if r.returncode != 0:
        return name, ["<crashed>"]
    line = [l for l in r.stdout.splitlines() if l.startswith("FAILED:")][-1]
    return name, [t for t in line[len("FAILED:"):].split(",") if t]


def test_every_mutant_fails_a_pin():
    oracle.build()
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
            futs = [ex.submit(_run_mutant, k, o, n, tmp) for k, (o, n) in MUTANTS.items()]
            results = dict(f.result() for f in futs)
    survivors = [k for k, v in results.items() if not v]
    assert not survivors, f"mutants that pass every pin: {survivors}"
