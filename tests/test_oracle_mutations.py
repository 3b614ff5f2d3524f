"""The pins must reject plausible mistakes in the oracle.

Each case copies the oracle's C source, plants one mistake by text
substitution (a wrong index, shift direction, dropped term, transposed
operand, ...), compiles the copy, and runs the pin suite against it in a
subprocess.  The pin suite has to fail for every planted mistake.  CPU only.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "successor_index": ("uint32_t y = (x[i] & p->mask) ^ x[i + 1];",
                        "uint32_t y = (x[i] & p->mask) ^ x[i + 2];"),
    "pos_index": ("y ^= x[i + p->pos] >> p->sh2;", "y ^= x[i + p->pos + 1] >> p->sh2;"),
    "sh1_direction": ("y ^= y << p->sh1;", "y ^= y >> p->sh1;"),
    "sh2_direction": ("y ^= x[i + p->pos] >> p->sh2;", "y ^= x[i + p->pos] << p->sh2;"),
    "mask_dropped": ("uint32_t y = (x[i] & p->mask) ^ x[i + 1];",
                     "uint32_t y = x[i] ^ x[i + 1];"),
    "mask_on_successor": ("uint32_t y = (x[i] & p->mask) ^ x[i + 1];",
                          "uint32_t y = x[i] ^ (x[i + 1] & p->mask);"),
    "rec_index_bits": ("x[i + n] = y ^ p->rec_tbl[y & 0xFu];",
                       "x[i + n] = y ^ p->rec_tbl[(y >> 28) & 0xFu];"),
    "tempering_word": ("uint32_t t = x[i + p->pos - 1];", "uint32_t t = x[i + p->pos];"),
    "fold_dropped": ("t ^= t >> 8;\n", "\n"),
    "temper_pre_table": ("uint32_t o = x[i + n] ^ p->tmp_tbl[t & 0xFu];",
                         "uint32_t o = y ^ p->tmp_tbl[t & 0xFu];"),
    "mantissa_shift": ("uint32_t bits12 = 0x3F800000u | (o >> 9);",
                       "uint32_t bits12 = 0x3F800000u | (o >> 9) | 1u;"),
    "state_save_offset": ("memcpy(state, x + count, (size_t)n * sizeof(uint32_t));",
                          "memcpy(state, x + count + 1, (size_t)(n - 1) * sizeof(uint32_t));"),
    "seed_shift": ("(state[i - 1] ^ (state[i - 1] >> 30)) + i;",
                   "(state[i - 1] ^ (state[i - 1] >> 29)) + i;"),
    "table_span": ("if (k & (1u << b))", "if (k & (1u << (3 - b)))"),
    "mask_width": ("p->mask = 0xFFFFFFFFu << (uint32_t)r;",
                   "p->mask = 0xFFFFFFFFu << (uint32_t)(r - 1);"),
}

# Mistakes in the statistics of tests 35 / 100, caught by their own pins.
QUALITY_MUTANTS = {
    "gap_off_by_one": ("hist[run < t ? run : t] += 1;", "hist[run + 1 < t ? run + 1 : t] += 1;"),
    "gap_run_not_reset": ("            run = 0;\n        } else {",
                          "            run = 1;\n        } else {"),
    "gap_field_position": ("uint64_t v = ((uint64_t)x << r) & 0xFFFFFFFFull;   /* drop r leading bits */",
                           "uint64_t v = ((uint64_t)x << (r + 1)) & 0xFFFFFFFFull;"),
    "hamming_class_strict": ("if (bounds[i] <= w)", "if (bounds[i] < w)"),
    "hamming_pair_transposed": ("table[cls[0] * C + cls[1]] += 1;", "table[cls[1] * C + cls[0]] += 1;"),
    "hamming_field_width": ("uint32_t field = (uint32_t)(v >> (32 - s));",
                            "uint32_t field = (uint32_t)(v >> (31 - s));"),
}


# Mistakes in the original-MT oracle (the comparison generator of Sec. 5.3).
MT_MUTANTS = {
    "mt_successor_index": ("(x[k + 1] & lower)", "(x[k + 2] & lower)"),
    "mt_middle_index": ("x[k + n] = x[k + q->m] ^ ya;", "x[k + n] = x[k + q->m - 1] ^ ya;"),
    "mt_upper_lower_swapped": ("uint32_t y = (x[k] & upper) | (x[k + 1] & lower);",
                               "uint32_t y = (x[k] & lower) | (x[k + 1] & upper);"),
    "mt_twist_test_bit": ("((y & 1u) ? q->a : 0u)", "((y & 2u) ? q->a : 0u)"),
    "mt_twist_shift_direction": ("uint32_t ya = (y >> 1)", "uint32_t ya = (y << 1)"),
    "mt_separation_width": ("0xFFFFFFFFu << q->r : 0xFFFFFFFFu;",
                            "0xFFFFFFFFu << (q->r - 1u) : 0xFFFFFFFFu;"),
    "mt_temper_b_direction": ("z ^= (z << q->s) & q->b;", "z ^= (z >> q->s) & q->b;"),
    "mt_temper_c_mask": ("z ^= (z << q->t) & q->c;", "z ^= (z << q->t) & q->b;"),
    "mt_temper_last_shift": ("z ^= z >> q->l;", "z ^= z >> q->u;"),
    "mt_temper_before_twist": ("uint32_t z = x[k + n];", "uint32_t z = x[k + q->m];"),
    "mt_seed_multiplier": ("1812433253u * (state[i - 1]", "1812433255u * (state[i - 1]"),
    "mt_state_save_offset": ("memcpy(state, x + count, (size_t)n * sizeof(uint32_t));",
                             "memcpy(state, x + count + 1, (size_t)(n - 1) * sizeof(uint32_t));"),
    "mt_middle_draw": ("q->m = q->n / 2u;", "q->m = (q->n + 1u) / 2u;"),
    "mt_a_top_bit": ("| 0x80000000u;", "| 0x40000000u;"),
}

# group -> (oracle source, library override variable, pin suite, mutants)
GROUPS = {
    "mtgp": ("mtgp_oracle.c", "MTGP_ORACLE_LIB", "test_oracle_pins.py", MUTANTS),
    "quality": ("mtgp_oracle.c", "MTGP_ORACLE_LIB", "test_quality_oracle.py", QUALITY_MUTANTS),
    "mt": ("mt_oracle.c", "MT_ORACLE_LIB", "test_mt_oracle.py", MT_MUTANTS),
}
CASES = [(g, name) for g in GROUPS for name in sorted(GROUPS[g][3])]


@pytest.mark.parametrize("group,name", CASES, ids=["%s-%s" % c for c in CASES])
def test_pins_reject_planted_mistake(group, name, tmp_path):
    src_name, env_var, pins, mutants = GROUPS[group]
    before, after = (x.replace("\\n", "\n") for x in mutants[name])
    src = open(os.path.join(ROOT, "oracle", src_name)).read()
    assert src.count(before) == 1, name
    mutant_c = tmp_path / "mutant.c"
    mutant_c.write_text(src.replace(before, after))
    # the header sits beside the original source
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-shared", "-fPIC",
                           "-I", os.path.join(ROOT, "oracle"), "-o", str(lib), str(mutant_c),
                           "-lpthread"])
    env = dict(os.environ, **{env_var: str(lib)})
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "pins accepted mutant %s:\n%s" % (name, r.stdout[-2000:])
