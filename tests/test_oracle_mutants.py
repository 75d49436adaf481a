"""Every plausible mistake planted in a copy of the oracle is caught by a pin.

Each mutant is the oracle's C source with one textual change (a wrong
constant, shift, operator, word order, layout or emit order).  It is compiled
to a temporary library and the pins of ``tests/pins.py`` are run against it:
at least one must fail.  The real oracle is never modified.
"""
import os

import pytest

import oracle
from tests import pins

MUTANTS = {
    "hash_low_shift12": ("(r << 12)", "(r << 13)"),
    "hash_low_const2": ("0xc761c23cu", "0xc761c23du"),
    "hash_low_dir19": ("(r >> 19)", "(r << 19)"),
    "hash_low_round4_op": ("(r + 0xd3a2646cu) ^ (r << 9)", "(r + 0xd3a2646cu) + (r << 9)"),
    "hash_low_dropped_term": ("r = (r + 0xfd7046c5u) + (r << 3);", "r = (r + 0xfd7046c5u);"),
    "hash_high_round2_op": ("r = r + (r << 3);", "r = r ^ (r << 3);"),
    "hash_high_mult": ("r * 0x27d4eb2du", "r * 0x27d4eb2cu"),
    "hash_high_xor61": ("(r ^ 61u)", "(r ^ 60u)"),
    "step_shift21": ("s ^ (s << 21)", "s ^ (s << 20)"),
    "step_dir35": ("s ^ (s >> 35)", "s ^ (s << 35)"),
    "step_shift4": ("s ^ (s << 4)", "s ^ (s << 5)"),
    "word_order": ("((uint64_t)y << 32) | (uint64_t)x", "((uint64_t)x << 32) | (uint64_t)y"),
    "hash_input_not_id": ("oracle_hash_low(id32 ^ oracle_seed_key(seed))", "oracle_hash_low(id32 + oracle_seed_key(seed))"),
    "emit_after_step": ("row[g] = oracle_output(state[g], mode);\n            state[g] = oracle_step(state[g]);",
                        "state[g] = oracle_step(state[g]);\n            row[g] = oracle_output(state[g], mode);"),
    "stream_major_layout": ("uint64_t *row = out + i * n_streams;", "uint64_t *row = out + i;"),
    "dropped_g0": ("state[g] = oracle_step_k(oracle_initial_state(g0 + g, seed), p0);\n    for (uint64_t i = 0; i < iterations; ++i) {\n        uint64_t *row",
                   "state[g] = oracle_step_k(oracle_initial_state(g, seed), p0);\n    for (uint64_t i = 0; i < iterations; ++i) {\n        uint64_t *row"),
    "mix64_const": ("0xbf58476d1ce4e5b9ull", "0xbf58476d1ce4e5b8ull"),
    "mix64_shift": ("z = z ^ (z >> 31);", "z = z ^ (z >> 32);"),
    "seed_fold": ("(uint32_t)(m & 0xffffffffu) ^ (uint32_t)(m >> 32)", "(uint32_t)(m & 0xffffffffu)"),
    "xor_checksum_or": ("x ^= v;", "x |= v;"),
    "sum_checksum_xor": ("s += v;", "s ^= v;"),
    "star_constant": ("s * 2685821657736338717ull", "s * 2685821657736338719ull"),
    "star_on_next_state": ("uint64_t v = oracle_output(state[g], mode);",
                           "uint64_t v = oracle_output(oracle_step(state[g]), mode);"),
    "star_always": ("return mode ? s * 2685821657736338717ull : s;", "return s * 2685821657736338717ull;"),
}


def _run_pins(o):
    failures = []
    for check in pins.ALL_CHECKS:
        try:
            check(o)
        except AssertionError as e:  # the pin caught the planted mistake
            failures.append(f"{check.__name__}: {e}")
    return failures


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(oracle.SOURCE).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique in the oracle source"
    mutated = tmp_path / f"{name}.c"
    mutated.write_text(src.replace(old, new))
    lib_path = oracle.compile_source(str(mutated), str(tmp_path / f"lib{name}.so"))
    failures = _run_pins(oracle.OracleLib(lib_path))
    assert failures, f"planted mistake {name!r} passed every pin"
