"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake (a wrong comparison, a dropped term, a wrong
index) in a temporary copy of ``oracle/peel_oracle.c``, compiles it on the CPU,
swaps it in, and runs the pin tests against it: at least one pin has to fail.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_subrounds as sub
import test_oracle_signed as signed

MUTANTS = [
    ("round removes degree <= k",
     "if (vround[v] == 0 && deg[v] < (int64_t)k) ++nr;",
     "if (vround[v] == 0 && deg[v] <= (int64_t)k) ++nr;"),
    ("removed edge decrements only its first endpoint",
     "for (uint32_t j = 0; j < r; ++j) deg[edges[e * r + j]] -= 1;",
     "for (uint32_t j = 0; j < 1; ++j) deg[edges[e * r + j]] -= 1;"),
    ("queue peeler pushes at the wrong crossing",
     "if (deg[u] == (int64_t)k - 1 && v_core[u]) stack[top++] = u;",
     "if (deg[u] == (int64_t)k && v_core[u]) stack[top++] = u;"),
    ("edge removal tested against the previous round",
     "if (vround[edges[e * r + j]] == (int32_t)round) hit = 1;",
     "if (vround[edges[e * r + j]] == (int32_t)round - 1) hit = 1;"),
    ("hash uses sub-table 0's seed for every sub-table",
     "uint64_t h = mix64(x ^ seeds[j]);",
     "uint64_t h = mix64(x ^ seeds[0]);"),
    ("checksum not removed on recovery",
     "        keyx[c] ^= x;\n        chkx[c] ^= cs;\n      }\n      out_keys[total + i] = x;",
     "        keyx[c] ^= x;\n      }\n      out_keys[total + i] = x;"),
    ("pure test drops the checksum comparison",
     "return count[c] == 1 && chkx[c] == checksum_of(keyx[c], seeds, r);",
     "return count[c] == 1 || chkx[c] == checksum_of(keyx[c], seeds, r);"),
    ("checksum keeps only the upper half of mix64",
     "  return mix64(x ^ seeds[r]);\n}",
     "  return mix64(x ^ seeds[r]) >> 32;\n}"),
    ("checksum summed instead of XORed",
     "      chkx[c] ^= cs;\n    }\n  }\n  return ORC_OK;",
     "      chkx[c] += (uint64_t)sign * cs;\n    }\n  }\n  return ORC_OK;"),
    ("checksum taken of the key's cell seed instead of its own",
     "  return mix64(x ^ seeds[r]);\n}",
     "  return mix64(x ^ seeds[0]);\n}"),
    ("a key pure in two cells is recovered twice",
     "if (i == 0 || pure_keys[i] != pure_keys[i - 1]) pure_keys[nk++] = pure_keys[i];",
     "pure_keys[nk++] = pure_keys[i];"),
    ("surviving cells counted from degree 1",
     "if (count[c] >= 2) ++alive;",
     "if (count[c] >= 1) ++alive;"),
    ("sub-table split puts the remainder last",
     "off[j + 1] = off[j] + q + (j < rem ? 1 : 0);",
     "off[j + 1] = off[j] + q + (j >= r - rem ? 1 : 0);"),
    ("sub-round looks at every part at once",
     "    for (uint32_t v = part_off[j]; v < part_off[j + 1]; ++v)\n      if (vround[v] == 0 && deg[v] < (int64_t)k) ++nrem;\n",
     "    for (uint32_t v = 0; v < n; ++v)\n      if (vround[v] == 0 && deg[v] < (int64_t)k) ++nrem;\n"),
    ("sub-round process stops at the first idle sub-round",
     "while (idle < p) {",
     "while (idle < 1) {"),
    ("sub-round count includes the trailing idle sub-rounds",
     "  *S_out = S;\n  free(deg);",
     "  *S_out = s;\n  free(deg);"),
    ("IBLT sub-round scans every sub-table",
     "for (uint64_t c = off[j]; c < off[j + 1]; ++c)",
     "for (uint64_t c = 0; c < n; ++c)"),
    ("IBLT sub-tables visited in reverse order",
     "    const uint32_t j = s % r;",
     "    const uint32_t j = r - 1 - s % r;"),
    ("signed removal ignores the sign",
     "        count[c] -= sg;",
     "        count[c] -= 1;"),
    ("signed purity misses negative counts",
     "if ((count[c] == 1 || count[c] == -1) &&",
     "if ((count[c] == 1) &&"),
    ("signed purity compares against a signed checksum",
     "          chkx[c] == checksum_of(keyx[c], seeds, r)) {",
     "          chkx[c] == (uint64_t)count[c] * checksum_of(keyx[c], seeds, r)) {"),
    ("signed recovery leaves the checksum in",
     "        keyx[c] ^= x;\n        chkx[c] ^= cs;\n      }\n    }\n    total += nk;",
     "        keyx[c] ^= x;\n      }\n    }\n    total += nk;"),
    ("mix64 shift constant off by one",
     "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;",
     "z = (z ^ (z >> 28)) * 0x94D049BB133111EBULL;"),
]

PINS = [
    lambda: pins.test_mix64_published_splitmix_vector(),
    lambda: pins.test_hash_known_answers(),
    lambda: pins.test_part_offsets_headline(),
    lambda: [pins.test_handmade_cores(*h) for h in pins.HANDMADE],
    lambda: pins.test_handmade_expected_values(),
    lambda: pins.test_random_tiny_hypergraphs_vs_brute_force(),
    lambda: pins.test_iblt_build_definition(),
    lambda: pins.test_iblt_checksum_field_is_an_xor(),
    lambda: pins.test_cell_map_boundaries(),
    lambda: pins.test_iblt_rounds_equal_kcore_rounds(4000, 3, 0.7, 1),
    lambda: pins.test_iblt_rounds_equal_kcore_rounds(3000, 4, 0.85, 3),
    lambda: pins.test_iblt_below_threshold_recovered_inserted_set_wrapper(),
    lambda: pins.test_iblt_residue_invariants_above_threshold(),
    lambda: pins.test_iblt_checksum_rejects_impure_count_one(),
    lambda: sub.test_hand_worked_path(),
    lambda: sub.test_hand_worked_idle_part_in_the_middle(),
    lambda: sub.test_one_part_is_the_round_process(),
    lambda: sub.test_tiny_hypergraphs_vs_sets(),
    lambda: sub.test_iblt_subrounds_equal_kcore_subrounds(2000, 3, 0.75, 1),
    lambda: sub.test_iblt_subrounds_recover_inserted_set_below_threshold(),
    lambda: signed.test_insert_only_equals_unsigned(3000, 3, 0.7, 1),
    lambda: signed.test_set_difference_recovered(4000, 3, 4),
    lambda: signed.test_rounds_equal_the_k2_peel_of_the_difference(4000, 3, 9, 0.4, 0.35),
]


def _compile_mutant(tmp_path, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "peel_oracle.c")).read()
    assert src.count(old) == 1, old
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(path)])
    return oracle.configure(ctypes.CDLL(str(so)))


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, monkeypatch, name, old, new):
    mutant = _compile_mutant(tmp_path, old, new)
    monkeypatch.setattr(oracle, "_lib", mutant)
    caught = []
    for i, pin in enumerate(PINS):
        try:
            pin()
        except Exception as exc:   # an assertion or a crash-free error both count
            caught.append((i, type(exc).__name__))
    assert caught, f"no pin failed for planted mistake: {name}"


def test_unmutated_oracle_passes_every_pin():
    for pin in PINS:
        pin()
