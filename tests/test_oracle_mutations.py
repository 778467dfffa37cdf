"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of oracle/flash_oracle.c
(a dropped term, a wrong index or sign, a swapped order, an off-by-one) and
runs the pin that is meant to catch it against that copy, in a subprocess.
The pin must fail.  CPU only; nothing here touches the CUDA path.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = "tests/test_oracle_pins.py"

# name: (original text, planted mistake, pin expected to fail)
MUTATIONS = {
    "max_instead_of_min": ("if (!filled[bin] || off < v[bin])", "if (!filled[bin] || off > v[bin])",
                           "test_minhash_is_a_min_over_elements"),
    "bin_from_low_bits": ("uint32_t bin = (uint32_t)(p >> 32);", "uint32_t bin = (uint32_t)(pi % B);",
                          "test_oph_bins_split_one_permutation_into_equal_ranges"),
    "additive_seed_dropped": ("uint32_t pi = (uint32_t)((s->a1 * i + s->b1) >> 32);",
                              "uint32_t pi = (uint32_t)((s->a1 * i) >> 32);",
                              "test_each_column_lands_in_a_uniform_bin_over_seeds"),
    "rotation_offset_dropped": ("h[j] = v[src] + t * 0x9E3779B9u;", "h[j] = v[src];",
                                "test_densification_closed_form_from_singletons"),
    "rotation_distance_sign": ("uint32_t t = src >= j ? src - j : src + B - j;",
                               "uint32_t t = src >= j ? j - src : j + B - src;",
                               "test_densification_closed_form_from_singletons"),
    "tuple_contiguous_not_interleaved": ("x = x * s->a2 + (uint64_t)h[t + j * L];",
                                         "x = x * s->a2 + (uint64_t)h[t * K + j];",
                                         "test_table_key_collision_rate_is_jaccard_to_the_K"),
    "fold_without_multiply": ("x = x * s->a2 + (uint64_t)h[t + j * L];", "x = x + (uint64_t)h[t + j * L];",
                              "test_address_map_is_universal_on_k_tuples"),
    "fold_uses_one_hash": ("for (j = 0; j < K; ++j) x = x * s->a2", "for (j = 0; j < 1; ++j) x = x * s->a2",
                           "test_table_key_collision_rate_is_jaccard_to_the_K"),
    "address_from_low_bits": ("return (uint32_t)((s->a2 * x + s->b2) >> (64 - rb));",
                              "return (uint32_t)((s->a2 * x + s->b2) & ((1ULL << rb) - 1));",
                              "test_table_keys_are_uniform_over_the_range"),
    "random_range_one_short": ("return (uint32_t)(((u >> 32) * (i + 1)) >> 32);",
                               "return (uint32_t)(((u >> 32) * (i)) >> 32);",
                               "test_reservoir_is_a_uniform_sample"),
    "no_fill_first": ("  if (i < R) {\n    reservoir[i] = point;\n  } else {", "  if (0) {\n  } else {",
                      "test_reservoir_keeps_every_arrival_while_not_full"),
    "draw_ignores_table": ("splitmix64_mix(r ^ (((uint64_t)t << 32) + (uint64_t)b))",
                           "splitmix64_mix(r ^ ((uint64_t)b))", "test_reservoir_is_a_uniform_sample"),
    "run_length_minus_one": ("kv[m].count = 1;", "kv[m].count = 0;",
                             "test_kselect_matches_counting_by_dictionary"),
    "ties_to_larger_id": ("return (x->id > y->id) - (x->id < y->id);",
                          "return (x->id < y->id) - (x->id > y->id);", "test_kselect_matches_counting_by_dictionary"),
    "exclude_not_dropped": ("if (kv[i].id != exclude) kv[w++] = kv[i];", "kv[w++] = kv[i];",
                            "test_kselect_matches_counting_by_dictionary"),
    "empty_rows_inserted": ("    if (nnz == 0) continue;\n    doph_row", "    doph_row",
                            "test_empty_rows_are_not_inserted_and_report_nothing"),
    "gather_one_slot_short": ("uint32_t m = counts[bucket] < R ? counts[bucket] : R, j;",
                              "uint32_t m = counts[bucket] < R ? counts[bucket] : R - 1, j;",
                              "test_candidate_count_total_is_the_gathered_reservoir_size"),
    "seed_not_forced_odd": ("s.a1 = splitmix64_next(&st) | 1ULL;", "s.a1 = splitmix64_next(&st) & ~1ULL;",
                            "test_seed_words_are_published_splitmix64_outputs"),
    "optimal_copy_with_offset": ("      h[j] = v[src];\n", "      h[j] = v[src] + 0x9E3779B9u;\n",
                                 "test_optimal_densification_copies_non_empty_bins"),
    "optimal_probe_ignores_bin": ("splitmix64_mix(s->d ^ (((uint64_t)j << 32) | i))", "splitmix64_mix(s->d ^ i)",
                                  "test_optimal_densification_picks_sources_independently_per_bin"),
    "optimal_probe_ignores_attempt": ("splitmix64_mix(s->d ^ (((uint64_t)j << 32) | i))",
                                      "splitmix64_mix(s->d ^ (((uint64_t)j << 32) | 1))",
                                      "test_optimal_densification_picks_sources_independently_per_bin"),
    "pool_ignores_table": ("splitmix64_mix(s->e ^ (((uint64_t)t << 32) + (uint64_t)b))",
                           "splitmix64_mix(s->e ^ ((uint64_t)b))",
                           "test_shared_pool_map_is_uniform_and_independent_across_tables"),
    "shared_build_wrong_reservoir": ("uint32_t x = pool_index(&s, t, key, P);", "uint32_t x = key % P;",
                                     "test_shared_reservoirs_receive_arrivals_point_by_point_then_table_by_table"),
    "shared_query_ignores_table": ("uint32_t x = pool_index(&s, t, key, P), m", "uint32_t x = pool_index(&s, 0, key, P), m",
                                   "test_collision_free_pool_changes_nothing"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pin_catches_planted_mistake(name, tmp_path):
    orig, bad, pin = MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "flash_oracle.c")).read()
    assert src.count(orig) >= 1, f"mutation site for {name} not found"
    work = tmp_path / "repo"
    (work / "oracle").mkdir(parents=True)
    (work / "tests").mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), work / "oracle" / "__init__.py")
    (work / "oracle" / "flash_oracle.c").write_text(src.replace(orig, bad, 1))
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), work / "tests" / f)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), work / "tests" / "golden")
    shutil.copytree(os.path.join(ROOT, "paper_1709_01190_gb300", "synth"), work / "pkg_synth",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    # the pins draw small workloads from the input generator: give the copy the same package name
    pkg = work / "paper_1709_01190_gb300"
    pkg.mkdir()
    (pkg / "__init__.py").write_text("")
    shutil.move(str(work / "pkg_synth"), str(pkg / "synth"))
    env = dict(os.environ, PYTHONPATH=str(work))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py", "-k", pin], cwd=work, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and " failed" in r.stdout, f"{name} survived {pin}:\n{r.stdout[-2000:]}"
