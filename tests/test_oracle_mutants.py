"""Each pin of the oracle must be able to fail.  Every mutant below plants
one plausible mistake in a copy of oracle/ifa_oracle.c (a dropped term, a
wrong sign, bound or index, a missing complement or reversal, a changed
constant), is built with gcc, and must make at least one pin fail."""
import os
import subprocess
import tempfile

import pytest

import oracle
import test_oracle_brute as tb
import test_oracle_clip as tc
import test_oracle_indexed as ti

SRC = os.path.join(os.path.dirname(oracle.__file__), "ifa_oracle.c")

MUTANTS = {
    "N equals N": ("if (x == 'N' || y == 'N' || x != y) {", "if (x != y) {"),
    "last window dropped": ("for (uint64_t p = 0; p + L <= rlen[c]; p++) {\n                    uint32_t mm = window_mismatches(qq, r + p, L, max_subs);\n                    if (mm <= max_subs) {",
                            "for (uint64_t p = 0; p + L < rlen[c]; p++) {\n                    uint32_t mm = window_mismatches(qq, r + p, L, max_subs);\n                    if (mm <= max_subs) {"),
    "strict threshold": ("                    if (mm <= max_subs) {\n                        put_hit", "                    if (mm < max_subs) {\n                        put_hit"),
    "no complement": ("out[i] = complement_base(q[L - 1 - i]);", "out[i] = fold_base(q[L - 1 - i]);"),
    "no reversal": ("out[i] = complement_base(q[L - 1 - i]);", "out[i] = complement_base(q[i]);"),
    "lower case not a base": ("case 'A': case 'a': return 'A';", "case 'A': return 'A';"),
    "Philox multiplier": ("(uint64_t)0xD2511F53u * c0", "(uint64_t)0xD2511F55u * c0"),
    "Philox word order": ("uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi0 ^ c1 ^ k0;"),
    "Philox key bump": ("k1 += 0xBB67AE85u;", "k1 += 0xBB67AE84u;"),
    "biased shuffle": ("uint32_t j = i + ws_below(&ws, L - i);", "uint32_t j = ws_below(&ws, L);"),
    "survivor range": ("        for (uint32_t o = 0; o + k <= L; o += step) {\n            int ok = 1;\n            for (uint32_t j = 0; j < k; j++) {\n                if (mask_w && j >= mlo && j < mlo + mask_w)\n                    continue;\n                if (hitpos[o + j]) {",
                       "        for (uint32_t o = 0; o + k < L; o += step) {\n            int ok = 1;\n            for (uint32_t j = 0; j < k; j++) {\n                if (mask_w && j >= mlo && j < mlo + mask_w)\n                    continue;\n                if (hitpos[o + j]) {"),
    "quantile strict": ("if ((unsigned __int128)tail * den >= need)", "if ((unsigned __int128)tail * den > need)"),
    "bound clips sign": ("- (int64_t)(k - mask_w) * (int64_t)subs - (int64_t)max_clips;", "- (int64_t)(k - mask_w) * (int64_t)subs + (int64_t)max_clips;"),
    "bound ignores mask": ("- (int64_t)(k - mask_w) * (int64_t)subs - (int64_t)max_clips;", "- (int64_t)k * (int64_t)subs - (int64_t)max_clips;"),
    "mask not centred": ("static uint32_t window_seeds(const uint8_t *qq, const uint8_t *r, uint32_t L, uint32_t k,\n                             uint32_t step, uint32_t mask_w)\n{\n    uint32_t seeds = 0;\n    uint32_t mlo = (k - mask_w) / 2;",
                         "static uint32_t window_seeds(const uint8_t *qq, const uint8_t *r, uint32_t L, uint32_t k,\n                             uint32_t step, uint32_t mask_w)\n{\n    uint32_t seeds = 0;\n    uint32_t mlo = 0;"),
    "seed threshold strict": ("if (sd < minhits[j])", "if (sd <= minhits[j])"),
    "seed ignores N": ("            if (a == 'N' || b == 'N' || a != b)\n                ok = 0;", "            if (a != b)\n                ok = 0;"),
    "choose shortest k": ("if (m >= 1 && k > best_k) {", "if (m >= 1 && (best_k == 0 || k < best_k)) {"),
    "clip range start": ("for (int64_t p = -C; p <= len - (int64_t)L + C; p++) {",
                         "for (int64_t p = -C + 1; p <= len - (int64_t)L + C; p++) {"),
    "clip range end": ("for (int64_t p = -C; p <= len - (int64_t)L + C; p++) {",
                       "for (int64_t p = -C; p < len - (int64_t)L + C; p++) {"),
    "clip budget strict": ("if (clips == 0 || clips > C || clips >= (int64_t)L)",
                           "if (clips == 0 || clips >= C || clips >= (int64_t)L)"),
    "clips counted as mismatches": ("uint32_t mm = window_mismatches(qq + left, r + p + left, aligned, max_subs);",
                                    "uint32_t mm = window_mismatches(qq + left, r + p + left, aligned, max_subs) + (uint32_t)clips;"),
    "clipped query not shifted": ("uint32_t mm = window_mismatches(qq + left, r + p + left, aligned, max_subs);",
                                  "uint32_t mm = window_mismatches(qq, r + p + left, aligned, max_subs);"),
    "clip sides swapped": ("(uint16_t)(left | (right << 8))", "(uint16_t)(right | (left << 8))"),
    "clipped pos off by one": ("(uint64_t)(p + left), t, mm,", "(uint64_t)(p + left + 1), t, mm,"),
    "digest ignores clips": ("((uint64_t)h[i].clips << 16) | ", ""),
}


def _pins():
    """The pin checks, each a callable that raises when it fails."""
    wl = tb.synth.small_workload()
    wl2 = ti.synth.small_workload(seed=31, n_queries=5, lmin=14, lmax=36, n_contigs=8, cmin=100,
                                  cmax=1500, plant_ks=[0, 1, 1, 2, 2, 3, 4, 6] * 2)
    return [
        lambda: tb.test_brute_matches_scipy_hamming(7, 3),
        lambda: tb.test_brute_with_n_in_query(),
        lambda: tb.test_exact_matching_is_substring_search(wl),
        lambda: tb.test_every_window_when_subs_reach_length(wl),
        lambda: tb.test_planted_hits_present_with_exact_count(),
        lambda: tb.test_reverse_complement_symmetry(wl),
        lambda: ti.test_philox_known_answers([0, 0, 0, 0], [0, 0],
                                             [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
        lambda: ti.test_minhits_matches_exact_enumeration(12, 2, 4, 1, 0, 1, 2),
        lambda: ti.test_minhits_matches_exact_enumeration(14, 2, 5, 1, 1, 3, 4),
        lambda: ti.test_minhits_matches_exact_enumeration(20, 4, 8, 1, 0, 99, 100),
        lambda: ti.test_minhits_closed_forms(20, 8, 1),
        lambda: ti.test_deterministic_bound(30, 2, 8, 2, 1),
        lambda: ti.test_choose_k_closed_forms(),
        lambda: ti.test_quantile_rule_on_hand_histograms(),
        lambda: ti.test_n_is_never_part_of_a_seed(),
        lambda: ti.test_minhits_one_equals_text_seed_test(wl2, 7, 1, 3),
        lambda: ti.test_indexed_subset_and_degenerate_cases(wl2),
        lambda: ti.test_seed_counts_closed_forms(wl2),
        lambda: tc.test_closed_form_count_when_every_window_passes(25),
        lambda: tc.test_planted_overhangs_are_found_with_their_clips("start"),
        lambda: tc.test_planted_overhangs_are_found_with_their_clips("end"),
        lambda: tc.test_digest_sees_the_clips(),
        lambda: tc.test_matches_plain_python_definition_on_tiny_inputs(0),
    ]


@pytest.fixture(scope="module")
def pins():
    return _pins()


def test_pins_pass_on_the_oracle(pins):
    for p in pins:
        p()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_mutant_fails_a_pin(name, pins):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found uniquely: " + name
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mutant.c")
        so = os.path.join(d, "libmutant.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", so, c])
        failed = 0
        with oracle.use_library(so):
            for p in pins:
                try:
                    p()
                except AssertionError:
                    failed += 1
        assert failed > 0, "no pin caught mutant: " + name
