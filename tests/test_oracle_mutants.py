"""Planted mistakes in the oracle must be caught by its pins.

Each mutant is a copy of the oracle source with one plausible mistake (a
wrong character class, a reversed comparison, an off-by-one, a dropped step),
compiled on the CPU into a temporary library.  The test passes when at least
one pin fails on it, which shows the pins constrain that part of the oracle.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle
import oracle_pins

MUTANTS = {
    "digits_are_letters": ("return (c >= 'A' && c <= 'Z') || (c >= 'a' && c <= 'z');",
                           "return (c >= 'A' && c <= 'Z') || (c >= 'a' && c <= 'z') || (c >= '0' && c <= '9');"),
    "only_space_and_lf_split": ("return c == 0x20 || (c >= 0x09 && c <= 0x0D);", "return c == 0x20 || c == 0x0A;"),
    "punctuation_splits_A": ("    if (is_space(c)) {\n      if (!cur.empty()) {",
                             "    if (!is_letter(c)) {\n      if (!cur.empty()) {"),
    "drops_last_word_A": ("  if (!cur.empty()) words.push_back(cur);\n  return words;",
                          "  return words;"),
    "descending_rows": ("if (a[i] != b[i]) return a[i] > b[i];", "if (a[i] != b[i]) return a[i] < b[i];"),
    "first_byte_only": ("for (uint32_t i = 0; i < len; ++i) {\n    if (a[i] != b[i])",
                        "for (uint32_t i = 0; i < 1; ++i) {\n    if (a[i] != b[i])"),
    "bubble_skips_last_pair": ("for (uint64_t j = 0; j + 1 < count - pass; ++j) {",
                               "for (uint64_t j = 0; j + 2 < count - pass; ++j) {"),
    "bubble_stops_on_swap": ("if (!swapped) break;", "if (swapped) break;"),
    "bubble_one_pass_short": ("for (uint64_t pass = 0; pass + 1 < count; ++pass) {",
                              "for (uint64_t pass = 0; pass + 2 < count; ++pass) {"),
    "compares_not_counted": ("      ++*compares;\n", "\n"),
    "counts_shifted": ("out->counts[L] = buckets[L].size();", "out->counts[L - 1] = buckets[L].size();"),
    "last_offset_wrong": ("out->offsets[j] = static_cast<uint32_t>(pos);\n  return 0;",
                          "out->offsets[j] = static_cast<uint32_t>(pos - 1);\n  return 0;"),
    "longest_bucket_first": ("for (uint32_t L = 1; L <= max_len; ++L) {\n    out->counts[L]",
                             "for (uint32_t L = max_len; L >= 1; --L) {\n    out->counts[L]"),
    "stable_descending": ("return static_cast<unsigned char>(x) < static_cast<unsigned char>(y);",
                          "return static_cast<unsigned char>(x) > static_cast<unsigned char>(y);"),
    "split_filter_keeps_punct": ("if (is_letter(b[k])) w.push_back", "if (b[k] != ',') w.push_back"),
    "case_folded": ("      cur.push_back(static_cast<char>(c));",
                    "      cur.push_back(static_cast<char>(c | 0x20));"),
    "folded_ties_reversed": ("  return bytes_less(a, b);\n}", "  return bytes_less(b, a);\n}"),
    "folded_letters_reversed": ("return fold(a[i]) < fold(b[i]);", "return fold(a[i]) > fold(b[i]);"),
    "folded_ignores_case_ties": ("  if (a.size() != b.size()) return a.size() < b.size();\n  return bytes_less(a, b);",
                                 "  return a.size() < b.size();"),
    "whole_by_length_first": ("    case 2: return bytes_less(b, a);",
                              "    case 2: return a.size() != b.size() ? a.size() > b.size() : bytes_less(b, a);"),
    "length_order_unstable": ("    case 3: return a.size() > b.size();", "    case 3: return a.size() >= b.size();"),
    "max_len_off_by_one": ("if (!buckets[L].empty()) max_len = static_cast<uint32_t>(L);",
                           "if (!buckets[L].empty()) max_len = static_cast<uint32_t>(L) + 1;"),
}


def _build_mutant(tmpdir: str, name: str, find: str, repl: str) -> str:
    src = open(oracle.SOURCE).read()
    assert src.count(find) == 1, f"mutation site for {name} not found exactly once"
    path = os.path.join(tmpdir, f"{name}.cpp")
    with open(path, "w") as f:
        f.write(src.replace(find, repl))
    return oracle.compile_library(path, os.path.join(tmpdir, f"lib{name}.so"))


_RUNNER = """
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle, oracle_pins
lib = oracle.bind({lib!r})
failed = []
for pin in oracle_pins.ALL_PINS:
    try:
        pin(lib)
    except (AssertionError, RuntimeError):
        failed.append(pin.__name__)
print("FAILED_PINS", failed)
sys.exit(3 if failed else 0)
"""


def _run_pins(lib_path: str) -> subprocess.CompletedProcess:
    here = os.path.dirname(os.path.abspath(__file__))
    code = _RUNNER.format(root=os.path.dirname(here), tests=here, lib=lib_path)
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)


@pytest.fixture(scope="module")
def mutant_runs(tmp_path_factory):
    d = str(tmp_path_factory.mktemp("mutants"))

    def one(item):
        name, (find, repl) = item
        return name, _run_pins(_build_mutant(d, name, find, repl))

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return dict(ex.map(one, MUTANTS.items()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(mutant_runs, name):
    # Non-zero exit: a pin failed, or the mutant crashed the process outright.
    proc = mutant_runs[name]
    assert proc.returncode != 0, f"no pin catches mutant {name}: {proc.stdout[-500:]}"


def test_unmutated_copy_passes(tmp_path):
    """Control: the same harness on an unmodified copy passes every pin."""
    lib = _build_mutant(str(tmp_path), "control", "#include <omp.h>", "#include <omp.h>")
    proc = _run_pins(lib)
    assert proc.returncode == 0, proc.stdout + proc.stderr
