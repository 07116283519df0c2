"""The rules the bucket layout is built by, on the host (no GPU).

The device layout (K2) and the host's plan of the launches both take a
bucket's sort group, the table order of the groups and the merge-pass count
from inline functions of csrc/bsort_dev.cuh.  This test compiles those
functions as plain C++ and checks them against their definitions:

* sort group of n keys of W words (T = keys of one K4 tile): groups 0..3 for
  W = 1, 2, 4, 8 and more than 8T keys; 5 for (4T, 8T]; 6 for (2T, 4T];
  7 for (T, 2T]; 8 for (32 x keys per thread, T]; 9 below that; 10 and 11
  for keys of 16 and 32 words;
* table order: every group once, groups 9, 10, 11 last, and groups 0..4
  together, just before the group whose K4 clusters make the merge runs (of
  `runs` tiles; before group 5 when runs exceed one cluster of 8), so that
  each K4 launch and each merge chain covers one contiguous range;
* merge passes: the doublings that take runs of `tile` keys to one run of n;
* ceil(log2 n);
* the bucket table's capacity per document (layout_bounds.h): the most
  distinct word lengths len bytes can hold, against a search over every set
  of lengths for small documents.
"""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1407_6603_gb300", "csrc")

PROGRAM = r"""
#include "bsort_dev.cuh"
#include "layout_bounds.h"
#include <cstdio>
int main() {
  using namespace bsort;
  int order[kGroups], pos[kGroups];
  for (uint32_t runs : {1u, 2u, 4u, 8u, 16u}) {
    table_order(runs, order, pos);
    printf("order %u", runs);
    for (int i = 0; i < kGroups; ++i) printf(" %d", order[i]);
    printf("\n");
    for (int g = 0; g < kGroups; ++g) printf("pos %u %d %d\n", runs, g, pos[g]);
  }
  for (int W : {1, 2, 4, 8, 16, 32}) {
    const uint32_t T = tile2_keys(W), wk = warp_keys(W);
    for (uint32_t n : {1u, wk, wk + 1, T, T + 1, 2 * T, 2 * T + 1, 4 * T, 4 * T + 1, 8 * T, 8 * T + 1, 100000u,
                       4000000000u})
      printf("group %d %u %d %u %u\n", W, n, sort_group(n, W), T, wk);
  }
  for (uint64_t n : {1ull, 255ull, 256ull, 257ull, 512ull, 513ull, 100000ull, 4000000000ull})
    for (uint64_t tile : {256ull, 2048ull, 16384ull})
      printf("passes %llu %llu %u\n", (unsigned long long)n, (unsigned long long)tile, merge_passes(n, tile));
  for (uint64_t n : {0ull, 1ull, 2ull, 3ull, 4ull, 5ull, 1023ull, 1024ull, 1025ull, (1ull << 40) + 1})
    printf("clog %llu %u\n", (unsigned long long)n, ceil_log2_u(n));
  for (uint64_t len = 0; len <= 300; ++len)
    printf("mdl %llu %llu\n", (unsigned long long)len, (unsigned long long)max_distinct_lengths(len));
  for (uint64_t len : {1000ull, 1447000ull, 268435456ull, 4294967295ull})
    printf("mdl %llu %llu\n", (unsigned long long)len, (unsigned long long)max_distinct_lengths(len));
  return 0;
}
"""


def _cuda_include():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            return os.path.join(cand, "include")
    nv = shutil.which("nvcc")
    if nv:
        inc = os.path.join(os.path.dirname(os.path.dirname(nv)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


@pytest.fixture(scope="module")
def rules(tmp_path_factory):
    gxx, inc = shutil.which("g++"), _cuda_include()
    if not gxx or not inc:
        pytest.skip("g++ or the CUDA headers are missing")
    d = tmp_path_factory.mktemp("layout_rules")
    src, exe = d / "rules.cpp", d / "rules"
    src.write_text(PROGRAM)
    subprocess.run([gxx, "-std=c++17", "-O1", f"-I{inc}", f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}",
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return [line.split() for line in out.splitlines()]


def test_sort_groups_follow_their_thresholds(rules):
    seen = 0
    for r in (r for r in rules if r[0] == "group"):
        W, n, g, T, wk = (int(x) for x in r[1:])
        assert T == (256 if W >= 16 else 2048 // W)
        if W >= 16:
            want = 10 if W == 16 else 11
        elif n <= wk:
            want = 9
        elif n <= T:
            want = 8
        elif n <= 2 * T:
            want = 7
        elif n <= 4 * T:
            want = 6
        elif n <= 8 * T:
            want = 5
        else:
            want = {1: 0, 2: 1, 4: 2, 8: 3}[W]
        assert g == want, (W, n)
        seen += 1
    assert seen == 6 * 13


def test_table_order_keeps_each_launch_contiguous(rules):
    orders = {int(r[1]): [int(x) for x in r[2:]] for r in rules if r[0] == "order"}
    assert sorted(orders) == [1, 2, 4, 8, 16]
    for runs, order in orders.items():
        assert sorted(order) == list(range(12))
        assert order[-3:] == [9, 10, 11]
        at = order.index(0)
        assert order[at:at + 5] == [0, 1, 2, 3, 4]
        # the group after them is the one whose clusters (8, 4, 2, 1 CTAs for
        # groups 5..8) make runs of `runs` tiles, group 5 for runs of 16
        nxt = order[at + 5]
        assert nxt == (5 if runs == 16 else {8: 5, 4: 6, 2: 7, 1: 8}[runs])
        # the groups K4 finishes keep the order of their cluster sizes
        assert [g for g in order if 5 <= g <= 8] == [5, 6, 7, 8]
        pos = {int(r[2]): int(r[3]) for r in rules if r[0] == "pos" and int(r[1]) == runs}
        assert all(order[pos[g]] == g for g in range(12))


def test_merge_passes_and_ceil_log2(rules):
    for r in (r for r in rules if r[0] == "passes"):
        n, tile, p = (int(x) for x in r[1:])
        runs = -(-n // tile)
        assert p == (0 if runs <= 1 else math.ceil(math.log2(runs))), (n, tile)
        assert tile << p >= n and (p == 0 or tile << (p - 1) < n)
    for r in (r for r in rules if r[0] == "clog"):
        n, v = int(r[1]), int(r[2])
        assert v == (0 if n <= 1 else (n - 1).bit_length()), n


def test_distinct_length_bound(rules):
    mdl = {int(r[1]): int(r[2]) for r in rules if r[0] == "mdl"}
    # small documents: the largest set of distinct lengths whose words fit,
    # each word its letters and one whitespace byte before every word but the first
    for length in range(0, 17):
        best = 0
        for mask in range(1 << length):
            ls = [i + 1 for i in range(length) if mask >> i & 1]
            if ls and sum(ls) + len(ls) - 1 <= length:
                best = max(best, len(ls))
        assert mdl[length] == best, length
    # every size: the largest k with k(k + 1)/2 + k - 1 <= len, never decreasing
    prev = 0
    for length, k in sorted(mdl.items()):
        assert k * (k + 1) // 2 + k - 1 <= length or k == 0
        assert (k + 1) * (k + 2) // 2 + k > length
        assert k >= prev
        prev = k
    assert mdl[1000] == 43 and mdl[1447000] == 1699
