"""Host check of the byte-parallel character classes of the tokenize kernel
(csrc/swar.h): every 32-bit word, each of its four bytes against the plain
per-byte definition of Section II (letters A-Z a-z; whitespace ' ' and
0x09..0x0D; every other byte, 0x80..0xFF included, is neither).  The header
compiles as plain C++, so the same arithmetic the kernel runs is checked
here with g++."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1407_6603_gb300", "csrc")

CHECK = r"""
#include <cstdio>
#include "swar.h"
static bool is_letter(unsigned b) { return (b >= 'A' && b <= 'Z') || (b >= 'a' && b <= 'z'); }
static bool is_space(unsigned b) { return b == ' ' || (b >= 0x09 && b <= 0x0D); }
int main() {
  unsigned long long bad = 0;
  unsigned first = 0;
  bool seen = false;
  unsigned cls[256];
  for (unsigned b = 0; b < 256; ++b) cls[b] = (is_letter(b) ? 1u : 0u) | (is_space(b) ? 0x10u : 0u);
  for (unsigned long long v = 0; v <= 0xFFFFFFFFull; ++v) {
    const unsigned x = (unsigned)v;
    const unsigned c = bsort::class_nibbles(x);
    const unsigned want = cls[x & 0xFFu] | cls[(x >> 8) & 0xFFu] << 1 | cls[(x >> 16) & 0xFFu] << 2 | cls[x >> 24] << 3;
    if (c != want) {
      if (!seen) first = x;
      seen = true;
      ++bad;
    }
  }
  std::printf("%llu %08x\n", bad, first);
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_class_nibbles_every_word(tmp_path):
    src = tmp_path / "swar_check.cpp"
    src.write_text(CHECK)
    exe = tmp_path / "swar_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    bad, first = subprocess.run([str(exe)], capture_output=True, text=True, check=True, timeout=600).stdout.split()
    assert int(bad) == 0, f"{bad} words misclassified, first 0x{first}"
