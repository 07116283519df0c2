// Character classes of four bytes at once in a 32-bit word, for the strip +
// tokenize step (Section II: a word is a run of letters; spaces, tabs and
// line breaks separate words; every other byte is dropped).
//
// Plain integer arithmetic, no byte-SIMD intrinsics: each byte is first
// masked to 7 bits so that adding a per-byte constant cannot carry into the
// next byte; bit 7 of the sum then says whether the byte reached a threshold.
// Bytes of 0x80 and above belong to neither class.  The header compiles as
// plain C++ too, so its tests run on the host.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define BSORT_HD __host__ __device__ __forceinline__
#else
#define BSORT_HD inline
#endif

namespace bsort {

// Bit 7 of byte k is set iff byte k of x is an ASCII letter (A-Z, a-z).
BSORT_HD uint32_t letter_bits(uint32_t x) {
  const uint32_t y = x | 0x20202020u;       // upper case folds onto lower case
  const uint32_t t = y & 0x7F7F7F7Fu;
  const uint32_t ge_a = t + 0x1F1F1F1Fu;    // bit 7: t >= 'a' (0x61)
  const uint32_t ge_brace = t + 0x05050505u;  // bit 7: t >= '{' (0x7B)
  return ge_a & ~ge_brace & ~y & 0x80808080u;
}

// Bit 7 of byte k is set iff byte k of x is whitespace: ' ' or one of
// '\t' '\n' '\v' '\f' '\r' (0x09..0x0D).
BSORT_HD uint32_t space_bits(uint32_t x) {
  const uint32_t t = x & 0x7F7F7F7Fu;
  const uint32_t ne_sp = (t ^ 0x20202020u) + 0x7F7F7F7Fu;  // bit 7: t != ' '
  const uint32_t ge_tab = t + 0x77777777u;                 // bit 7: t >= 0x09
  const uint32_t ge_so = t + 0x72727272u;                  // bit 7: t >= 0x0E
  return (~ne_sp | (ge_tab & ~ge_so)) & ~x & 0x80808080u;
}

// Both classes of four bytes as two nibbles: bits 0..3 the letters, bits
// 4..7 the whitespace (bit k of a nibble = byte k).  One multiply gathers
// the flags: with letters in bit 7 and whitespace in bit 3 of each byte, the
// multiplier 1 + 2^7 + 2^14 + 2^21 moves byte k's flags to bits 28+k and
// 24+k, and no two partial products share a bit, so nothing carries.
BSORT_HD uint32_t class_nibbles(uint32_t x) {
  const uint32_t p = (letter_bits(x) | (space_bits(x) >> 4)) * 0x00204081u;
  return ((p >> 28) & 0xFu) | ((p >> 20) & 0xF0u);
}

}  // namespace bsort
