// Capacity bounds of the bucket table, known before the length counts.
#pragma once

#include <stdint.h>

#include <cmath>

namespace bsort {

// The most distinct word lengths a document of len bytes can hold (each
// (document, length) with words is one bucket): k words of k different
// lengths take at least 1 + 2 + ... + k letters and k - 1 whitespace bytes
// between them, so the largest k with k(k + 1)/2 + k - 1 <= len, that is
// k(k + 3)/2 <= len + 1.
inline uint64_t max_distinct_lengths(uint64_t len) {
  uint64_t k = (uint64_t)((std::sqrt(8.0 * (double)len + 17.0) - 3.0) / 2.0);
  while (k > 0 && k * (k + 3) / 2 > len + 1) --k;
  while ((k + 1) * (k + 4) / 2 <= len + 1) ++k;
  return k;
}

}  // namespace bsort
