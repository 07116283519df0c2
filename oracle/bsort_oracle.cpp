// ORACLE — test infrastructure, not product code.
//
// A plain, slow, obviously correct CPU restatement of the length-bucketed
// bubble sort of a text's words from "Parallelize Bubble Sort Algorithm Using
// OpenMP" (arXiv 1407.6603).  Only the tests, the smoke check and the CPU
// baseline of the benchmark may load it; the CUDA library shares no code,
// header or table with it.
//
// What it computes (Section II "Pre-processing", three phases; Section III
// "Approach one", steps 1-4):
//   1. strip: remove the special characters from the text (every byte that
//      is not an ASCII letter), with whitespace separating the words;
//   2. bucket: put the words in sub-arrays by their number of characters,
//      shorter words first, the sub-array sizes being the per-length counts;
//   3. sort: bubble sort each sub-array by the ASCII codes of its letters;
//   4. emit: the buckets in ascending length, concatenated.
//
// Two independent paths compute the same result:
//   O1 (oracle_bubble): a state-machine tokenizer, the paper's 3-D char
//      array (one contiguous [count][L] block per length, Section III
//      "Approach Second"), textbook bubble sort with early exit on each block
//      (Section I), OpenMP over the buckets as in Section "Bubble sort in
//      OpenMP" (one bucket per thread, no dependence between buckets).
//   O2 (oracle_stable): a split-then-filter tokenizer and std::stable_sort by
//      (length, bytes), for inputs too large for an O(n^2) sort.
//
// Readings of the paper (it gives only examples of the special characters
// and prints no listing of its sort):
//   * a letter is a byte in [A-Za-z]; whitespace is 0x20 and 0x09..0x0D;
//     every other byte (digits, punctuation, bytes >= 0x80) is deleted from
//     inside its word, it does not split words ("don't" -> "dont");
//   * words that are empty after stripping are dropped;
//   * order is by unsigned byte value with case kept ("Zebra" < "apple");
//     duplicates are kept;
//   * bucket lengths run 1..max_len; counts[0] is always 0.
#include <omp.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

extern "C" {

// Result layout mirrors the boundary's output (counts, offsets, stream) but
// is declared here on its own.
typedef struct {
  uint32_t max_len;       // longest word after stripping, 0 if there is none
  uint64_t n_words;       // number of words kept
  uint64_t stream_bytes;  // total letters kept
  uint64_t* counts;       // [max_len + 1]; counts[L] = words of length L
  uint32_t* offsets;      // [n_words + 1]; word j = stream[offsets[j] .. offsets[j+1])
  uint8_t* stream;        // sorted words back to back, no separators
  uint64_t compares;      // O1 only: adjacent comparisons made by bubble sort
  uint64_t swaps;         // O1 only: exchanges made by bubble sort
} oracle_result;

}  // extern "C"

namespace {

bool is_space(uint8_t c) { return c == 0x20 || (c >= 0x09 && c <= 0x0D); }
bool is_letter(uint8_t c) { return (c >= 'A' && c <= 'Z') || (c >= 'a' && c <= 'z'); }

// ---------------------------------------------------------------- O1 ----

// Tokenizer A (phase 1): one left-to-right pass.  Whitespace closes the
// current word if it has letters; a letter is appended; anything else is
// skipped.
std::vector<std::string> tokenize_state_machine(const uint8_t* b, uint64_t n) {
  std::vector<std::string> words;
  std::string cur;
  for (uint64_t i = 0; i < n; ++i) {
    const uint8_t c = b[i];
    if (is_space(c)) {
      if (!cur.empty()) {
        words.push_back(cur);
        cur.clear();
      }
    } else if (is_letter(c)) {
      cur.push_back(static_cast<char>(c));
    }
  }
  if (!cur.empty()) words.push_back(cur);
  return words;
}

// ASCII order of two equal-length rows: first differing byte decides, bytes
// compared as unsigned values.  Returns true when row a must come after b.
bool row_greater(const uint8_t* a, const uint8_t* b, uint32_t len) {
  for (uint32_t i = 0; i < len; ++i) {
    if (a[i] != b[i]) return a[i] > b[i];
  }
  return false;
}

// Bubble sort of `count` rows of `len` bytes stored back to back (one plane
// of the 3-D char array).  Adjacent rows are compared and exchanged when out
// of order; passes repeat until one makes no exchange.  Pass p needs only
// count-1-p comparisons, as the largest p rows have sunk to the end, which
// gives n(n-1)/2 comparisons in the worst case.
void bubble_sort_rows(uint8_t* rows, uint64_t count, uint32_t len, uint64_t* compares, uint64_t* swaps) {
  std::vector<uint8_t> tmp(len);
  for (uint64_t pass = 0; pass + 1 < count; ++pass) {
    bool swapped = false;
    for (uint64_t j = 0; j + 1 < count - pass; ++j) {
      uint8_t* a = rows + j * len;
      uint8_t* b = a + len;
      ++*compares;
      if (row_greater(a, b, len)) {
        std::memcpy(tmp.data(), a, len);
        std::memcpy(a, b, len);
        std::memcpy(b, tmp.data(), len);
        ++*swaps;
        swapped = true;
      }
    }
    if (!swapped) break;
  }
}

// ---------------------------------------------------------------- O2 ----

// Tokenizer B (phase 1), written differently from A: first cut the text into
// whitespace-separated fields, then keep each field's letters, then drop the
// fields left empty.
std::vector<std::string> tokenize_split_filter(const uint8_t* b, uint64_t n) {
  std::vector<std::pair<uint64_t, uint64_t>> fields;  // [begin, end)
  uint64_t i = 0;
  while (i < n) {
    while (i < n && is_space(b[i])) ++i;
    const uint64_t begin = i;
    while (i < n && !is_space(b[i])) ++i;
    if (i > begin) fields.emplace_back(begin, i);
  }
  std::vector<std::string> words;
  words.reserve(fields.size());
  for (const auto& f : fields) {
    std::string w;
    for (uint64_t k = f.first; k < f.second; ++k)
      if (is_letter(b[k])) w.push_back(static_cast<char>(b[k]));
    if (!w.empty()) words.push_back(std::move(w));
  }
  return words;
}

bool bytes_less(const std::string& a, const std::string& b) {
  return std::lexicographical_compare(a.begin(), a.end(), b.begin(), b.end(), [](char x, char y) {
    return static_cast<unsigned char>(x) < static_cast<unsigned char>(y);
  });
}

// ------------------------------------------------------------- output ----

int fill_result(const std::vector<std::vector<std::string>>& buckets, oracle_result* out) {
  uint32_t max_len = 0;
  uint64_t n_words = 0, bytes = 0;
  for (size_t L = 1; L < buckets.size(); ++L) {
    if (!buckets[L].empty()) max_len = static_cast<uint32_t>(L);
    n_words += buckets[L].size();
    bytes += buckets[L].size() * L;
  }
  out->max_len = max_len;
  out->n_words = n_words;
  out->stream_bytes = bytes;
  out->counts = static_cast<uint64_t*>(std::calloc(max_len + 1, sizeof(uint64_t)));
  out->offsets = static_cast<uint32_t*>(std::malloc((n_words + 1) * sizeof(uint32_t)));
  out->stream = static_cast<uint8_t*>(std::malloc(bytes ? bytes : 1));
  if (!out->counts || !out->offsets || !out->stream) return -2;
  uint64_t j = 0, pos = 0;
  for (uint32_t L = 1; L <= max_len; ++L) {
    out->counts[L] = buckets[L].size();
    for (const std::string& w : buckets[L]) {
      out->offsets[j++] = static_cast<uint32_t>(pos);
      std::memcpy(out->stream + pos, w.data(), L);
      pos += L;
    }
  }
  out->offsets[j] = static_cast<uint32_t>(pos);
  return 0;
}

}  // namespace

extern "C" {

// O1: strip, bucket into the 3-D char array, bubble sort every bucket with
// `nthreads` OpenMP threads (one bucket per thread at a time), emit.
// Returns 0, or -1 on bad arguments / -2 on allocation failure.
int oracle_bubble(const uint8_t* bytes, uint64_t len, int nthreads, oracle_result* out) {
  if (!out || (!bytes && len)) return -1;
  std::memset(out, 0, sizeof(*out));
  const std::vector<std::string> words = tokenize_state_machine(bytes, len);
  size_t longest = 0;
  for (const auto& w : words) longest = std::max(longest, w.size());
  // Sizes of the sub-arrays are the per-length counts (Section II).
  std::vector<uint64_t> count(longest + 1, 0);
  for (const auto& w : words) ++count[w.size()];
  // The 3-D char array: plane L holds count[L] rows of L bytes.
  std::vector<std::vector<uint8_t>> plane(longest + 1);
  std::vector<uint64_t> fill(longest + 1, 0);
  for (size_t L = 1; L <= longest; ++L) plane[L].resize(count[L] * L);
  for (const auto& w : words) {
    const size_t L = w.size();
    std::memcpy(plane[L].data() + fill[L] * L, w.data(), L);
    ++fill[L];
  }
  uint64_t compares = 0, swaps = 0;
  const long nb = static_cast<long>(longest);
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 1) reduction(+ : compares, swaps)
  for (long L = 1; L <= nb; ++L) {
    uint64_t c = 0, s = 0;
    bubble_sort_rows(plane[L].data(), count[L], static_cast<uint32_t>(L), &c, &s);
    compares += c;
    swaps += s;
  }
  std::vector<std::vector<std::string>> buckets(longest + 1);
  for (size_t L = 1; L <= longest; ++L) {
    buckets[L].reserve(count[L]);
    for (uint64_t r = 0; r < count[L]; ++r)
      buckets[L].emplace_back(reinterpret_cast<const char*>(plane[L].data() + r * L), L);
  }
  const int rc = fill_result(buckets, out);
  out->compares = compares;
  out->swaps = swaps;
  return rc;
}

// O2: strip with tokenizer B, group by length (a stable partition), then
// std::stable_sort each group by its bytes; OpenMP over the groups.  The
// result equals one std::stable_sort of all words by (length, bytes).
int oracle_stable(const uint8_t* bytes, uint64_t len, int nthreads, oracle_result* out) {
  if (!out || (!bytes && len)) return -1;
  std::memset(out, 0, sizeof(*out));
  std::vector<std::string> words = tokenize_split_filter(bytes, len);
  size_t longest = 0;
  for (const auto& w : words) longest = std::max(longest, w.size());
  std::vector<std::vector<std::string>> buckets(longest + 1);
  for (auto& w : words) buckets[w.size()].push_back(std::move(w));
  const long nb = static_cast<long>(longest);
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 1)
  for (long L = 1; L <= nb; ++L) std::stable_sort(buckets[L].begin(), buckets[L].end(), bytes_less);
  return fill_result(buckets, out);
}

// Phase 1 alone (tokenizer A): the stripped words in input order, back to
// back, with their lengths.  Returns the word count, or -1 / -2 on error.
int64_t oracle_tokenize(const uint8_t* bytes, uint64_t len, uint8_t** letters_out, uint32_t** lengths_out) {
  if (!letters_out || !lengths_out || (!bytes && len)) return -1;
  const std::vector<std::string> words = tokenize_state_machine(bytes, len);
  uint64_t total = 0;
  for (const auto& w : words) total += w.size();
  *letters_out = static_cast<uint8_t*>(std::malloc(total ? total : 1));
  *lengths_out = static_cast<uint32_t*>(std::malloc(words.empty() ? 4 : words.size() * 4));
  if (!*letters_out || !*lengths_out) return -2;
  uint64_t pos = 0;
  for (size_t i = 0; i < words.size(); ++i) {
    std::memcpy(*letters_out + pos, words[i].data(), words[i].size());
    pos += words[i].size();
    (*lengths_out)[i] = static_cast<uint32_t>(words[i].size());
  }
  return static_cast<int64_t>(words.size());
}

// ------------------------------------------------------ other orders ----
//
// The same words in the other orders the paper names or leaves open:
//   order 1, folded: length buckets (Section II phase 2), each in alphabetic
//            order: letters compared with case ignored, and words whose
//            letters agree that way in ASCII order (a reading of "alphabetic
//            order", Section II phase 3, against "ASCII code for each
//            letter", Section III step 4);
//   order 2, whole: no length buckets: all words in ASCII order, a word
//            before every longer word it begins (Table 1, "bubble sort based
//            on alphabetic order");
//   order 3, length: length buckets, each in input order (Table 1, "bubble
//            sort based on the length of the word": bubble sort exchanges
//            only on a strictly greater length, so equal lengths keep their
//            order).
// O1 (oracle_bubble_order) bubble sorts with the order's comparison: each
// length bucket for orders 1 and 3 (every comparison inside a bucket of
// order 3 finds equal lengths, so a bucket stays in input order), all words
// at once for order 2.  O2 (oracle_stable_order) uses std::stable_sort with
// the same comparisons.

namespace {

unsigned char fold(char c) { return static_cast<unsigned char>((c >= 'A' && c <= 'Z') ? c + 32 : c); }

// order 1 within one length: case-blind letters first, then ASCII
bool folded_less(const std::string& a, const std::string& b) {
  for (size_t i = 0; i < a.size() && i < b.size(); ++i)
    if (fold(a[i]) != fold(b[i])) return fold(a[i]) < fold(b[i]);
  if (a.size() != b.size()) return a.size() < b.size();
  return bytes_less(a, b);
}

// true when a must come after b under `order`
bool order_greater(int order, const std::string& a, const std::string& b) {
  switch (order) {
    case 1: return folded_less(b, a);
    case 2: return bytes_less(b, a);      // lexicographic by unsigned bytes: a prefix comes first
    case 3: return a.size() > b.size();
    default: return bytes_less(b, a);
  }
}

// Textbook bubble sort of whole words (Section I), early exit as above.
void bubble_sort_words(std::vector<std::string>& v, int order) {
  for (size_t sweep = 1; sweep < v.size(); ++sweep) {
    bool moved = false;
    for (size_t j = 0; j + sweep < v.size(); ++j)
      if (order_greater(order, v[j], v[j + 1])) {
        std::swap(v[j], v[j + 1]);
        moved = true;
      }
    if (!moved) return;
  }
}

// Counts per length as in fill_result; offsets and stream in the order of `words`.
int fill_flat(const std::vector<std::string>& words, oracle_result* out) {
  uint32_t max_len = 0;
  uint64_t bytes = 0;
  for (const auto& w : words) {
    max_len = std::max<uint32_t>(max_len, static_cast<uint32_t>(w.size()));
    bytes += w.size();
  }
  out->max_len = max_len;
  out->n_words = words.size();
  out->stream_bytes = bytes;
  out->counts = static_cast<uint64_t*>(std::calloc(max_len + 1, sizeof(uint64_t)));
  out->offsets = static_cast<uint32_t*>(std::malloc((words.size() + 1) * sizeof(uint32_t)));
  out->stream = static_cast<uint8_t*>(std::malloc(bytes ? bytes : 1));
  if (!out->counts || !out->offsets || !out->stream) return -2;
  uint64_t pos = 0;
  for (size_t j = 0; j < words.size(); ++j) {
    ++out->counts[words[j].size()];
    out->offsets[j] = static_cast<uint32_t>(pos);
    std::memcpy(out->stream + pos, words[j].data(), words[j].size());
    pos += words[j].size();
  }
  out->offsets[words.size()] = static_cast<uint32_t>(pos);
  return 0;
}

}  // namespace

// O1 for every order (0 as oracle_bubble, without its counters): bubble sort
// per length bucket, OpenMP over the buckets, or (order 2) of all words.
int oracle_bubble_order(const uint8_t* bytes, uint64_t len, int order, int nthreads, oracle_result* out) {
  if (!out || (!bytes && len) || order < 0 || order > 3) return -1;
  std::memset(out, 0, sizeof(*out));
  std::vector<std::string> words = tokenize_state_machine(bytes, len);
  if (order == 2) {
    bubble_sort_words(words, 2);
    return fill_flat(words, out);
  }
  size_t longest = 0;
  for (const auto& w : words) longest = std::max(longest, w.size());
  std::vector<std::vector<std::string>> buckets(longest + 1);
  for (auto& w : words) buckets[w.size()].push_back(std::move(w));
  const long nb = static_cast<long>(longest);
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 1)
  for (long L = 1; L <= nb; ++L) bubble_sort_words(buckets[L], order);
  return fill_result(buckets, out);
}

// O2 for every order: tokenizer B, then std::stable_sort with the order's
// comparison (per length bucket, or all words for order 2).
int oracle_stable_order(const uint8_t* bytes, uint64_t len, int order, int nthreads, oracle_result* out) {
  if (!out || (!bytes && len) || order < 0 || order > 3) return -1;
  std::memset(out, 0, sizeof(*out));
  std::vector<std::string> words = tokenize_split_filter(bytes, len);
  auto less = [order](const std::string& a, const std::string& b) { return order_greater(order, b, a); };
  if (order == 2) {
    std::stable_sort(words.begin(), words.end(), less);
    return fill_flat(words, out);
  }
  size_t longest = 0;
  for (const auto& w : words) longest = std::max(longest, w.size());
  std::vector<std::vector<std::string>> buckets(longest + 1);
  for (auto& w : words) buckets[w.size()].push_back(std::move(w));
  const long nb = static_cast<long>(longest);
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 1)
  for (long L = 1; L <= nb; ++L) std::stable_sort(buckets[L].begin(), buckets[L].end(), less);
  return fill_result(buckets, out);
}

void oracle_free(oracle_result* r) {
  if (!r) return;
  std::free(r->counts);
  std::free(r->offsets);
  std::free(r->stream);
  r->counts = nullptr;
  r->offsets = nullptr;
  r->stream = nullptr;
}

void oracle_free_buffer(void* p) { std::free(p); }

int oracle_max_threads(void) { return omp_get_max_threads(); }

}  // extern "C"
