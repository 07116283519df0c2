/*
 * Seeded synthetic text generator.
 *
 * This module produces the input documents only.  It holds none of the
 * sorting method's arithmetic (no stripping, no bucketing, no comparing):
 * both the CPU oracle and the CUDA path consume its bytes as plain input.
 *
 * The documents stand in for the paper's two Hamlet text files (Section II:
 * 190 KB and 1.38 MB of English text), which are not available here.  The
 * recipe imitates their shape: a vocabulary of distinct lower-case words whose
 * lengths follow 1 + Poisson(lambda) clipped to [1, lmax], a Zipf(1.07) token
 * draw, occasional capitalisation and trailing punctuation, single spaces
 * between tokens and a newline every 10..14 tokens.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both written from their published
 * definitions.  Every floating-point step uses plain double arithmetic; the
 * library is built with -ffp-contract=off so that x86_64 and aarch64 hosts
 * produce the same bytes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint64_t s[4];
} rng_t;

static uint64_t splitmix64_next(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t *r) {
  uint64_t *s = r->s;
  const uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return out;
}

/* One independent stream per (tag, seed, stream): the tag keeps workloads
 * apart that share a seed number (document i of the batch uses seed 3+i, the
 * serving stream uses seed 4). */
static void rng_init(rng_t *r, uint32_t tag, uint64_t seed, uint64_t stream) {
  uint64_t x = ((uint64_t)tag << 40) ^ (seed * 0xD6E8FEB86659FD93ull) ^ (stream * 0xA0761D6478BD642Full);
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

/* Uniform double in [0, 1) from the top 53 bits. */
static double rng_uniform(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* Poisson(lambda) by Knuth's multiplication method (lambda here is <= 6). */
static uint32_t rng_poisson(rng_t *r, double exp_neg_lambda) {
  uint32_t k = 0;
  double p = 1.0;
  do {
    ++k;
    p *= rng_uniform(r);
  } while (p > exp_neg_lambda);
  return k - 1;
}

/* ---- vocabulary of distinct words (open-addressing set of byte strings) ---- */

typedef struct {
  char *chars;      /* all words back to back */
  uint32_t *off;    /* word i = chars[off[i] .. off[i+1]) */
  uint32_t n;
  uint64_t *slots;  /* hash table: 0 = empty, else word index + 1 */
  uint64_t mask;
} vocab_t;

static uint64_t fnv1a(const char *p, uint32_t n) {
  uint64_t h = 0xCBF29CE484222325ull;
  for (uint32_t i = 0; i < n; ++i) {
    h ^= (unsigned char)p[i];
    h *= 0x100000001B3ull;
  }
  return h;
}

/* Inserts w if new; returns 1 when inserted, 0 when already present. */
static int vocab_insert(vocab_t *v, const char *w, uint32_t len) {
  uint64_t h = fnv1a(w, len) & v->mask;
  for (;;) {
    uint64_t s = v->slots[h];
    if (s == 0) break;
    uint32_t idx = (uint32_t)(s - 1);
    uint32_t l2 = v->off[idx + 1] - v->off[idx];
    if (l2 == len && memcmp(v->chars + v->off[idx], w, len) == 0) return 0;
    h = (h + 1) & v->mask;
  }
  uint32_t at = v->off[v->n];
  memcpy(v->chars + at, w, len);
  v->off[v->n + 1] = at + len;
  v->slots[h] = (uint64_t)v->n + 1;
  v->n += 1;
  return 1;
}

static int vocab_build(vocab_t *v, rng_t *r, uint32_t nwords, double lambda, uint32_t lmax) {
  uint64_t cap = 1;
  while (cap < 2ull * nwords + 2) cap <<= 1;
  v->slots = (uint64_t *)calloc(cap, sizeof(uint64_t));
  v->mask = cap - 1;
  v->chars = (char *)malloc((size_t)nwords * lmax + 1);
  v->off = (uint32_t *)malloc(((size_t)nwords + 1) * sizeof(uint32_t));
  v->n = 0;
  if (!v->slots || !v->chars || !v->off) return -1;
  v->off[0] = 0;
  const double e = exp(-lambda);
  char buf[256];
  uint64_t attempts = 0;
  while (v->n < nwords) {
    /* A repeated word is redrawn whole, its length included. */
    uint32_t len = 1 + rng_poisson(r, e);
    if (len > lmax) len = lmax;
    for (uint32_t i = 0; i < len; ++i) buf[i] = (char)('a' + (int)(rng_uniform(r) * 26.0));
    vocab_insert(v, buf, len);
    if (++attempts > 200ull * nwords + 100000ull) return -2; /* vocabulary cannot be that large */
  }
  return 0;
}

static void vocab_free(vocab_t *v) {
  free(v->chars);
  free(v->off);
  free(v->slots);
}

/* Zipf(s) over ranks 1..V: cumulative weights k^-s, drawn by binary search. */
static double *zipf_cdf(uint32_t V, double s) {
  double *c = (double *)malloc((size_t)V * sizeof(double));
  if (!c) return NULL;
  double acc = 0.0;
  for (uint32_t k = 0; k < V; ++k) {
    acc += pow((double)(k + 1), -s);
    c[k] = acc;
  }
  return c;
}

static uint32_t zipf_draw(const double *cdf, uint32_t V, double u) {
  const double x = u * cdf[V - 1];
  uint32_t lo = 0, hi = V - 1;
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo) / 2;
    if (cdf[mid] > x)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

static const char k_punct[9] = {',', '.', ';', ':', '?', '!', '"', '\'', '-'};

/*
 * Writes exactly nbytes of text into out.  Returns 0 on success, a negative
 * value on bad arguments or allocation failure.
 *   tag, seed : stream selection (see rng_init)
 *   vocab     : number of distinct words V
 *   lambda    : word length is 1 + Poisson(lambda), clipped to [1, lmax]
 *   zipf_s    : Zipf exponent of the token draw (1.07 for every workload)
 *   p_cap     : probability that a token's first letter is upper-cased
 *   p_punct   : probability that one punctuation byte trails a token
 */
int synth_text(uint32_t tag, uint64_t seed, uint64_t nbytes, uint32_t vocab, double lambda, uint32_t lmax,
               double zipf_s, double p_cap, double p_punct, uint8_t *out) {
  if (nbytes == 0) return 0;
  if (!out || vocab == 0 || lmax == 0 || lmax > 255) return -1;
  rng_t r;
  rng_init(&r, tag, seed, 0);
  vocab_t v;
  memset(&v, 0, sizeof(v));
  int rc = vocab_build(&v, &r, vocab, lambda, lmax);
  if (rc != 0) {
    vocab_free(&v);
    return rc;
  }
  double *cdf = zipf_cdf(vocab, zipf_s);
  if (!cdf) {
    vocab_free(&v);
    return -3;
  }
  uint64_t pos = 0;
  uint32_t line_left = 10 + (uint32_t)(rng_uniform(&r) * 5.0);
  while (pos < nbytes) {
    const uint32_t w = zipf_draw(cdf, vocab, rng_uniform(&r));
    const int cap = rng_uniform(&r) < p_cap;
    const int punct = rng_uniform(&r) < p_punct;
    const char *src = v.chars + v.off[w];
    const uint32_t len = v.off[w + 1] - v.off[w];
    for (uint32_t i = 0; i < len && pos < nbytes; ++i) {
      char c = src[i];
      if (i == 0 && cap) c = (char)(c - 'a' + 'A');
      out[pos++] = (uint8_t)c;
    }
    if (punct && pos < nbytes) out[pos++] = (uint8_t)k_punct[(int)(rng_uniform(&r) * 9.0)];
    if (pos < nbytes) {
      if (--line_left == 0) {
        out[pos++] = '\n';
        line_left = 10 + (uint32_t)(rng_uniform(&r) * 5.0);
      } else {
        out[pos++] = ' ';
      }
    }
  }
  free(cdf);
  vocab_free(&v);
  return 0;
}

/* Log-uniform document shape (byte size and vocabulary size) for the batched
 * and served workloads, from a stream separate from the text's. */
void synth_doc_shape(uint32_t tag, uint64_t seed, uint64_t nmin, uint64_t nmax, uint32_t vmin, uint32_t vmax,
                     uint64_t *n_out, uint32_t *v_out) {
  rng_t r;
  rng_init(&r, tag, seed, 1);
  const double un = rng_uniform(&r), uv = rng_uniform(&r);
  double n = exp(log((double)nmin) + un * (log((double)nmax) - log((double)nmin)));
  double v = exp(log((double)vmin) + uv * (log((double)vmax) - log((double)vmin)));
  uint64_t ni = (uint64_t)n;
  uint32_t vi = (uint32_t)v;
  if (ni < nmin) ni = nmin;
  if (ni > nmax) ni = nmax;
  if (vi < vmin) vi = vmin;
  if (vi > vmax) vi = vmax;
  *n_out = ni;
  *v_out = vi;
}

/* Poisson arrival times (seconds) at `rate` per second, for the request stream. */
void synth_arrivals(uint32_t tag, uint64_t seed, double rate, uint64_t count, double *t_out) {
  rng_t r;
  rng_init(&r, tag, seed, 2);
  double t = 0.0;
  for (uint64_t i = 0; i < count; ++i) {
    t += -log(1.0 - rng_uniform(&r)) / rate;
    t_out[i] = t;
  }
}
