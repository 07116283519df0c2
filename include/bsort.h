/*
 * bsort.h — C ABI of the GB300 length-bucketed word sort.
 *
 * The operation (arXiv 1407.6603, Section II "Pre-processing", three phases;
 * Section III "Approach one", steps 1-4):
 *   1. strip the special characters from a text: every byte that is not an
 *      ASCII letter [A-Za-z] is deleted, and whitespace (0x20, 0x09..0x0D)
 *      separates words; words left empty are dropped;
 *   2. put the words in buckets by their number of characters, shorter
 *      buckets first (the bucket sizes are the per-length counts);
 *   3. sort each bucket by the ASCII codes of its letters (unsigned byte
 *      order, case kept, duplicates kept).
 * The result is unique: two equal-length words compare equal only when they
 * are the same bytes, so every correct sort returns the same stream.
 *
 * Every step runs in CUDA kernels on one GPU (sm_103a).  There is no CPU
 * fallback: a context cannot be created without a CUDA device.
 *
 * Conventions for every function below:
 *   - No call aborts or throws.  Each returns a bsort_status; the message of
 *     the last failure on a context is available from bsort_last_error().
 *   - A failed call leaves its output struct(s) zeroed.
 *   - A context is not thread-safe: one host thread at a time.
 *   - Host-side fault injection for tests: the environment variable
 *     BSORT_FAULT=alloc makes every allocation a call needs fail
 *     (BSORT_E_NOMEM), BSORT_FAULT=timeout makes every call report a bounded
 *     device wait as run out (BSORT_E_TIMEOUT); both leave the context usable.
 *   - Output buffers belong to the context.  They stay valid until the next
 *     bsort_text / bsort_text_device / bsort_batch call on the same context,
 *     bsort_result_release() or bsort_destroy(), whichever comes first.
 */
#ifndef BSORT_H
#define BSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsort_ctx bsort_ctx; /* opaque */

typedef enum {
  BSORT_OK = 0,
  BSORT_E_INVAL = 1,         /* a NULL pointer where one is required, or a bad config value */
  BSORT_E_NOMEM = 2,         /* device or pinned host memory could not be allocated */
  BSORT_E_CUDA = 3,          /* a CUDA runtime call or a kernel launch failed */
  BSORT_E_TOO_LARGE = 4,     /* a document of 2^32 bytes or more (offsets are 32-bit) */
  BSORT_E_WORD_TOO_LONG = 5, /* a word longer than the context's l_cap letters */
  BSORT_E_TIMEOUT = 6,       /* a bounded device-side wait gave up (the context stays usable) */
  BSORT_E_BUSY = 7           /* the context is in use by another call */
} bsort_status;

/* Context configuration.  Fill with bsort_config_default() and change fields. */
typedef struct {
  uint32_t l_cap;        /* longest word accepted, 1..255 letters (default 255).  A longer word
                            makes the call fail with BSORT_E_WORD_TOO_LONG. */
  int32_t want_offsets;  /* 1 (default): produce per-word offsets; 0: counts and stream only */
  int32_t device;        /* CUDA device ordinal; -1 (default) = the current device */
  int32_t profile;       /* 1: time every kernel launch with CUDA events (see bsort_profile_read);
                            0 (default): no events are recorded */
  uint64_t wait_limit;   /* iteration limit of every device-side spin wait on other CTAs
                            (0 = default, about a second); when one runs out the call returns
                            BSORT_E_TIMEOUT (the device entry points: see bsort_device_finish).
                            A CTA's wait for its own bulk copy into shared memory never gives up
                            sooner than the default, whatever this value. */
  const char* tune_table; /* NULL (default): built-in tuning.  Otherwise text of `key=value`
                            items separated by spaces, semicolons or newlines, '#' to end of
                            line a comment (the autotuner, paper_1407_6603_gb300/autotune.py,
                            writes it):
                              k4_lanes=a,b,c,d  lanes per odd-even transposition group of the
                                                tile sort (the odd-even/merge cutoff: runs of
                                                lanes x keys-per-thread keys leave odd-even
                                                transposition) for buckets sorted by clusters
                                                of 1, 2, 4 and 8 CTAs; each 2, 4 or 8
                              k4_threads=a,b,c,d  threads per tile-sort CTA (256 or 512; 512
                                                takes effect for launches whose keys are at
                                                most 4 words) for the same classes: keys per
                                                thread 2048 / (threads x key words)
                              piped_min=k       merge passes with at least k tiles per resident
                                                CTA use the pipelined merge (1..1000000)
                              k4_runs=c         buckets too large for one cluster of 8 tiles
                                                are sorted by K4 into runs of c tiles (clusters
                                                of c CTAs: 1, 2, 4 or 8), which the merge
                                                passes take up, when their merges are large
                                                enough to be pipelined (see piped_min); else
                                                into runs of k4_runs_small tiles
                              k4_runs_small=8|16  that run for the smaller merges (16: clusters
                                                of 16 CTAs, beyond the portable cluster size)
                              dedupe=0|1|2      the duplicate-aware sort for the buckets too
                                                large for one cluster of 8 tiles (keys of up
                                                to 8 words): 1 (default) on inputs whose
                                                merges would be pipelined (see piped_min;
                                                smaller ones gain nothing), 2 always, 0
                                                never (merge passes).  The tile sort hands
                                                each sorted run's distinct words, with their
                                                counts, to a hash table per bucket; the
                                                distinct words are sorted and written out
                                                count times each.  The result is the same
                                                either way.
                              k4_streams=0|1    1 (default): the tile sort that makes the
                                                merge passes' runs runs first on the call's
                                                stream, the others beside it on side
                                                streams; 0: one after another on the call's
                                                stream (how the autotuner times a class)
                            Copied at bsort_create; an unknown key or a bad value makes
                            bsort_create fail with BSORT_E_INVAL. */
  uint32_t order;        /* bsort_order: the order of the result (default BSORT_ORDER_ASCII) */
  uint32_t key_pack;     /* bsort_key_pack: how the sort kernels encode a word's letters; it
                            changes the speed, not the result (default BSORT_KEYS_BYTES) */
} bsort_config;

/* Orders of the result.  Each one's oracle and reading of the paper: */
typedef enum {
  BSORT_ORDER_ASCII = 0,  /* length buckets, shorter first, each sorted by the ASCII codes of its
                             letters (Section III step 4): the paper's method */
  BSORT_ORDER_FOLDED = 1, /* length buckets, each in alphabetic order: letters compared with case
                             ignored, words whose letters then agree in ASCII order (a reading of
                             Section II phase 3, "alphabetic order") */
  BSORT_ORDER_WHOLE = 2,  /* no length buckets: every word in ASCII order, a word before each
                             longer word it begins (Table 1, bubble sort of the file "based on
                             alphabetic order") */
  BSORT_ORDER_LENGTH = 3  /* length buckets, each in input order: a stable sort by length alone
                             (Table 1, bubble sort "based on the length of the word") */
} bsort_order;

/* Key encodings of the sort kernels (an option of the GPU path; the paper
 * sorts characters): */
typedef enum {
  BSORT_KEYS_BYTES = 0,   /* one byte a letter, 8 letters a 64-bit key word */
  BSORT_KEYS_LETTERS6 = 1 /* six bits a letter (A..Z, a..z in ASCII order), 10 letters a key word:
                             fewer key bytes to move for words of 9, 10, 17..21, 33..42 letters */
} bsort_key_pack;

/*
 * One document's result.
 *   counts[L], 0 <= L <= max_len: number of words of L letters; counts[0] == 0.
 *   stream: the sorted words back to back, no separators: bucket 1 first,
 *           each bucket in ascending unsigned byte order (in the context's
 *           bsort_order: the words of every order but BSORT_ORDER_WHOLE still
 *           come in length buckets, shorter first).
 *   offsets[j], 0 <= j <= n_words: word j is stream[offsets[j] .. offsets[j+1]);
 *           offsets[0] == 0 and offsets[n_words] == stream_bytes.  NULL when the
 *           context was created with want_offsets == 0.
 * A document with no words has max_len 0, counts = {0}, offsets = {0} and an
 * empty stream.
 */
typedef struct {
  uint32_t max_len;         /* longest word, 0 if there is none */
  uint32_t status;          /* bsort_status of this document (batch calls) */
  uint64_t n_words;         /* number of words */
  uint64_t stream_bytes;    /* total letters = sum over L of L * counts[L] */
  const uint64_t* counts;   /* [max_len + 1] */
  const uint32_t* offsets;  /* [n_words + 1] or NULL */
  const uint8_t* stream;    /* [stream_bytes] */
} bsort_result;

/* Default configuration: l_cap 255, offsets on, current device, default wait limit,
 * built-in tuning, ASCII order, byte keys. */
void bsort_config_default(bsort_config* cfg);

/*
 * Creates a context on the configured device (cfg may be NULL for the
 * defaults).  The context owns a CUDA stream, a device arena and pinned host
 * buffers, all grown on demand.  Errors: BSORT_E_INVAL (out == NULL or a bad
 * config value), BSORT_E_CUDA (no usable device), BSORT_E_NOMEM.
 */
bsort_status bsort_create(bsort_ctx** out, const bsort_config* cfg);

/* Frees everything the context owns.  NULL is accepted. */
void bsort_destroy(bsort_ctx* ctx);

/* Message of the last failure on ctx ("" if none); valid until the next call on ctx. */
const char* bsort_last_error(const bsort_ctx* ctx);

/*
 * Sorts one document held in host memory (bytes may be NULL when len == 0).
 * Synchronous: on return, *out holds HOST pointers into buffers owned by the
 * context.  When the document lies in page-locked memory (cudaHostAlloc,
 * cudaHostRegister; its first and last bytes are checked, so a buffer must not
 * straddle page-locked and pageable memory) the copy engine reads it in
 * place; otherwise it is first copied into the context's page-locked staging
 * buffer.  Errors: BSORT_E_INVAL, BSORT_E_TOO_LARGE (len >= 2^32),
 * BSORT_E_WORD_TOO_LONG, BSORT_E_NOMEM, BSORT_E_CUDA, BSORT_E_TIMEOUT.
 */
bsort_status bsort_text(bsort_ctx* ctx, const uint8_t* bytes, size_t len, bsort_result* out);

/*
 * Sorts one document already in device memory.  d_bytes is a device pointer
 * (any alignment) to len bytes; it must stay unchanged until the work
 * enqueued on `stream` has finished.  `stream` is a cudaStream_t (NULL = the
 * legacy default stream).
 * The call enqueues the whole path on `stream` and waits only for the summary
 * of the bucket layout (computed on the device from the length histograms),
 * which fixes the later launches' sizes; it returns with the scalar fields
 * of *out filled and with DEVICE pointers in counts, offsets and stream, whose
 * contents are complete once `stream` reaches the point of return (for
 * example after cudaStreamSynchronize(stream)).
 * Errors: as bsort_text.  A bounded wait of the tokenize kernel that runs
 * out is reported by this call (BSORT_E_TIMEOUT); one of the sort kernels,
 * which run after the call returns, by bsort_device_finish().
 */
bsort_status bsort_text_device(bsort_ctx* ctx, const uint8_t* d_bytes, size_t len, void* stream,
                               bsort_result* out);

/*
 * Sorts n independent documents held in host memory in one pass of the path:
 * every kernel launch covers all documents.  docs[i] points to lens[i] bytes.
 * outs[i] receives document i's result (HOST pointers), with outs[i].status
 * set per document; the call returns BSORT_OK when every document succeeded,
 * otherwise the first failing document's status.  Each document's result is
 * identical to what bsort_text returns for it alone.  Documents that lie back
 * to back in host memory (docs[i + 1] == docs[i] + lens[i], empty ones
 * anywhere) move to the device as one region, read in place when it is
 * page-locked (as in bsort_text); others are gathered into the staging buffer.
 */
bsort_status bsort_batch(bsort_ctx* ctx, const uint8_t* const* docs, const size_t* lens, size_t n,
                         bsort_result* outs);

/*
 * Sorts n independent documents already in device memory, in one pass of the
 * path (every kernel launch covers all documents).  Document i is the lens[i]
 * bytes at d_base + offs[i] (any alignment; documents may be packed back to
 * back).  offs and lens are HOST arrays.  The total must stay below 2^32
 * bytes (BSORT_E_TOO_LARGE otherwise).  Like bsort_text_device, the call
 * enqueues the path on `stream`, waits only for the length histograms, and
 * returns with the scalar fields of outs[i] filled and DEVICE pointers whose
 * contents are complete once `stream` reaches the point of return.  Each
 * document's result is identical to bsort_text_device on that document alone.
 * Returns BSORT_OK when every document succeeded, otherwise the first failing
 * document's status (outs[i].status per document).
 */
bsort_status bsort_batch_device(bsort_ctx* ctx, const uint8_t* d_base, const uint64_t* offs, const uint64_t* lens,
                                size_t n, void* stream, bsort_result* outs);

/*
 * Status of the device work that the last bsort_text_device or
 * bsort_batch_device call on ctx enqueued.  Waits until `stream` (the one
 * that call was given) has finished it; returns BSORT_E_TIMEOUT when a
 * bounded device wait of the sort kernels ran out in it (its outputs are
 * then not valid) and clears that record, else BSORT_OK.  A record that is
 * never collected this way makes the next call on the context fail with
 * BSORT_E_TIMEOUT instead.  Errors: BSORT_E_INVAL, BSORT_E_BUSY, BSORT_E_CUDA.
 */
bsort_status bsort_device_finish(bsort_ctx* ctx, void* stream);

/*
 * Kernel tracing.  Every launch is counted; with config.profile == 1 each one
 * is also bracketed by two CUDA events on the stream it runs on, and tagged
 * with the algorithmic bytes it must move (the reads and writes the method
 * needs: input, stripped letters, word starts, keys, output).
 */
typedef struct {
  const char* name;   /* kernel family: "tokenize", "scatter", "tile_sort", "merge_pass",
                         "merge_cut" (the tile cuts of a pipelined merge pass), "emit";
                         "layout" (the bucket layout: one segment per (document, length) from
                         the length histograms, ordered by the kernels that sort them);
                         "dedupe" (the duplicate-aware sort's hash aggregation of the large
                         buckets) and "expand" (its expansion of the sorted distinct words);
                         and "host_gap", the device time of the call's host round trips (the
                         layout's summary read back, until the next launch; with the
                         duplicate-aware sort, also its distinct-key counts) (static string) */
  uint64_t launches;  /* kernel launches since the last read */
  double ms;          /* summed device time of those launches (0 when profiling is off) */
  double bytes;       /* summed algorithmic bytes of those launches */
  double key_levels;  /* sort kernels: summed key-levels, each key counted once per doubling of the
                         sorted run it ends in (n * ceil(log2 run) per bucket); 0 for the others */
} bsort_kernel_stat;

/* Writes up to `max` per-family statistics accumulated since the last read
 * into out[], waits for the recorded events, resets the accumulators and
 * returns the number of families written (or -1 on error). */
int bsort_profile_read(bsort_ctx* ctx, bsort_kernel_stat* out, int max);

/* One traced launch (config.profile == 1): its family, when it ran and the
 * algorithmic bytes it moved. */
typedef struct {
  const char* name;   /* kernel family, as in bsort_kernel_stat (static string) */
  double start_ms;    /* start, in ms after the first traced launch since the last bsort_profile_read */
  double end_ms;      /* end, on the same clock */
  double bytes;       /* algorithmic bytes */
  uint32_t stream;    /* 0: the call's stream; 1..5: the side streams of the tile sorts, 6..9: those of the merge chains */
  uint32_t variant;   /* tile_sort: CTAs per cluster (0: the one-warp sort of tiny buckets);
                         merge_pass / merge_cut: key width in u64 words; else 0 */
  uint32_t kernels;   /* kernels the launch comprises (layout: 1 or 3, dedupe: 2, expand: up to 4, the
                         length order and the whole-text emit: 3; host_gap: 0; else 1) */
  uint32_t reserved;
} bsort_trace_rec;

/* Writes up to `max` traced launches, in launch order, into out[] (waiting for
 * their events) and returns how many there are (may exceed max), or -1 on
 * error.  Leaves them in place: bsort_profile_read clears them. */
int bsort_trace_read(bsort_ctx* ctx, bsort_trace_rec* out, int max);

/* Kernel launches made by this context since it was created. */
uint64_t bsort_launch_count(const bsort_ctx* ctx);

/*
 * Strip + tokenize without allocating (the paper has no counterpart: this is
 * an entry point for callers that cannot call cudaMalloc, such as code running
 * while a CUDA graph is being captured, plugins whose host framework owns all
 * device memory, or processes that must not grow their device footprint).
 *
 * Runs phase 1 of the method (strip the special characters, split the words)
 * on one document in device memory, as one kernel, and writes:
 *   d_letters[0 .. L)  the document's letters in input order (capacity >= len bytes),
 *   d_starts[0 .. n]   d_starts[w] = offset in d_letters of word w's first letter,
 *                      d_starts[n] = L (capacity >= len/2 + 2 entries),
 *   d_totals[0..2]     n (words), L (letters), and a status: 0, or BSORT_E_TIMEOUT
 *                      when a bounded device wait ran out (outputs then invalid).
 * Every pointer is a device pointer; d_bytes may have any alignment.  The work
 * is enqueued on `stream` (a cudaStream_t, NULL = legacy default stream) and
 * the outputs are complete when the stream reaches that point; the call does
 * not wait for it.
 *
 * Allocation: none.  The call makes no cudaMalloc, cudaFree or other
 * allocating call.  Its scratch, one 32-byte record per 16 KiB of input, lives
 * in a 131,328-byte array inside the library that every GPU which loads the
 * library holds until the process exits.  Hence the limit: len must be at most
 * 64 MiB - 16 bytes (67,108,848); a longer document returns BSORT_E_TOO_LARGE
 * before any GPU work.  The first call on each device looks up the array's
 * device address (with that device current), so make that first call before
 * any stream capture.
 *
 * Sharing: every call on a device uses the same array, and it keeps the last
 * call's contents (each call clears what must start at zero).  Calls whose
 * work overlaps on the GPU (for example on two streams) race on it and give
 * wrong results: order them on one stream or synchronise between them.
 *
 * Errors: BSORT_E_INVAL (a NULL pointer where one is required),
 * BSORT_E_TOO_LARGE, BSORT_E_CUDA (no current device, or a launch failed).
 */
bsort_status bsort_strip_noalloc(const uint8_t* d_bytes, size_t len, void* stream, uint8_t* d_letters,
                                 uint32_t* d_starts, uint32_t* d_totals);

/* The configuration a context was created with (device resolved). */
bsort_status bsort_context_config(const bsort_ctx* ctx, bsort_config* out);

/*
 * Serving: a request loop with continuous batching (no counterpart in the
 * paper; it serves many documents as they arrive, with the batch path).
 *
 * bsort_serve_start() starts `workers` threads on the context's device, each
 * with a context of its own.  bsort_submit() copies a document into the
 * request queue (the caller may reuse its buffer at once).  A worker takes the
 * queued requests in arrival order, as many as fit max_batch_docs and the
 * device-memory budget hbm_budget of the requests in flight (a document of n
 * bytes counts 16 n + 64 KiB), and sorts them with one bsort_batch call; the
 * workers' batches overlap on the GPU, and requests arriving meanwhile are
 * admitted as soon as a worker and enough budget are free.  bsort_poll()
 * hands out finished requests: their tags, their results (HOST pointers,
 * outs[i].status per request) and, when latency_ns is not NULL, the time from
 * submission to completion.  Each result equals what bsort_text returns for
 * the document alone.  Results are not copied: they point into the
 * page-locked buffers their batch was read back into, which stay held until
 * every result of that batch has been passed to bsort_result_release(ctx,
 * &out) (the server then writes a later batch into them).  So each polled
 * result stays valid until it is released, or until bsort_serve_start
 * restarts the server or bsort_destroy; release every result once it has
 * been used, or the server keeps allocating new buffers.
 *
 * Threads: bsort_submit may run on several threads at once (producers),
 * bsort_poll on one other thread (the consumer), and bsort_result_release of
 * polled results on any threads, all at the same time; no other call on the
 * context may run meanwhile.
 * bsort_serve_stop() finishes the queued requests and stops the workers;
 * finished results stay pollable (and, once polled, valid until released).
 * bsort_destroy() stops a running server and frees every result.
 */
typedef struct {
  uint64_t hbm_budget;      /* device bytes the in-flight requests may use (0 = 64 GiB) */
  uint32_t workers;         /* batches in flight at once, 1..16 (0 = 2) */
  uint32_t max_batch_docs;  /* requests per batch (0 = 1024) */
} bsort_serve_config;

void bsort_serve_config_default(bsort_serve_config* cfg);

/* Errors: BSORT_E_INVAL, BSORT_E_BUSY (already serving), and those of bsort_create. */
bsort_status bsort_serve_start(bsort_ctx* ctx, const bsort_serve_config* cfg);

/* Errors: BSORT_E_INVAL (not serving, NULL bytes), BSORT_E_TOO_LARGE (1 GiB or more,
 * or more than the whole budget), BSORT_E_BUSY (stopping). */
bsort_status bsort_submit(bsort_ctx* ctx, const uint8_t* bytes, size_t len, uint64_t tag);

/* bsort_submit without the copy: the server reads the caller's bytes, which
 * must stay valid and unchanged until the request's result has been polled.
 * Page-locked bytes are read by the copy engine in place (no host copy at
 * all); pageable ones are copied by the worker that takes the request.
 * Errors as bsort_submit. */
bsort_status bsort_submit_borrowed(bsort_ctx* ctx, const uint8_t* bytes, size_t len, uint64_t tag);

/* Writes up to max finished requests; returns how many. */
size_t bsort_poll(bsort_ctx* ctx, uint64_t* tags, bsort_result* outs, uint64_t* latency_ns, size_t max);

/* Requests submitted and not yet taken by a worker. */
size_t bsort_serve_pending(const bsort_ctx* ctx);

bsort_status bsort_serve_stop(bsort_ctx* ctx);

/* Marks a result's buffers as no longer needed and zeroes *res.  The memory
 * itself stays with the context for reuse. */
void bsort_result_release(bsort_ctx* ctx, bsort_result* res);

#ifdef __cplusplus
}
#endif

#endif /* BSORT_H */
