/*
 * kc_oracle.c - TEST INFRASTRUCTURE ONLY: the plain CPU k-mer counter that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no code,
 * header, table or constant with the GPU library.
 *
 * What it computes (Section II, problem statement; Algorithm 1, serial counter):
 * the histogram of all length-k substrings ("k-mers") of the input reads, returned
 * as an ordered array of {k-mer, count} pairs.  Written as the definition, slowly:
 *
 *   for every read R and every start j with j + k <= |R|:
 *     the window R[j .. j+k) counts iff every byte is one of ACGTacgt;
 *     its forward value is  sum_{t<k} code(R[j+t]) * 4^(k-1-t),
 *       code: A=0 C=1 G=2 T=3 (lowercase the same), first base most significant;
 *     its reverse-complement value is the same sum over the reversed window with
 *       every code c replaced by 3 - c;
 *     key = canonical ? min(forward, reverse complement) : forward.
 *   collect all keys (Algorithm 1: T.add), Sort, then Accumulate (run-length
 *   encode the sorted array) into ascending (key, count) pairs.
 *
 * Readings where the paper is silent (listed with their reasons in the design
 * notes): the 2-bit code order A<C<G<T; only the low 2k bits are kept (the key is
 * a k-digit base-4 number); canonical form = min of the two values as unsigned
 * integers; a window containing any byte outside ACGTacgt is skipped whole;
 * windows never span two reads; keys are 64-bit for k <= 32 and 128-bit for
 * 33 <= k <= 64 (Section VII names 128-bit k-mers as the extension); counts are
 * 32-bit and a larger count is an error.
 *
 * Nothing here is blocked, fused or reordered: each window's key is computed from
 * its own k bytes (no rolling update), the sort is the C library qsort.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_EOVERFLOW = 4 };

typedef struct {
  uint64_t n;               /* distinct keys */
  uint32_t key_words;       /* 1: uint64 keys; 2: (lo, hi) uint64 pairs */
  uint64_t *keys;           /* n * key_words words, ascending */
  uint32_t *counts;         /* n counts */
  uint64_t n_valid_windows; /* number of windows that counted */
} oracle_result;

/* code of one byte, or -1 for any byte that is not a base */
static int base_code(uint8_t b) {
  switch (b) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
  }
}

/* key of the window w[0..k), or -1 if a byte is not a base (Section II: a k-mer is a
   length-k string over {A,C,G,T}) */
static int window_key(const uint8_t *w, int k, int canonical, u128 *key) {
  u128 fwd = 0, rc = 0;
  for (int t = 0; t < k; ++t) {
    int c = base_code(w[t]);
    if (c < 0) return -1;
    fwd = fwd * 4 + (u128)c;
  }
  for (int t = k - 1; t >= 0; --t) rc = rc * 4 + (u128)(3 - base_code(w[t]));
  *key = (canonical && rc < fwd) ? rc : fwd;
  return 0;
}

static int cmp_u128(const void *a, const void *b) {
  u128 x = *(const u128 *)a, y = *(const u128 *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

static int check_args(const uint8_t *reads, const uint64_t *offsets, uint64_t n_reads, int k) {
  if (k < 1 || k > 64) return OR_EINVAL;
  if (n_reads > 0 && (!offsets || (!reads && offsets[n_reads] > 0))) return OR_EINVAL;
  if (n_reads > 0 && offsets[0] != 0) return OR_EINVAL;
  for (uint64_t i = 0; i < n_reads; ++i)
    if (offsets[i + 1] < offsets[i]) return OR_EINVAL;
  return OR_OK;
}

/* number of windows that count: k consecutive bases inside one read */
uint64_t oracle_valid_windows(const uint8_t *reads, const uint64_t *offsets, uint64_t n_reads, int k) {
  if (check_args(reads, offsets, n_reads, k)) return 0;
  uint64_t n = 0;
  for (uint64_t i = 0; i < n_reads; ++i) {
    uint64_t len = offsets[i + 1] - offsets[i];
    const uint8_t *r = reads + offsets[i];
    for (uint64_t j = 0; j + (uint64_t)k <= len; ++j) {
      int ok = 1;
      for (int t = 0; t < k; ++t) if (base_code(r[j + t]) < 0) { ok = 0; break; }
      n += (uint64_t)ok;
    }
  }
  return n;
}

/* Algorithm 1: collect every window's key, Sort, Accumulate. */
int oracle_count(const uint8_t *reads, const uint64_t *offsets, uint64_t n_reads, int k, int canonical,
                 oracle_result *out) {
  memset(out, 0, sizeof(*out));
  int rc = check_args(reads, offsets, n_reads, k);
  if (rc) return rc;
  out->key_words = k <= 32 ? 1 : 2;
  uint64_t cap = 0;
  for (uint64_t i = 0; i < n_reads; ++i) {
    uint64_t len = offsets[i + 1] - offsets[i];
    if (len >= (uint64_t)k) cap += len - (uint64_t)k + 1;
  }
  u128 *T = (u128 *)malloc(sizeof(u128) * (cap ? cap : 1));
  if (!T) return OR_ENOMEM;
  uint64_t m = 0;
  for (uint64_t i = 0; i < n_reads; ++i) {
    uint64_t len = offsets[i + 1] - offsets[i];
    const uint8_t *r = reads + offsets[i];
    for (uint64_t j = 0; j + (uint64_t)k <= len; ++j) {
      u128 key;
      if (window_key(r + j, k, canonical, &key) == 0) T[m++] = key;
    }
  }
  out->n_valid_windows = m;
  qsort(T, m, sizeof(u128), cmp_u128);
  /* Accumulate: one (key, count) pair per run of equal keys */
  uint64_t d = 0;
  for (uint64_t i = 0; i < m; ++i)
    if (i == 0 || T[i] != T[i - 1]) ++d;
  out->keys = (uint64_t *)malloc(sizeof(uint64_t) * out->key_words * (d ? d : 1));
  out->counts = (uint32_t *)malloc(sizeof(uint32_t) * (d ? d : 1));
  if (!out->keys || !out->counts) { free(T); free(out->keys); free(out->counts); memset(out, 0, sizeof(*out)); return OR_ENOMEM; }
  uint64_t q = 0;
  for (uint64_t i = 0; i < m;) {
    uint64_t j = i;
    while (j < m && T[j] == T[i]) ++j;
    if (j - i > 0xffffffffull) rc = OR_EOVERFLOW;
    if (out->key_words == 1) {
      out->keys[q] = (uint64_t)T[i];
    } else {
      out->keys[2 * q] = (uint64_t)T[i];
      out->keys[2 * q + 1] = (uint64_t)(T[i] >> 64);
    }
    out->counts[q] = (uint32_t)(j - i);
    ++q;
    i = j;
  }
  out->n = d;
  free(T);
  return rc;
}

void oracle_free(oracle_result *r) {
  free(r->keys); free(r->counts);
  memset(r, 0, sizeof(*r));
}

/*
 * Count chosen keys only: for the n_q keys in `query` (ascending, distinct; same
 * word layout as oracle_result.keys) add up how many windows have that key.  Used
 * to check sampled entries of a result too large for oracle_count, and absent
 * keys (count 0).  Same per-window definition as oracle_count; lookup by binary search.
 */
int oracle_count_keys(const uint8_t *reads, const uint64_t *offsets, uint64_t n_reads, int k, int canonical,
                      const uint64_t *query, uint64_t n_q, uint64_t *counts_out) {
  int rc = check_args(reads, offsets, n_reads, k);
  if (rc) return rc;
  int kw = k <= 32 ? 1 : 2;
  u128 *Q = (u128 *)malloc(sizeof(u128) * (n_q ? n_q : 1));
  if (!Q) return OR_ENOMEM;
  for (uint64_t i = 0; i < n_q; ++i) {
    Q[i] = kw == 1 ? (u128)query[i] : ((u128)query[2 * i + 1] << 64) | (u128)query[2 * i];
    counts_out[i] = 0;
    if (i > 0 && Q[i] <= Q[i - 1]) { free(Q); return OR_EINVAL; }
  }
  for (uint64_t i = 0; i < n_reads; ++i) {
    uint64_t len = offsets[i + 1] - offsets[i];
    const uint8_t *r = reads + offsets[i];
    for (uint64_t j = 0; j + (uint64_t)k <= len; ++j) {
      u128 key;
      if (window_key(r + j, k, canonical, &key)) continue;
      uint64_t lo = 0, hi = n_q;
      while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (Q[mid] < key) lo = mid + 1; else hi = mid;
      }
      if (lo < n_q && Q[lo] == key) ++counts_out[lo];
    }
  }
  free(Q);
  return OR_OK;
}
