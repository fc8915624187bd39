/*
 * synth.c - seeded synthetic DNA read sets shaped like the paper's workloads.
 *
 * This module only produces ASCII bases and read offsets.  It holds none of the
 * counting method's arithmetic (no base encoding, no k-mer keys): the oracle and
 * the CUDA path both consume its output and nothing else from here.
 *
 * The paper simulates Illumina reads from uniform random genomes (Section VI,
 * "Datasets", Table VI) and uses real SRA genomes; neither the simulator nor the
 * SRA data exist here, so the generator below stands in for them:
 *   RNG: xoshiro256** seeded through splitmix64.
 *   WL_UNIFORM_SHORT   1 Mbp i.i.d. genome, 100 bp reads at 10x, both strands,
 *                      0.5% substitutions, then 0.01% of bases set to 'N'.
 *   WL_REPEAT_SHORT    100 Mbp genome, 20% of it copies of 500 repeat families
 *                      (consensus length U[300,6000], copy numbers ~ Zipf(1.2) by
 *                      rank, 2% substitutions per copy), 150 bp reads at 30x,
 *                      0.5% substitutions.
 *   WL_LONG_NOISY      50 Mbp i.i.d. genome, read spans log-normal (median 10 kbp,
 *                      sigma 0.5, at least 64), 20x by span, 5% errors per base
 *                      split 60/20/20 substitution/insertion/deletion.
 *   WL_SAMPLE          one sample of the batched workload: genome log-uniform in
 *                      [0.1, 50] Mbp, 150 bp reads, coverage U[5,40], 0.5% subst.
 *   WL_SERVE           one request's read set of the served workload: genome
 *                      log-uniform in [0.05, 20] Mbp, 150 bp reads, coverage U[10,30],
 *                      0.5% subst.
 * A scale factor multiplies the genome size (and the number of repeat families)
 * so the same shapes can be produced at sizes a slow checker finishes quickly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
  uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
static void rng_seed(rng_t *r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t rng_next(rng_t *r) {
  uint64_t *s = r->s;
  uint64_t out = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl(s[3], 45);
  return out;
}
/* uniform integer in [0, n), n >= 1 (Lemire's multiply-shift, rejection-free bias < 2^-32 for our n) */
static inline uint64_t rng_below(rng_t *r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}
/* uniform double in [0, 1) from the top 53 bits */
static inline double rng_unit(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
/* event with probability p, decided in integer arithmetic on a 2^32 grid */
static inline int rng_event(rng_t *r, uint32_t p32) { return (uint32_t)(rng_next(r) >> 32) < p32; }
static uint32_t prob32(double p) { return (uint32_t)(p * 4294967296.0); }

static const char BASES[4] = {'A', 'C', 'G', 'T'};

static char other_base(rng_t *r, char b) {
  /* one of the three bases different from b, uniformly */
  int idx = 0;
  for (int i = 0; i < 4; ++i) if (BASES[i] == b) idx = i;
  int j = (int)rng_below(r, 3);
  if (j >= idx) ++j;
  return BASES[j];
}
static char comp_base(char b) {
  switch (b) { case 'A': return 'T'; case 'C': return 'G'; case 'G': return 'C'; case 'T': return 'A'; default: return b; }
}
static void random_seq(rng_t *r, char *dst, uint64_t n) {
  uint64_t i = 0;
  while (i < n) {
    uint64_t w = rng_next(r);
    for (int t = 0; t < 32 && i < n; ++t, ++i) { dst[i] = BASES[w & 3]; w >>= 2; }
  }
}

typedef struct {
  uint8_t *reads;    /* concatenated read bytes */
  uint64_t *offsets; /* n_reads + 1 entries */
  uint64_t n_reads;
  uint64_t n_bytes;
  uint64_t genome_len;
} synth_out;

/* growable output */
typedef struct { uint8_t *b; uint64_t n, cap; uint64_t *o; uint64_t nr, ocap; } sink_t;
static int sink_reserve(sink_t *s, uint64_t extra) {
  if (s->n + extra <= s->cap) return 0;
  uint64_t nc = s->cap ? s->cap : (1u << 20);
  while (nc < s->n + extra) nc *= 2;
  uint8_t *nb = (uint8_t *)realloc(s->b, nc);
  if (!nb) return -1;
  s->b = nb; s->cap = nc; return 0;
}
static int sink_end_read(sink_t *s) {
  if (s->nr + 2 > s->ocap) {
    uint64_t nc = s->ocap ? s->ocap * 2 : 1024;
    uint64_t *no = (uint64_t *)realloc(s->o, nc * sizeof(uint64_t));
    if (!no) return -1;
    s->o = no; s->ocap = nc;
  }
  if (s->nr == 0) s->o[0] = 0;
  s->o[++s->nr] = s->n;
  return 0;
}

/* short reads of length L from genome g, strand +/- with p = 1/2, substitutions at rate ps,
   then bases set to 'N' at rate pn; n_reads reads */
static int emit_short_reads(rng_t *r, const char *g, uint64_t G, uint64_t L, uint64_t n_reads,
                            double ps, double pn, sink_t *s) {
  uint32_t ps32 = prob32(ps), pn32 = prob32(pn);
  if (L > G) L = G;
  if (sink_reserve(s, n_reads * L)) return -1;
  for (uint64_t i = 0; i < n_reads; ++i) {
    uint64_t st = rng_below(r, G - L + 1);
    int rev = (int)(rng_next(r) >> 63);
    uint8_t *dst = s->b + s->n;
    for (uint64_t j = 0; j < L; ++j) {
      char b = rev ? comp_base(g[st + L - 1 - j]) : g[st + j];
      if (ps32 && rng_event(r, ps32)) b = other_base(r, b);
      if (pn32 && rng_event(r, pn32)) b = 'N';
      dst[j] = (uint8_t)b;
    }
    s->n += L;
    if (sink_end_read(s)) return -1;
  }
  return 0;
}

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : x > y;
}

/* genome of length G with a fraction `rep_frac` made of copies of n_fam repeat families */
static char *repeat_genome(rng_t *r, uint64_t G, int n_fam, double rep_frac, double div) {
  char *g = (char *)malloc(G);
  if (!g) return NULL;
  uint64_t *flen = (uint64_t *)malloc(sizeof(uint64_t) * n_fam);
  char **cons = (char **)malloc(sizeof(char *) * n_fam);
  double *w = (double *)malloc(sizeof(double) * n_fam);
  if (!flen || !cons || !w) return NULL;
  double wsum = 0.0;
  for (int f = 0; f < n_fam; ++f) {
    flen[f] = 300 + rng_below(r, 5701);
    cons[f] = (char *)malloc(flen[f]);
    random_seq(r, cons[f], flen[f]);
    w[f] = pow((double)(f + 1), -1.2);
    wsum += w[f] * (double)flen[f];
  }
  double c = rep_frac * (double)G / wsum;
  uint64_t n_copies = 0, rep_len = 0;
  uint64_t *ncp = (uint64_t *)malloc(sizeof(uint64_t) * n_fam);
  for (int f = 0; f < n_fam; ++f) {
    uint64_t n = (uint64_t)llround(c * w[f]);
    if (n < 1) n = 1;
    ncp[f] = n; n_copies += n; rep_len += n * flen[f];
  }
  /* keep the repeats within the genome: drop copies from the tail families if needed */
  for (int f = n_fam - 1; f >= 0 && rep_len > G / 2; --f)
    while (ncp[f] > 0 && rep_len > G / 2) { --ncp[f]; --n_copies; rep_len -= flen[f]; }
  /* copy order: a random permutation of all copies */
  int *order = (int *)malloc(sizeof(int) * (n_copies ? n_copies : 1));
  uint64_t q = 0;
  for (int f = 0; f < n_fam; ++f) for (uint64_t j = 0; j < ncp[f]; ++j) order[q++] = f;
  for (uint64_t i = n_copies; i > 1; --i) { uint64_t j = rng_below(r, i); int t = order[i - 1]; order[i - 1] = order[j]; order[j] = t; }
  /* background gaps: n_copies uniform cut points over the background length */
  uint64_t bg = G - rep_len;
  uint64_t *cut = (uint64_t *)malloc(sizeof(uint64_t) * (n_copies + 1));
  for (uint64_t i = 0; i < n_copies; ++i) cut[i] = rng_below(r, bg + 1);
  qsort(cut, n_copies, sizeof(uint64_t), cmp_u64);
  cut[n_copies] = bg;
  uint32_t div32 = prob32(div);
  uint64_t pos = 0, prev = 0;
  for (uint64_t i = 0; i <= n_copies; ++i) {
    uint64_t gap = cut[i] - prev; prev = cut[i];
    random_seq(r, g + pos, gap); pos += gap;
    if (i == n_copies) break;
    int f = order[i];
    for (uint64_t j = 0; j < flen[f]; ++j) {
      char b = cons[f][j];
      if (rng_event(r, div32)) b = other_base(r, b);
      g[pos + j] = b;
    }
    pos += flen[f];
  }
  for (int f = 0; f < n_fam; ++f) free(cons[f]);
  free(cons); free(flen); free(w); free(ncp); free(order); free(cut);
  return g;
}

/* long noisy reads: spans log-normal(median, sigma) >= 64, coverage by span, per-base error rate pe
   split into substitution / insertion / deletion by the given fractions */
static int emit_long_reads(rng_t *r, const char *g, uint64_t G, double median, double sigma, double cov,
                           double pe, double fs, double fi, sink_t *s) {
  uint32_t pe32 = prob32(pe), fs32 = prob32(fs), fsi32 = prob32(fs + fi);
  double need = cov * (double)G, got = 0.0;
  while (got < need) {
    /* Box-Muller normal deviate */
    double u1 = rng_unit(r), u2 = rng_unit(r);
    if (u1 < 1e-300) u1 = 1e-300;
    double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    uint64_t span = (uint64_t)llround(median * exp(sigma * z));
    if (span < 64) span = 64;
    if (span > G) span = G;
    uint64_t st = rng_below(r, G - span + 1);
    int rev = (int)(rng_next(r) >> 63);
    if (sink_reserve(s, 2 * span + 1)) return -1;
    uint8_t *dst = s->b + s->n;
    uint64_t o = 0;
    for (uint64_t j = 0; j < span; ++j) {
      char b = rev ? comp_base(g[st + span - 1 - j]) : g[st + j];
      if (rng_event(r, pe32)) {
        uint32_t kind = (uint32_t)(rng_next(r) >> 32);
        if (kind < fs32) { dst[o++] = (uint8_t)other_base(r, b); }
        else if (kind < fsi32) { dst[o++] = (uint8_t)BASES[rng_below(r, 4)]; dst[o++] = (uint8_t)b; }
        /* else: deletion, the base is dropped */
      } else {
        dst[o++] = (uint8_t)b;
      }
    }
    s->n += o;
    if (sink_end_read(s)) return -1;
    got += (double)span;
  }
  return 0;
}

enum { WL_UNIFORM_SHORT = 0, WL_REPEAT_SHORT = 1, WL_LONG_NOISY = 2, WL_SAMPLE = 3, WL_SERVE = 4 };

/* Generate one read set.  Returns 0 on success; the caller releases it with synth_free. */
int synth_generate(int workload, uint64_t seed, double scale, synth_out *out) {
  rng_t r;
  rng_seed(&r, seed);
  sink_t s;
  memset(&s, 0, sizeof(s));
  memset(out, 0, sizeof(*out));
  char *g = NULL;
  uint64_t G = 0;
  int rc = 0;
  if (workload == WL_UNIFORM_SHORT) {
    G = (uint64_t)llround(1e6 * scale); if (G < 200) G = 200;
    g = (char *)malloc(G); if (!g) return -1;
    random_seq(&r, g, G);
    uint64_t n = (uint64_t)llround(10.0 * (double)G / 100.0);
    rc = emit_short_reads(&r, g, G, 100, n, 0.005, 0.0001, &s);
  } else if (workload == WL_REPEAT_SHORT) {
    G = (uint64_t)llround(1e8 * scale); if (G < 20000) G = 20000;
    int nf = (int)llround(500 * scale); if (nf < 1) nf = 1; if (nf > 500) nf = 500;
    g = repeat_genome(&r, G, nf, 0.20, 0.02); if (!g) return -1;
    uint64_t n = (uint64_t)llround(30.0 * (double)G / 150.0);
    rc = emit_short_reads(&r, g, G, 150, n, 0.005, 0.0, &s);
  } else if (workload == WL_LONG_NOISY) {
    G = (uint64_t)llround(5e7 * scale); if (G < 2000) G = 2000;
    g = (char *)malloc(G); if (!g) return -1;
    random_seq(&r, g, G);
    rc = emit_long_reads(&r, g, G, 10000.0, 0.5, 20.0, 0.05, 0.6, 0.2, &s);
  } else if (workload == WL_SAMPLE) {
    double lg = log(0.1e6) + rng_unit(&r) * (log(50e6) - log(0.1e6));
    G = (uint64_t)llround(exp(lg) * scale); if (G < 200) G = 200;
    double cov = 5.0 + 35.0 * rng_unit(&r);
    g = (char *)malloc(G); if (!g) return -1;
    random_seq(&r, g, G);
    uint64_t n = (uint64_t)llround(cov * (double)G / 150.0);
    rc = emit_short_reads(&r, g, G, 150, n, 0.005, 0.0, &s);
  } else if (workload == WL_SERVE) {
    double lg = log(0.05e6) + rng_unit(&r) * (log(20e6) - log(0.05e6));
    G = (uint64_t)llround(exp(lg) * scale); if (G < 200) G = 200;
    double cov = 10.0 + 20.0 * rng_unit(&r);
    g = (char *)malloc(G); if (!g) return -1;
    random_seq(&r, g, G);
    uint64_t n = (uint64_t)llround(cov * (double)G / 150.0);
    rc = emit_short_reads(&r, g, G, 150, n, 0.005, 0.0, &s);
  } else {
    return -2;
  }
  free(g);
  if (rc) { free(s.b); free(s.o); return rc; }
  if (s.nr == 0) { s.o = (uint64_t *)malloc(sizeof(uint64_t)); s.o[0] = 0; }
  out->reads = s.b; out->offsets = s.o; out->n_reads = s.nr; out->n_bytes = s.n; out->genome_len = G;
  return 0;
}

void synth_free(synth_out *out) {
  free(out->reads); free(out->offsets);
  memset(out, 0, sizeof(*out));
}

/* splitmix64 step exposed so callers derive per-sample seeds the same way everywhere */
uint64_t synth_mix_seed(uint64_t seed, uint64_t index) {
  uint64_t x = seed ^ index;
  return splitmix64(&x);
}
