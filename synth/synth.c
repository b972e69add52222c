/*
 * Seeded synthetic read / reference-segment pairs shaped like the thesis's
 * short-read workloads (100/150/250 bp reads, edit-distance thresholds of
 * 0-10% of the read length, most candidate locations incorrect).
 *
 * This module holds input generation only: it draws random sequences and
 * random edits and writes ASCII.  It computes nothing of the filtering
 * method.  Both the CUDA path and the CPU oracle consume its output.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  Every pair owns its own
 * stream, seeded from (seed, pair index), so any pair or any range of
 * pairs is regenerated identically, in any order, on any machine: all
 * arithmetic is on 64-bit unsigned integers.
 *
 * Recipes (kind):
 *   0  uniform:   m fixed, E fixed, bases i.i.d. uniform ACGT,
 *                 k ~ U{0..kmax} edits.
 *   1  skewed:    m fixed, E fixed, bases 0.1% N, otherwise 41% GC
 *                 (C, G 20.5% each; A, T 29.5% each); 20% of pairs draw
 *                 k ~ U{0..E}, 80% draw k ~ U{E+1..kmax}.
 *   2  mixed:     m in {100,150,250} with probability .4/.4/.2, r in
 *                 {.02,.05,.08} uniformly, E = round-half-up(r*m); then as
 *                 recipe 1 (20/80 mix relative to each pair's E).
 *   3  skewed_all: m fixed, E fixed, skewed bases, k ~ U{0..kmax} for all.
 *   4  serve:     m uniform over {100,150,250}, r ~ U[0, 0.10),
 *                 E = round-half-up(r*m), then as recipe 1.
 * Edits: each is a substitution, insertion or deletion with probability
 * .6/.2/.2 at a uniform position of the current read (insertion positions
 * range over 0..len); a substitution draws a base different from the old
 * one; an insertion draws a base from the recipe's base distribution.  The
 * read starts as the first m bases of a source string of m + k bases whose
 * first m bases are the reference segment; after the edits it is cut to m
 * bases or extended with the source bases that follow.
 */
#include <stdint.h>
#include <string.h>
#include <pthread.h>

static uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s; } sm_rng;

static uint64_t sm_next(sm_rng *r)
{
    r->s += 0x9E3779B97F4A7C15ull;
    return sm_mix(r->s);
}

static sm_rng sm_for_pair(uint64_t seed, int64_t pair)
{
    sm_rng r;
    r.s = sm_mix(seed + 0x632BE59BD9B4E019ull) ^ sm_mix((uint64_t)pair * 0xD1B54A32D192ED03ull + 1);
    return r;
}

/* uniform integer in [0, n) from the high 32 bits (n < 2^32) */
static uint32_t sm_below(sm_rng *r, uint32_t n)
{
    return (uint32_t)(((sm_next(r) >> 32) * (uint64_t)n) >> 32);
}

/* uniform integer in [a, b] */
static int sm_range(sm_rng *r, int a, int b)
{
    return a + (int)sm_below(r, (uint32_t)(b - a + 1));
}

/* 32-bit probability thresholds */
#define P_N      4294967u    /* 0.001 * 2^32 */
#define P_GC     1760936591u /* 0.41  * 2^32 */
#define P_SUB    2576980378u /* 0.6   * 2^32 */
#define P_INS    3435973837u /* 0.8   * 2^32 */
#define P_MIX    858993459u  /* 0.2   * 2^32 */

static const char BASES[4] = {'A', 'C', 'G', 'T'};

static char draw_base(sm_rng *r, int skewed)
{
    if (!skewed) return BASES[sm_next(r) >> 62];
    uint32_t u = (uint32_t)(sm_next(r) >> 32);
    if (u < P_N) return 'N';
    uint32_t v = (uint32_t)(sm_next(r) >> 32);
    uint32_t b = (uint32_t)(sm_next(r) >> 63);
    if (v < P_GC) return b ? 'G' : 'C';
    return b ? 'T' : 'A';
}

static int is_skewed(int kind) { return kind != 0; }

/* Per-pair (m, E) for the recipe; draws the first values of the pair's
 * stream so that lengths are known before any bytes are written. */
static void pair_shape(int kind, int m_fixed, int E_fixed, sm_rng *r, int *m, int *E)
{
    if (kind == 2) {
        uint32_t u = (uint32_t)(sm_next(r) >> 32);
        /* .4 / .4 / .2 */
        int mm = u < 1717986918u ? 100 : (u < 3435973836u ? 150 : 250);
        int ri = (int)sm_below(r, 3);
        static const int rnum[3] = {2, 5, 8};           /* r = rnum/100 */
        /* round half up of mm*rnum/100 */
        *m = mm;
        *E = (mm * rnum[ri] + 50) / 100;
    } else if (kind == 4) {
        int mm = (int)sm_below(r, 3);
        mm = mm == 0 ? 100 : (mm == 1 ? 150 : 250);
        uint64_t u = sm_next(r) >> 32;                  /* r = u/2^32 * 0.10 */
        /* E = floor(r*m + 1/2) = floor((u*m + 5*2^32) / (10*2^32)) */
        *m = mm;
        *E = (int)((u * (uint64_t)mm + (5ull << 32)) / (10ull << 32));
    } else {
        *m = m_fixed;
        *E = E_fixed;
    }
}

static int draw_k(int kind, int E, int kmax, sm_rng *r)
{
    if (kind == 0 || kind == 3) return sm_range(r, 0, kmax);
    uint32_t u = (uint32_t)(sm_next(r) >> 32);
    if (u < P_MIX || E + 1 > kmax) return sm_range(r, 0, E < kmax ? E : kmax);
    return sm_range(r, E + 1, kmax);
}

/* Shapes of pairs [p0, p1): lens and E per pair. */
void synth_shapes(int kind, uint64_t seed, int m_fixed, int E_fixed,
                  int64_t p0, int64_t p1, int32_t *lens, int16_t *E)
{
    for (int64_t p = p0; p < p1; ++p) {
        sm_rng r = sm_for_pair(seed, p);
        int m, e;
        pair_shape(kind, m_fixed, E_fixed, &r, &m, &e);
        lens[p - p0] = m;
        E[p - p0] = (int16_t)e;
    }
}

#define SYN_MAXLEN 4096

static void gen_pair(int kind, uint64_t seed, int m_fixed, int E_fixed, int kmax,
                     int64_t p, char *read, char *ref)
{
    sm_rng r = sm_for_pair(seed, p);
    int m, E;
    pair_shape(kind, m_fixed, E_fixed, &r, &m, &E);
    int k = draw_k(kind, E, kmax, &r);
    int skew = is_skewed(kind);
    char src[2 * SYN_MAXLEN + 8];
    char cur[3 * SYN_MAXLEN + 8];
    int srclen = m + k;
    if (srclen > 2 * SYN_MAXLEN) srclen = 2 * SYN_MAXLEN;
    for (int i = 0; i < srclen; ++i) src[i] = draw_base(&r, skew);
    memcpy(ref, src, (size_t)m);
    int len = m;
    memcpy(cur, src, (size_t)m);
    for (int e = 0; e < k; ++e) {
        uint32_t u = (uint32_t)(sm_next(&r) >> 32);
        int type = u < P_SUB ? 0 : (u < P_INS ? 1 : 2);
        if (len == 0) type = 1;
        if (len >= 3 * SYN_MAXLEN) type = 0;
        if (type == 0) {
            int pos = (int)sm_below(&r, (uint32_t)len);
            char old = cur[pos];
            int oc = old == 'A' ? 0 : old == 'C' ? 1 : old == 'G' ? 2 : old == 'T' ? 3 : -1;
            if (oc < 0) cur[pos] = BASES[sm_below(&r, 4)];
            else cur[pos] = BASES[(oc + 1 + (int)sm_below(&r, 3)) & 3];
        } else if (type == 1) {
            int pos = (int)sm_below(&r, (uint32_t)(len + 1));
            char b = draw_base(&r, skew);
            memmove(cur + pos + 1, cur + pos, (size_t)(len - pos));
            cur[pos] = b;
            len++;
        } else {
            int pos = (int)sm_below(&r, (uint32_t)len);
            memmove(cur + pos, cur + pos + 1, (size_t)(len - pos - 1));
            len--;
        }
    }
    /* extend with the source bases that follow the segment, then cut */
    int next = m;
    while (len < m && next < srclen) cur[len++] = src[next++];
    while (len < m) cur[len++] = draw_base(&r, skew);
    memcpy(read, cur, (size_t)m);
}

typedef struct {
    int kind, m_fixed, E_fixed, kmax;
    uint64_t seed;
    int64_t p0, begin, end;
    const int64_t *read_off, *ref_off;
    char *reads, *refs;
} syn_job;

static void *syn_run(void *arg)
{
    syn_job *j = (syn_job *)arg;
    for (int64_t p = j->begin; p < j->end; ++p)
        gen_pair(j->kind, j->seed, j->m_fixed, j->E_fixed, j->kmax, p,
                 j->reads + j->read_off[p - j->p0], j->refs + j->ref_off[p - j->p0]);
    return NULL;
}

/* Pairs [p0, p1) into reads/refs at byte offsets read_off/ref_off (indexed
 * from p0).  Lengths must match synth_shapes.  Returns 0, or -1 if a
 * length is out of range. */
int synth_fill(int kind, uint64_t seed, int m_fixed, int E_fixed, int kmax,
               int64_t p0, int64_t p1, const int64_t *read_off, const int64_t *ref_off,
               char *reads, char *refs, int nthreads)
{
    if (m_fixed > SYN_MAXLEN || kmax > SYN_MAXLEN) return -1;
    int64_t n = p1 - p0;
    if (n <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < nthreads) nthreads = (int)n;
    pthread_t tid[256];
    syn_job jobs[256];
    int64_t per = (n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        syn_job j = {kind, m_fixed, E_fixed, kmax, seed, p0, 0, 0, read_off, ref_off, reads, refs};
        j.begin = p0 + (per * t < n ? per * t : n);
        j.end = p0 + (per * (t + 1) < n ? per * (t + 1) : n);
        jobs[t] = j;
        if (nthreads == 1) syn_run(&jobs[t]);
        else pthread_create(&tid[t], NULL, syn_run, &jobs[t]);
    }
    if (nthreads > 1)
        for (int t = 0; t < nthreads; ++t) pthread_join(tid[t], NULL);
    return 0;
}

/* Raw stream values for tests of the generator itself. */
void synth_stream(uint64_t seed, int64_t pair, int64_t count, uint64_t *out)
{
    sm_rng r = sm_for_pair(seed, pair);
    for (int64_t i = 0; i < count; ++i) out[i] = sm_next(&r);
}
