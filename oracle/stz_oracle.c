/*
 * stz_oracle.c -- plain single-threaded CPU oracle of STZ (see stz_oracle.h).
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  It is written to be read against the
 * paper, not to be fast, and it shares nothing with the CUDA library.
 *
 * Parity pins (what fixes each part independently of this code; the tests
 * under tests/test_oracle_*.py hold them):
 *   - stencils: Eqs. 6-8 weights (impulse responses), exactness on every
 *     polynomial of total degree <= 3 at interior points, exactness of the
 *     boundary rules on multilinear fields, weights summing to one;
 *   - partition: level sizes 1/64, 7/64, 56/64 of the points (Sec. 3.2,
 *     Sec. 4.4 "87.5%"), brute-force enumeration of stream positions;
 *   - quantizer: |x - x'| <= eb at every point, checked in exact arithmetic
 *     by the tests; constant and linear fields give all-zero codes;
 *   - Huffman: total bits equal an independent heap Huffman's optimum when no
 *     length limit binds, Kraft sum, decode(encode) = identity;
 *   - streaming: progressive(k) equals the full decode at stride 2^(L-k) and
 *     a region equals the slice of the full decode (Sec. 3.3);
 *   - round trips on every tiny shape.
 * Compression ratio and PSNR against the paper's figures: parity unpinned
 * (the paper's datasets and its SZ3 base coder are not available).
 *
 * Byte format (little-endian; the paper fixes none of it):
 *   header, 256 bytes:
 *     0 "STZ1" | 4 u16 version=1 | 6 u8 dtype | 7 u8 ndim | 8 u8 levels |
 *     9 u8 eb_mode | 10 u8 max_code_len | 11 u8 nsub | 12 u32 radius |
 *     16 u32 brick z,y,x | 28 u32 nstreams | 32 i64 nz,ny,nx | 56 f64 eb |
 *     64 f64 eb_abs | 72 f64 min | 80 f64 max | 88 u64 total_bytes |
 *     96 f64 eb_level[6] | 144 f64 two_eb[6] | 192 f64 eb_ratio |
 *     200 u8 predictor (0 cubic, 1 multi-linear, 2 direct) | rest 0
 *   directory at 256, one 48-byte entry per stream:
 *     u64 section_offset | u64 nsym | u32 nchunks | u32 nlive |
 *     u64 payload_words | u64 noutliers | u64 0
 *   stream section (8-byte aligned):
 *     u16 sym[nlive], u8 len[nlive]  (canonical order: length, then symbol)
 *     pad to 4 | u32 chunk_word_offset[nchunks] |
 *     u16 sub_offset[nchunks][nsub-1] | pad to 4 | u32 payload[payload_words]
 *     | u32 outlier_pos[noutliers] | pad to 8 | P outlier_val[noutliers] |
 *     pad to 8
 *   Streams: 0 = level 1; 1 + 7(l-2) + (k-1) = level l, sub-block k, where
 *   k = 4*(z odd) + 2*(y odd) + (x odd).  A stream's symbols are in brick-major
 *   order: bricks of (bz, by, bx) cells in raster order, cells of a brick in
 *   raster order over the brick clipped to the sub-block.  Each brick is one
 *   chunk: its codes are written MSB-first into 32-bit words starting at its
 *   word offset, padded with zero bits to a whole word.  A chunk of n symbols
 *   is cut into nsub sub-chunks of q = ceil(n / nsub) symbols (the last ones
 *   shorter or empty) whose codes follow each other without padding;
 *   sub_offset[k-1] is the bit position, relative to the chunk's first bit,
 *   where sub-chunk k starts, so each sub-chunk decodes on its own.
 */
#include "stz_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Geometry: hierarchical partition (Sec. 3.1, Fig. 3; three levels Sec. 3.2) */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t n[3]; /* field dims (z, y, x) */
  int L;        /* number of levels */
  int b[3];     /* chunk brick */
} geom;

static int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

/* stride of level l: s_l = 2^(L-l) (level 1 coarsest, level L full grid) */
static int64_t stride_of(const geom* g, int l) { return (int64_t)1 << (g->L - l); }

/* extent of G_l, the grid of points whose coordinates are multiples of s_l */
static void grid_ext(const geom* g, int l, int64_t m[3]) {
  int64_t s = stride_of(g, l);
  for (int a = 0; a < 3; a++) m[a] = cdiv64(g->n[a], s);
}

static int nstreams_of(int L) { return 1 + 7 * (L - 1); }

/* Stream sid: its level, sub-block offsets o (odd axes) and extent e in
 * cells.  Level 1 is the whole of G_1; sub-block k of level l holds the points
 * 2c + o of G_l, c = cell. */
static void stream_ext(const geom* g, int sid, int64_t e[3], int o[3], int* level) {
  if (sid == 0) {
    *level = 1;
    grid_ext(g, 1, e);
    o[0] = o[1] = o[2] = 0;
    return;
  }
  int l = 2 + (sid - 1) / 7, k = 1 + (sid - 1) % 7;
  *level = l;
  o[0] = (k >> 2) & 1;
  o[1] = (k >> 1) & 1;
  o[2] = k & 1;
  int64_t m[3];
  grid_ext(g, l, m);
  for (int a = 0; a < 3; a++) e[a] = m[a] >= o[a] ? (m[a] - o[a] + 1) / 2 : 0;
}

static int64_t vol3(const int64_t e[3]) { return e[0] * e[1] * e[2]; }

int64_t ora_stream_pos(const int64_t e[3], const int b[3], const int64_t c[3]) {
  int64_t B[3], l[3], lc[3];
  for (int a = 0; a < 3; a++) {
    B[a] = c[a] / b[a];
    lc[a] = c[a] - B[a] * b[a];
    l[a] = e[a] - B[a] * b[a];
    if (l[a] > b[a]) l[a] = b[a];
  }
  return B[0] * b[0] * e[1] * e[2] + B[1] * b[1] * l[0] * e[2] +
         B[2] * b[2] * l[0] * l[1] + (lc[0] * l[1] + lc[1]) * l[2] + lc[2];
}

static void brick_grid(const int64_t e[3], const int b[3], int64_t nb[3]) {
  for (int a = 0; a < 3; a++) nb[a] = e[a] > 0 ? cdiv64(e[a], b[a]) : 0;
}

/* chunk j of a stream: first stream position, symbol count, brick origin and
 * clipped extent */
static void chunk_geom(const int64_t e[3], const int b[3], int64_t j, int64_t* start,
                       int64_t* count, int64_t org[3], int64_t lext[3]) {
  int64_t nb[3];
  brick_grid(e, b, nb);
  int64_t B[3] = {j / (nb[1] * nb[2]), (j / nb[2]) % nb[1], j % nb[2]};
  for (int a = 0; a < 3; a++) {
    org[a] = B[a] * b[a];
    lext[a] = e[a] - org[a];
    if (lext[a] > b[a]) lext[a] = b[a];
  }
  *start = ora_stream_pos(e, b, org);
  *count = lext[0] * lext[1] * lext[2];
}

/* ------------------------------------------------------------------------ */
/* Field-precision parts, instantiated for float and double                 */
/* ------------------------------------------------------------------------ */

enum { RULE_MID = 0, RULE_EXT = 1, RULE_COPY = 2 };

#define REAL float
#define SFX(name) name##_f32
#define FABS fabsf
#define RINT rintf
#define ISFINITE isfinite
#include "stz_oracle_real.inc"
#undef REAL
#undef SFX
#undef FABS
#undef RINT
#undef ISFINITE

#define REAL double
#define SFX(name) name##_f64
#define FABS fabs
#define RINT rint
#define ISFINITE isfinite
#include "stz_oracle_real.inc"
#undef REAL
#undef SFX
#undef FABS
#undef RINT
#undef ISFINITE

/* ------------------------------------------------------------------------ */
/* Error bounds: absolute or value-range relative bound, then the adaptive    */
/* per-level bound of Sec. 3.1 opt. 5 (eb_coarser = eb_finer / 2.5), applied  */
/* level by level in the three-level scheme (Sec. 3.2).                       */
/* ------------------------------------------------------------------------ */

static double eb_absolute(int eb_mode, double eb, int any_finite, double vmin, double vmax) {
  if (eb_mode == ORA_EB_ABS) return eb;
  double range = any_finite ? vmax - vmin : 0.0;
  double ea = eb * range;
  /* zero range (constant or all non-finite field): the bound is taken as
   * absolute; likewise when the product under- or overflows */
  if (!(ea > 0.0) || !isfinite(ea)) ea = eb;
  return ea;
}

/* ratio: 2.5 in the paper; ratio^k is formed by repeated multiplication in
 * double, in this order, so that a decoder or another implementation forms
 * the same bound (2.5^k is exact for k <= 6) */
static double eb_of_level(double eb_abs, int L, int l, double ratio) {
  double r = 1.0;
  for (int k = 0; k < L - l; k++) r *= ratio;
  return eb_abs / r;
}

static double ratio_of(const ora_params* p) { return p->eb_ratio == 0.0 ? 2.5 : p->eb_ratio; }

static float rz_float(double v) { /* largest float <= v, for v > 0 */
  float f = (float)v;
  if ((double)f > v) f = nextafterf(f, 0.0f);
  return f;
}

static void level_consts_f32(double ebl, int R, qc_f32* q) {
  q->two_eb = (float)(2.0 * ebl);
  q->inv2eb = (float)(1.0 / (2.0 * ebl));
  q->ebc = nextafterf(rz_float(ebl), 0.0f);
  q->rlim = (float)R - 0.5f;
}

static void level_consts_f64(double ebl, int R, qc_f64* q) {
  q->two_eb = 2.0 * ebl;
  q->inv2eb = 1.0 / (2.0 * ebl);
  q->ebc = nextafter(ebl, 0.0);
  q->rlim = (double)R - 0.5;
}

/* ------------------------------------------------------------------------ */
/* Huffman coding of each sub-block's codes (Sec. 2.1 step 3, Sec. 3.3)       */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t f;
  int sym;
} leaf;

static int leaf_cmp(const void* a, const void* b) {
  const leaf* x = (const leaf*)a;
  const leaf* y = (const leaf*)b;
  if (x->f != y->f) return x->f < y->f ? -1 : 1;
  return x->sym < y->sym ? -1 : (x->sym > y->sym);
}

/*
 * Code lengths.  Live symbols are sorted by (frequency, symbol) ascending.
 * Two-queue Huffman: repeatedly join the two lightest of (leaf queue head,
 * internal queue head), a leaf winning ties; internal nodes are queued in
 * creation order.  The depth of each leaf gives a count of codes per length.
 * If the longest exceeds max_len, the counts are repaired: every code longer
 * than max_len is shortened to max_len, which pushes the Kraft sum above 1 by
 * an excess E (in units of 2^-max_len); then, in passes from length
 * max_len-1 up to 1, as many codes as E allows (at most E / 2^(max_len-l-1)
 * of them) move from length l to l+1, each lowering E by 2^(max_len-l-1);
 * a pass that moves nothing while E > 0 moves one code of the largest length
 * below max_len that has codes.  The sum ends at or below 1.  Lengths are then
 * handed out by frequency rank: the most frequent symbols (the end of the
 * sorted order) receive the shortest lengths.  A single live symbol gets
 * length 1.
 */
int ora_huffman_lengths(const uint64_t* freq, int nsym, int max_len, uint8_t* len) {
  if (nsym <= 0 || max_len < 1 || max_len > 24) return ORA_ERR_ARG;
  memset(len, 0, (size_t)nsym);
  int n = 0;
  for (int s = 0; s < nsym; s++) n += freq[s] > 0;
  if (n == 0) return ORA_OK;
  if ((int64_t)n > ((int64_t)1 << max_len)) return ORA_ERR_ARG;
  leaf* lv = (leaf*)malloc(sizeof(leaf) * (size_t)n);
  if (!lv) return ORA_ERR_NOMEM;
  n = 0;
  for (int s = 0; s < nsym; s++)
    if (freq[s] > 0) {
      lv[n].f = freq[s];
      lv[n].sym = s;
      n++;
    }
  qsort(lv, (size_t)n, sizeof(leaf), leaf_cmp);
  if (n == 1) {
    len[lv[0].sym] = 1;
    free(lv);
    return ORA_OK;
  }
  uint64_t* wi = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  int* par_leaf = (int*)malloc(sizeof(int) * (size_t)n);
  int* par_int = (int*)malloc(sizeof(int) * (size_t)n);
  int* dep = (int*)malloc(sizeof(int) * (size_t)n);
  if (!wi || !par_leaf || !par_int || !dep) {
    free(lv); free(wi); free(par_leaf); free(par_int); free(dep);
    return ORA_ERR_NOMEM;
  }
  int i = 0, j = 0;
  for (int k = 0; k < n - 1; k++) {
    uint64_t w = 0;
    for (int pick = 0; pick < 2; pick++) {
      int take_leaf = i < n && (j >= k || lv[i].f <= wi[j]);
      if (take_leaf) {
        w += lv[i].f;
        par_leaf[i] = k;
        i++;
      } else {
        w += wi[j];
        par_int[j] = k;
        j++;
      }
    }
    wi[k] = w;
  }
  /* depths: the root is the last internal node */
  dep[n - 2] = 0;
  for (int k = n - 3; k >= 0; k--) dep[k] = dep[par_int[k]] + 1;
  int bl[64];
  memset(bl, 0, sizeof(bl));
  int maxd = 0;
  for (int k = 0; k < n; k++) {
    int d = dep[par_leaf[k]] + 1;
    bl[d]++;
    if (d > maxd) maxd = d;
  }
  if (maxd > max_len) {
    for (int l = maxd; l > max_len; l--) {
      bl[max_len] += bl[l];
      bl[l] = 0;
    }
    int64_t excess = -((int64_t)1 << max_len);
    for (int l = 1; l <= max_len; l++) excess += (int64_t)bl[l] << (max_len - l);
    while (excess > 0) {
      int moved = 0;
      for (int l = max_len - 1; l >= 1 && excess > 0; l--) {
        const int64_t unit = (int64_t)1 << (max_len - l - 1);
        int64_t t = excess / unit;
        if (t > bl[l]) t = bl[l];
        bl[l] -= (int)t;
        bl[l + 1] += (int)t;
        excess -= t * unit;
        moved += t > 0;
      }
      if (excess > 0 && !moved) {
        int l = max_len - 1;
        while (l >= 1 && bl[l] == 0) l--;
        bl[l] -= 1;
        bl[l + 1] += 1;
        excess -= (int64_t)1 << (max_len - l - 1);
      }
    }
  }
  /* hand out lengths by rank, most frequent first */
  int l = 1, left = bl[1];
  for (int k = n - 1; k >= 0; k--) {
    while (left == 0) {
      l++;
      left = bl[l];
    }
    len[lv[k].sym] = (uint8_t)l;
    left--;
  }
  free(lv); free(wi); free(par_leaf); free(par_int); free(dep);
  return ORA_OK;
}

/* Canonical code assignment: live symbols ordered by (length, symbol); each
 * code is the previous plus one, shifted left when the length grows. */
typedef struct {
  int nlive;
  uint16_t sym[65536]; /* canonical order */
  uint8_t len[65536];
  uint32_t code_of[65536];
  uint8_t len_of[65536];
} codebook;

static void canonical(const uint8_t* len, int nsym, codebook* cb) {
  cb->nlive = 0;
  memset(cb->len_of, 0, (size_t)nsym);
  for (int l = 1; l <= 24; l++)
    for (int s = 0; s < nsym; s++)
      if (len[s] == l) {
        cb->sym[cb->nlive] = (uint16_t)s;
        cb->len[cb->nlive] = (uint8_t)l;
        cb->nlive++;
      }
  uint32_t code = 0;
  int prev = cb->nlive ? cb->len[0] : 0;
  for (int k = 0; k < cb->nlive; k++) {
    if (cb->len[k] > prev) code <<= (cb->len[k] - prev);
    prev = cb->len[k];
    cb->code_of[cb->sym[k]] = code;
    cb->len_of[cb->sym[k]] = cb->len[k];
    code++;
  }
}

/* Decoding tables of a canonical code: per length the first code, the count
 * and the index of its first symbol in canonical order. */
typedef struct {
  uint32_t first[25];
  int count[25];
  int firstidx[25];
} cdec;

static void canonical_dec(const codebook* cb, cdec* d) {
  memset(d, 0, sizeof(*d));
  for (int k = 0; k < cb->nlive; k++) d->count[cb->len[k]]++;
  uint32_t code = 0;
  int idx = 0;
  for (int l = 1; l <= 24; l++) {
    code <<= 1;
    d->first[l] = code;
    d->firstidx[l] = idx;
    code += (uint32_t)d->count[l];
    idx += d->count[l];
  }
}

/* ------------------------------------------------------------------------ */
/* Container                                                                  */
/* ------------------------------------------------------------------------ */

static size_t al4(size_t v) { return (v + 3) & ~(size_t)3; }
static size_t al8(size_t v) { return (v + 7) & ~(size_t)7; }

typedef struct {
  size_t off_syms, off_lens, off_chunks, off_subs, off_payload, off_opos, off_oval, size;
} sect_layout;

static void sect_of(uint64_t nlive, uint64_t nchunks, uint64_t pw, uint64_t no,
                    size_t ps, int nsub, sect_layout* s) {
  s->off_syms = 0;
  s->off_lens = 2 * nlive;
  s->off_chunks = al4(3 * nlive);
  s->off_subs = s->off_chunks + 4 * nchunks;
  s->off_payload = al4(s->off_subs + 2 * nchunks * (uint64_t)(nsub - 1));
  s->off_opos = s->off_payload + 4 * pw;
  s->off_oval = al8(s->off_opos + 4 * no);
  s->size = al8(s->off_oval + ps * no);
}

static void put16(uint8_t* p, uint16_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void put64(uint8_t* p, uint64_t v) {
  for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void putf64(uint8_t* p, double v) {
  uint64_t u;
  memcpy(&u, &v, 8);
  put64(p, u);
}
static uint16_t get16(const uint8_t* p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t get32(const uint8_t* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
static uint64_t get64(const uint8_t* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i);
  return v;
}
static double getf64(const uint8_t* p) {
  uint64_t u = get64(p);
  double v;
  memcpy(&v, &u, 8);
  return v;
}

static int check_params(const ora_params* p) {
  if (p->dtype != ORA_F32 && p->dtype != ORA_F64) return ORA_ERR_ARG;
  if (p->ndim != 2 && p->ndim != 3) return ORA_ERR_ARG;
  for (int a = 0; a < 3; a++)
    if (p->dims[a] < 1) return ORA_ERR_ARG;
  if (p->ndim == 2 && p->dims[0] != 1) return ORA_ERR_ARG;
  if (p->eb_mode != ORA_EB_ABS && p->eb_mode != ORA_EB_REL) return ORA_ERR_ARG;
  if (!(p->eb > 0.0) || !isfinite(p->eb)) return ORA_ERR_ARG;
  if (p->levels < 1 || p->levels > ORA_MAX_LEVELS) return ORA_ERR_ARG;
  if (p->radius < 2 || p->radius > 32768) return ORA_ERR_ARG;
  if (p->max_code_len < 1 || p->max_code_len > 24) return ORA_ERR_ARG;
  if ((int64_t)2 * p->radius > ((int64_t)1 << p->max_code_len)) return ORA_ERR_ARG;
  for (int a = 0; a < 3; a++)
    if (p->brick[a] < 1 || p->brick[a] > 4096) return ORA_ERR_ARG;
  if ((int64_t)p->brick[0] * p->brick[1] * p->brick[2] * p->max_code_len > 65535) return ORA_ERR_ARG;
  if (p->nsub != 1 && p->nsub != 2 && p->nsub != 4 && p->nsub != 8) return ORA_ERR_ARG;
  if (p->predictor != ORA_PRED_CUBIC && p->predictor != ORA_PRED_LINEAR &&
      p->predictor != ORA_PRED_DIRECT)
    return ORA_ERR_ARG;
  if (p->eb_ratio != 0.0 && !(p->eb_ratio >= 1.0 && p->eb_ratio <= 64.0)) return ORA_ERR_ARG;
  return ORA_OK;
}

static void geom_of(const ora_params* p, geom* g) {
  for (int a = 0; a < 3; a++) {
    g->n[a] = p->dims[a];
    g->b[a] = p->brick[a];
  }
  g->L = p->levels;
}

size_t ora_compress_bound(const ora_params* p) {
  if (check_params(p) != ORA_OK) return 0;
  geom g;
  geom_of(p, &g);
  int ns = nstreams_of(g.L);
  size_t ps = p->dtype == ORA_F32 ? 4 : 8;
  size_t total = ORA_HEADER_BYTES + (size_t)ns * ORA_DIR_ENTRY_BYTES;
  for (int s = 0; s < ns; s++) {
    int64_t e[3], nb[3];
    int o[3], lvl;
    stream_ext(&g, s, e, o, &lvl);
    brick_grid(e, g.b, nb);
    uint64_t nsym = (uint64_t)vol3(e), nch = (uint64_t)(nb[0] * nb[1] * nb[2]);
    uint64_t nlive = nsym < (uint64_t)(2 * p->radius) ? nsym : (uint64_t)(2 * p->radius);
    uint64_t pw = (nsym * (uint64_t)p->max_code_len + 31) / 32 + nch;
    sect_layout sl;
    sect_of(nlive, nch, pw, nsym, ps, p->nsub, &sl);
    total += sl.size;
  }
  return total;
}

/* Visit the stream positions of stream sid in order, giving each one's field
 * index (inverse of the brick-major order). */
static void stream_field_index(const geom* g, int sid, int64_t* idx_out) {
  int64_t e[3], nb[3];
  int o[3], lvl;
  stream_ext(g, sid, e, o, &lvl);
  brick_grid(e, g->b, nb);
  int64_t s = stride_of(g, lvl), nch = nb[0] * nb[1] * nb[2];
  for (int64_t j = 0; j < nch; j++) {
    int64_t start, count, org[3], lx[3];
    chunk_geom(e, g->b, j, &start, &count, org, lx);
    int64_t k = 0;
    for (int64_t cz = 0; cz < lx[0]; cz++)
      for (int64_t cy = 0; cy < lx[1]; cy++)
        for (int64_t cx = 0; cx < lx[2]; cx++, k++) {
          int64_t c[3] = {org[0] + cz, org[1] + cy, org[2] + cx}, gg[3];
          for (int a = 0; a < 3; a++) gg[a] = sid == 0 ? c[a] : 2 * c[a] + o[a];
          idx_out[start + k] = ((gg[0] * s) * g->n[1] + gg[1] * s) * g->n[2] + gg[2] * s;
        }
  }
}

/* shared front half of compress and quantize: bounds, codes, reconstruction */
static int encode_all(const void* field, const ora_params* p, const geom* g,
                      uint16_t* codes, int64_t* soff, void* recon, double* eb_abs,
                      double eb_lv[ORA_MAX_LEVELS + 1], double two_eb_lv[ORA_MAX_LEVELS + 1],
                      double* vmin, double* vmax) {
  int ns = nstreams_of(g->L);
  int64_t n = vol3(g->n);
  soff[0] = 0;
  for (int s = 0; s < ns; s++) {
    int64_t e[3];
    int o[3], lvl;
    stream_ext(g, s, e, o, &lvl);
    soff[s + 1] = soff[s] + vol3(e);
  }
  uint16_t* cp[1 + 7 * (ORA_MAX_LEVELS - 1)];
  for (int s = 0; s < ns; s++) cp[s] = codes + soff[s];
  int any = 0;
  *vmin = *vmax = 0.0;
  if (p->eb_mode == ORA_EB_REL) {
    if (p->dtype == ORA_F32) any = value_range_f32((const float*)field, n, vmin, vmax);
    else any = value_range_f64((const double*)field, n, vmin, vmax);
  }
  *eb_abs = eb_absolute(p->eb_mode, p->eb, any, *vmin, *vmax);
  for (int l = 0; l <= ORA_MAX_LEVELS; l++) eb_lv[l] = two_eb_lv[l] = 0.0;
  if (p->dtype == ORA_F32) {
    ctx_f32 c;
    memset(&c, 0, sizeof(c));
    c.g = g;
    c.x = (const float*)field;
    c.r = (float*)recon;
    c.codes = cp;
    c.R = p->radius;
    c.predictor = p->predictor;
    for (int l = 1; l <= g->L; l++) {
      eb_lv[l] = eb_of_level(*eb_abs, g->L, l, ratio_of(p));
      level_consts_f32(eb_lv[l], p->radius, &c.q[l]);
      two_eb_lv[l] = (double)c.q[l].two_eb;
    }
    run_base_f32(&c);
    run_levels_f32(&c, g->L);
  } else {
    ctx_f64 c;
    memset(&c, 0, sizeof(c));
    c.g = g;
    c.x = (const double*)field;
    c.r = (double*)recon;
    c.codes = cp;
    c.R = p->radius;
    c.predictor = p->predictor;
    for (int l = 1; l <= g->L; l++) {
      eb_lv[l] = eb_of_level(*eb_abs, g->L, l, ratio_of(p));
      level_consts_f64(eb_lv[l], p->radius, &c.q[l]);
      two_eb_lv[l] = c.q[l].two_eb;
    }
    run_base_f64(&c);
    run_levels_f64(&c, g->L);
  }
  return ORA_OK;
}

int ora_quantize(const void* field, const ora_params* p, uint16_t* codes,
                 int64_t* stream_off, void* recon, double* eb_out) {
  int rc = check_params(p);
  if (rc) return rc;
  geom g;
  geom_of(p, &g);
  double eb_abs, eb_lv[ORA_MAX_LEVELS + 1], two[ORA_MAX_LEVELS + 1], vmin, vmax;
  rc = encode_all(field, p, &g, codes, stream_off, recon, &eb_abs, eb_lv, two, &vmin, &vmax);
  if (rc) return rc;
  if (eb_out) {
    eb_out[0] = eb_abs;
    for (int l = 1; l <= g.L; l++) eb_out[l] = eb_lv[l];
  }
  return ORA_OK;
}

int ora_compress(const void* field, const ora_params* p, uint8_t* out, size_t cap,
                 size_t* out_bytes) {
  int rc = check_params(p);
  if (rc) return rc;
  geom g;
  geom_of(p, &g);
  int ns = nstreams_of(g.L);
  int64_t n = vol3(g.n);
  size_t ps = p->dtype == ORA_F32 ? 4 : 8;
  int nsym_alpha = 2 * p->radius;
  int64_t soff[1 + 7 * (ORA_MAX_LEVELS - 1) + 1];
  uint16_t* codes = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)(n > 0 ? n : 1));
  void* recon = malloc(ps * (size_t)n);
  codebook* cb = (codebook*)malloc(sizeof(codebook));
  uint64_t* hist = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nsym_alpha);
  uint8_t* lens = (uint8_t*)malloc((size_t)nsym_alpha);
  if (!codes || !recon || !cb || !hist || !lens) {
    free(codes); free(recon); free(cb); free(hist); free(lens);
    return ORA_ERR_NOMEM;
  }
  double eb_abs, eb_lv[ORA_MAX_LEVELS + 1], two[ORA_MAX_LEVELS + 1], vmin, vmax;
  encode_all(field, p, &g, codes, soff, recon, &eb_abs, eb_lv, two, &vmin, &vmax);

  /* pass 1: sizes of every section (payload sizes need the codebooks) */
  uint64_t nlive[64], nch[64], pw[64], nout[64];
  size_t total = ORA_HEADER_BYTES + (size_t)ns * ORA_DIR_ENTRY_BYTES;
  size_t sect_off[64];
  for (int s = 0; s < ns; s++) {
    int64_t e[3], nb[3];
    int o[3], lvl;
    stream_ext(&g, s, e, o, &lvl);
    brick_grid(e, g.b, nb);
    nch[s] = (uint64_t)(nb[0] * nb[1] * nb[2]);
    memset(hist, 0, sizeof(uint64_t) * (size_t)nsym_alpha);
    uint64_t no = 0;
    for (int64_t i = soff[s]; i < soff[s + 1]; i++) {
      hist[codes[i]]++;
      no += codes[i] == 0;
    }
    nout[s] = no;
    ora_huffman_lengths(hist, nsym_alpha, p->max_code_len, lens);
    canonical(lens, nsym_alpha, cb);
    nlive[s] = (uint64_t)cb->nlive;
    uint64_t words = 0;
    for (int64_t j = 0; j < (int64_t)nch[s]; j++) {
      int64_t start, count, org[3], lx[3];
      chunk_geom(e, g.b, j, &start, &count, org, lx);
      uint64_t bits = 0;
      for (int64_t k = 0; k < count; k++) bits += cb->len_of[codes[soff[s] + start + k]];
      words += (bits + 31) / 32;
    }
    pw[s] = words;
    sect_layout sl;
    sect_of(nlive[s], nch[s], pw[s], nout[s], ps, p->nsub, &sl);
    sect_off[s] = total;
    total += sl.size;
  }
  *out_bytes = total;
  if (total > cap) {
    free(codes); free(recon); free(cb); free(hist); free(lens);
    return ORA_ERR_CAPACITY;
  }
  memset(out, 0, total);

  /* header */
  memcpy(out, "STZ1", 4);
  put16(out + 4, 1);
  out[6] = (uint8_t)p->dtype;
  out[7] = (uint8_t)p->ndim;
  out[8] = (uint8_t)g.L;
  out[9] = (uint8_t)p->eb_mode;
  out[10] = (uint8_t)p->max_code_len;
  out[11] = (uint8_t)p->nsub;
  put32(out + 12, (uint32_t)p->radius);
  for (int a = 0; a < 3; a++) put32(out + 16 + 4 * a, (uint32_t)g.b[a]);
  put32(out + 28, (uint32_t)ns);
  for (int a = 0; a < 3; a++) put64(out + 32 + 8 * a, (uint64_t)g.n[a]);
  putf64(out + 56, p->eb);
  putf64(out + 64, eb_abs);
  putf64(out + 72, vmin);
  putf64(out + 80, vmax);
  put64(out + 88, (uint64_t)total);
  for (int l = 1; l <= g.L; l++) {
    putf64(out + 96 + 8 * (l - 1), eb_lv[l]);
    putf64(out + 144 + 8 * (l - 1), two[l]);
  }
  putf64(out + 192, ratio_of(p));
  out[200] = (uint8_t)p->predictor;

  /* directory and sections */
  int64_t* fidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int s = 0; s < ns; s++) {
    uint8_t* d = out + ORA_HEADER_BYTES + (size_t)s * ORA_DIR_ENTRY_BYTES;
    put64(d + 0, (uint64_t)sect_off[s]);
    put64(d + 8, (uint64_t)(soff[s + 1] - soff[s]));
    put32(d + 16, (uint32_t)nch[s]);
    put32(d + 20, (uint32_t)nlive[s]);
    put64(d + 24, pw[s]);
    put64(d + 32, nout[s]);

    int64_t e[3];
    int o[3], lvl;
    stream_ext(&g, s, e, o, &lvl);
    memset(hist, 0, sizeof(uint64_t) * (size_t)nsym_alpha);
    for (int64_t i = soff[s]; i < soff[s + 1]; i++) hist[codes[i]]++;
    ora_huffman_lengths(hist, nsym_alpha, p->max_code_len, lens);
    canonical(lens, nsym_alpha, cb);
    sect_layout sl;
    sect_of(nlive[s], nch[s], pw[s], nout[s], ps, p->nsub, &sl);
    uint8_t* sec = out + sect_off[s];
    for (int k = 0; k < cb->nlive; k++) {
      put16(sec + sl.off_syms + 2 * (size_t)k, cb->sym[k]);
      sec[sl.off_lens + (size_t)k] = cb->len[k];
    }
    /* chunks: MSB-first bit packing into 32-bit words */
    uint64_t wpos = 0;
    for (int64_t j = 0; j < (int64_t)nch[s]; j++) {
      int64_t start, count, org[3], lx[3];
      chunk_geom(e, g.b, j, &start, &count, org, lx);
      put32(sec + sl.off_chunks + 4 * (size_t)j, (uint32_t)wpos);
      uint64_t acc = 0;
      int nacc = 0;
      const int64_t q = (count + p->nsub - 1) / p->nsub;
      uint64_t cbits = 0;
      for (int64_t k = 0; k <= count; k++) {
        /* sub-chunk boundaries: bit position of symbol k*q (or of the end) */
        for (int u = 1; u < p->nsub; u++)
          if ((u * q < count ? u * q : count) == k)
            put16(sec + sl.off_subs + 2 * ((size_t)j * (p->nsub - 1) + (u - 1)), (uint16_t)cbits);
        if (k == count) break;
        int sym = codes[soff[s] + start + k];
        cbits += cb->len_of[sym];
        acc = (acc << cb->len_of[sym]) | cb->code_of[sym];
        nacc += cb->len_of[sym];
        while (nacc >= 32) {
          put32(sec + sl.off_payload + 4 * (size_t)wpos, (uint32_t)(acc >> (nacc - 32)));
          wpos++;
          nacc -= 32;
          acc &= nacc ? (((uint64_t)1 << nacc) - 1) : 0;
        }
      }
      if (nacc > 0) {
        put32(sec + sl.off_payload + 4 * (size_t)wpos, (uint32_t)(acc << (32 - nacc)));
        wpos++;
      }
    }
    /* outliers: ascending stream positions, raw values */
    if (nout[s] > 0) {
      stream_field_index(&g, s, fidx);
      uint64_t k = 0;
      for (int64_t i = 0; i < soff[s + 1] - soff[s]; i++) {
        if (codes[soff[s] + i] != 0) continue;
        put32(sec + sl.off_opos + 4 * k, (uint32_t)i);
        if (p->dtype == ORA_F32) {
          float v = ((const float*)field)[fidx[i]];
          memcpy(sec + sl.off_oval + 4 * k, &v, 4);
        } else {
          double v = ((const double*)field)[fidx[i]];
          memcpy(sec + sl.off_oval + 8 * k, &v, 8);
        }
        k++;
      }
    }
  }
  free(fidx);
  free(codes); free(recon); free(cb); free(hist); free(lens);
  return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Parsing and validation                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  ora_info info;
  geom g;
  size_t ps;
  uint64_t sect_off[64], nsym[64], nch[64], nlive[64], pw[64], nout[64];
  sect_layout sl[64];
} parsed;

static int parse(const uint8_t* c, size_t nbytes, parsed* P) {
  memset(P, 0, sizeof(*P));
  if (!c || nbytes < ORA_HEADER_BYTES) return ORA_ERR_CORRUPT;
  if (memcmp(c, "STZ1", 4) != 0 || get16(c + 4) != 1) return ORA_ERR_CORRUPT;
  ora_params* p = &P->info.p;
  p->dtype = c[6];
  p->ndim = c[7];
  p->levels = c[8];
  p->eb_mode = c[9];
  p->max_code_len = c[10];
  p->nsub = c[11];
  p->radius = (int)get32(c + 12);
  for (int a = 0; a < 3; a++) p->brick[a] = (int)get32(c + 16 + 4 * a);
  P->info.nstreams = (int)get32(c + 28);
  for (int a = 0; a < 3; a++) p->dims[a] = (int64_t)get64(c + 32 + 8 * a);
  p->eb = getf64(c + 56);
  p->eb_ratio = getf64(c + 192);
  p->predictor = c[200];
  P->info.eb_abs = getf64(c + 64);
  P->info.total_bytes = get64(c + 88);
  if (check_params(p) != ORA_OK) return ORA_ERR_CORRUPT;
  if (P->info.nstreams != nstreams_of(p->levels)) return ORA_ERR_CORRUPT;
  if (P->info.total_bytes > nbytes) return ORA_ERR_CORRUPT;
  for (int l = 1; l <= p->levels; l++) {
    P->info.eb_level[l] = getf64(c + 96 + 8 * (l - 1));
    P->info.two_eb[l] = getf64(c + 144 + 8 * (l - 1));
  }
  geom_of(p, &P->g);
  P->ps = p->dtype == ORA_F32 ? 4 : 8;
  size_t total = (size_t)P->info.total_bytes;
  int ns = P->info.nstreams;
  if ((uint64_t)ORA_HEADER_BYTES + (uint64_t)ns * ORA_DIR_ENTRY_BYTES > total) return ORA_ERR_CORRUPT;
  for (int s = 0; s < ns; s++) {
    const uint8_t* d = c + ORA_HEADER_BYTES + (size_t)s * ORA_DIR_ENTRY_BYTES;
    P->sect_off[s] = get64(d);
    P->nsym[s] = get64(d + 8);
    P->nch[s] = get32(d + 16);
    P->nlive[s] = get32(d + 20);
    P->pw[s] = get64(d + 24);
    P->nout[s] = get64(d + 32);
    int64_t e[3], nb[3];
    int o[3], lvl;
    stream_ext(&P->g, s, e, o, &lvl);
    brick_grid(e, P->g.b, nb);
    if (P->nsym[s] != (uint64_t)vol3(e)) return ORA_ERR_CORRUPT;
    if (P->nch[s] != (uint64_t)(nb[0] * nb[1] * nb[2])) return ORA_ERR_CORRUPT;
    if (P->nlive[s] > (uint64_t)(2 * p->radius)) return ORA_ERR_CORRUPT;
    if (P->nsym[s] > 0 && P->nlive[s] == 0) return ORA_ERR_CORRUPT;
    if (P->nout[s] > P->nsym[s]) return ORA_ERR_CORRUPT;
    if (P->pw[s] > P->nsym[s] * 24 + P->nch[s]) return ORA_ERR_CORRUPT;
    if (P->sect_off[s] % 8 != 0 || P->sect_off[s] > total) return ORA_ERR_CORRUPT;
    sect_of(P->nlive[s], P->nch[s], P->pw[s], P->nout[s], P->ps, p->nsub, &P->sl[s]);
    if (P->sl[s].size > total - P->sect_off[s]) return ORA_ERR_CORRUPT;
  }
  return ORA_OK;
}

int ora_parse_info(const uint8_t* comp, size_t comp_bytes, ora_info* info) {
  parsed* P = (parsed*)malloc(sizeof(parsed));
  if (!P) return ORA_ERR_NOMEM;
  int rc = parse(comp, comp_bytes, P);
  if (rc == ORA_OK) *info = P->info;
  free(P);
  return rc;
}

/* Read the codebook of stream s and check it is a canonical prefix code. */
static int read_codebook(const uint8_t* c, const parsed* P, int s, codebook* cb) {
  const uint8_t* sec = c + P->sect_off[s];
  const sect_layout* sl = &P->sl[s];
  int nsym_alpha = 2 * P->info.p.radius;
  cb->nlive = (int)P->nlive[s];
  double kraft = 0.0;
  for (int k = 0; k < cb->nlive; k++) {
    cb->sym[k] = get16(sec + sl->off_syms + 2 * (size_t)k);
    cb->len[k] = sec[sl->off_lens + (size_t)k];
    if (cb->sym[k] >= nsym_alpha) return ORA_ERR_CORRUPT;
    if (cb->len[k] < 1 || cb->len[k] > P->info.p.max_code_len) return ORA_ERR_CORRUPT;
    if (k > 0 && !(cb->len[k] > cb->len[k - 1] ||
                   (cb->len[k] == cb->len[k - 1] && cb->sym[k] > cb->sym[k - 1])))
      return ORA_ERR_CORRUPT;
    kraft += ldexp(1.0, -cb->len[k]);
  }
  if (kraft > 1.0) return ORA_ERR_CORRUPT;
  return ORA_OK;
}

/* Entropy-decode stream s into dst[0..nsym), bit by bit against the
 * canonical code. */
static int decode_stream(const uint8_t* c, const parsed* P, int s, uint16_t* dst,
                         codebook* cb) {
  int rc = read_codebook(c, P, s, cb);
  if (rc) return rc;
  cdec dt;
  canonical_dec(cb, &dt);
  const uint8_t* sec = c + P->sect_off[s];
  const sect_layout* sl = &P->sl[s];
  int64_t e[3];
  int o[3], lvl;
  stream_ext(&P->g, s, e, o, &lvl);
  int maxl = P->info.p.max_code_len;
  for (int64_t j = 0; j < (int64_t)P->nch[s]; j++) {
    int64_t start, count, org[3], lx[3];
    chunk_geom(e, P->g.b, j, &start, &count, org, lx);
    uint64_t w0 = get32(sec + sl->off_chunks + 4 * (size_t)j);
    uint64_t w1 = j + 1 < (int64_t)P->nch[s] ? get32(sec + sl->off_chunks + 4 * (size_t)(j + 1))
                                             : P->pw[s];
    if (w0 > w1 || w1 > P->pw[s]) return ORA_ERR_CORRUPT;
    uint64_t bit = 0, nbits = (w1 - w0) * 32;
    const int nsub = P->info.p.nsub;
    const int64_t q = (count + nsub - 1) / nsub;
    for (int64_t k = 0; k <= count; k++) {
      for (int u = 1; u < nsub; u++)
        if ((u * q < count ? u * q : count) == k &&
            get16(sec + sl->off_subs + 2 * ((size_t)j * (nsub - 1) + (u - 1))) != bit)
          return ORA_ERR_CORRUPT;
      if (k == count) break;
      uint32_t code = 0;
      int l = 0, found = 0;
      while (!found) {
        if (bit >= nbits || l >= maxl) return ORA_ERR_CORRUPT;
        uint32_t word = get32(sec + sl->off_payload + 4 * (size_t)(w0 + bit / 32));
        code = (code << 1) | ((word >> (31 - bit % 32)) & 1u);
        bit++;
        l++;
        if (dt.count[l] > 0 && code >= dt.first[l] && code - dt.first[l] < (uint32_t)dt.count[l]) {
          dst[start + k] = cb->sym[dt.firstidx[l] + (int)(code - dt.first[l])];
          found = 1;
        }
      }
    }
  }
  /* outliers: ascending positions, each on a symbol 0, one per symbol 0 */
  uint64_t zeros = 0;
  for (uint64_t i = 0; i < P->nsym[s]; i++) zeros += dst[i] == 0;
  if (zeros != P->nout[s]) return ORA_ERR_CORRUPT;
  for (uint64_t k = 0; k < P->nout[s]; k++) {
    uint32_t pos = get32(sec + sl->off_opos + 4 * k);
    if (pos >= P->nsym[s] || dst[pos] != 0) return ORA_ERR_CORRUPT;
    if (k > 0 && pos <= get32(sec + sl->off_opos + 4 * (k - 1))) return ORA_ERR_CORRUPT;
  }
  return ORA_OK;
}

int ora_decode_streams(const uint8_t* comp, size_t comp_bytes, uint16_t* codes,
                       int64_t* stream_off) {
  parsed* P = (parsed*)malloc(sizeof(parsed));
  codebook* cb = (codebook*)malloc(sizeof(codebook));
  if (!P || !cb) { free(P); free(cb); return ORA_ERR_NOMEM; }
  int rc = parse(comp, comp_bytes, P);
  if (rc == ORA_OK) {
    stream_off[0] = 0;
    for (int s = 0; s < P->info.nstreams; s++) stream_off[s + 1] = stream_off[s] + (int64_t)P->nsym[s];
    for (int s = 0; s < P->info.nstreams && rc == ORA_OK; s++)
      rc = decode_stream(comp, P, s, codes + stream_off[s], cb);
  }
  free(P);
  free(cb);
  return rc;
}

/* Decode levels 1..level into a full-resolution array (points of G_level
 * filled).  *recon_out is allocated here. */
static int decode_to_level(const uint8_t* comp, size_t comp_bytes, int level, parsed* P,
                           void** recon_out) {
  int rc = parse(comp, comp_bytes, P);
  if (rc) return rc;
  if (level < 1 || level > P->info.p.levels) return ORA_ERR_ARG;
  int ns = 1 + 7 * (level - 1);
  int64_t n = vol3(P->g.n);
  int64_t soff[64];
  soff[0] = 0;
  for (int s = 0; s < ns; s++) soff[s + 1] = soff[s] + (int64_t)P->nsym[s];
  uint16_t* codes = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)(soff[ns] > 0 ? soff[ns] : 1));
  codebook* cb = (codebook*)malloc(sizeof(codebook));
  void* r = calloc((size_t)n, P->ps);
  if (!codes || !cb || !r) { free(codes); free(cb); free(r); return ORA_ERR_NOMEM; }
  for (int s = 0; s < ns && rc == ORA_OK; s++) rc = decode_stream(comp, P, s, codes + soff[s], cb);
  if (rc) { free(codes); free(cb); free(r); return rc; }
  uint16_t* cp[64];
  const uint32_t* opos[64];
  const float* ovf[64];
  const double* ovd[64];
  int64_t nout[64];
  uint32_t* posbuf[64];
  void* valbuf[64];
  for (int s = 0; s < ns; s++) {
    cp[s] = codes + soff[s];
    const uint8_t* sec = comp + P->sect_off[s];
    posbuf[s] = (uint32_t*)malloc(4 * (size_t)(P->nout[s] + 1));
    valbuf[s] = malloc(P->ps * (size_t)(P->nout[s] + 1));
    for (uint64_t k = 0; k < P->nout[s]; k++) posbuf[s][k] = get32(sec + P->sl[s].off_opos + 4 * k);
    memcpy(valbuf[s], sec + P->sl[s].off_oval, P->ps * (size_t)P->nout[s]);
    opos[s] = posbuf[s];
    ovf[s] = (const float*)valbuf[s];
    ovd[s] = (const double*)valbuf[s];
    nout[s] = (int64_t)P->nout[s];
  }
  int err = 0;
  if (P->info.p.dtype == ORA_F32) {
    ctx_f32 c;
    memset(&c, 0, sizeof(c));
    c.g = &P->g;
    c.decode = 1;
    c.r = (float*)r;
    c.codes = cp;
    c.opos = opos;
    c.oval = ovf;
    c.nout = nout;
    c.R = P->info.p.radius;
    c.predictor = P->info.p.predictor;
    for (int l = 1; l <= P->g.L; l++) c.q[l].two_eb = (float)P->info.two_eb[l];
    run_base_f32(&c);
    run_levels_f32(&c, level);
    err = c.err;
  } else {
    ctx_f64 c;
    memset(&c, 0, sizeof(c));
    c.g = &P->g;
    c.decode = 1;
    c.r = (double*)r;
    c.codes = cp;
    c.opos = opos;
    c.oval = ovd;
    c.nout = nout;
    c.R = P->info.p.radius;
    c.predictor = P->info.p.predictor;
    for (int l = 1; l <= P->g.L; l++) c.q[l].two_eb = P->info.two_eb[l];
    run_base_f64(&c);
    run_levels_f64(&c, level);
    err = c.err;
  }
  for (int s = 0; s < ns; s++) {
    free(posbuf[s]);
    free(valbuf[s]);
  }
  free(codes);
  free(cb);
  if (err) { free(r); return ORA_ERR_CORRUPT; }
  *recon_out = r;
  return ORA_OK;
}

int ora_decompress(const uint8_t* comp, size_t comp_bytes, int level, void* out,
                   size_t out_cap_bytes, int64_t out_dims[3]) {
  int64_t lo[3] = {0, 0, 0}, hi[3];
  parsed* P = (parsed*)malloc(sizeof(parsed));
  if (!P) return ORA_ERR_NOMEM;
  int rc = parse(comp, comp_bytes, P);
  if (rc) { free(P); return rc; }
  for (int a = 0; a < 3; a++) hi[a] = P->g.n[a];
  free(P);
  return ora_decompress_region(comp, comp_bytes, lo, hi, level, out, out_cap_bytes, out_dims);
}

/* A region is, by definition, the box's points of the level's lattice taken
 * from the decode to that level (Sec. 3.3: only the predictions a box needs
 * are made, and they equal those of the full decode). */
int ora_decompress_region(const uint8_t* comp, size_t comp_bytes, const int64_t lo[3],
                          const int64_t hi[3], int level, void* out, size_t out_cap_bytes,
                          int64_t out_dims[3]) {
  parsed* P = (parsed*)malloc(sizeof(parsed));
  if (!P) return ORA_ERR_NOMEM;
  int rc = parse(comp, comp_bytes, P);
  if (rc) { free(P); return rc; }
  if (level < 1 || level > P->info.p.levels) { free(P); return ORA_ERR_ARG; }
  for (int a = 0; a < 3; a++)
    if (lo[a] < 0 || hi[a] > P->g.n[a] || lo[a] >= hi[a]) { free(P); return ORA_ERR_ARG; }
  int64_t s = stride_of(&P->g, level), first[3];
  for (int a = 0; a < 3; a++) {
    first[a] = cdiv64(lo[a], s);
    out_dims[a] = cdiv64(hi[a], s) - first[a];
  }
  size_t need = (size_t)(out_dims[0] * out_dims[1] * out_dims[2]) * P->ps;
  if (need > out_cap_bytes) { free(P); return ORA_ERR_CAPACITY; }
  void* r = NULL;
  rc = decode_to_level(comp, comp_bytes, level, P, &r);
  if (rc) { free(P); return rc; }
  int64_t k = 0;
  for (int64_t z = 0; z < out_dims[0]; z++)
    for (int64_t y = 0; y < out_dims[1]; y++)
      for (int64_t x = 0; x < out_dims[2]; x++, k++) {
        int64_t idx = (((first[0] + z) * s) * P->g.n[1] + (first[1] + y) * s) * P->g.n[2] +
                      (first[2] + x) * s;
        if (P->ps == 4) ((float*)out)[k] = ((float*)r)[idx];
        else ((double*)out)[k] = ((double*)r)[idx];
      }
  free(r);
  free(P);
  return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Single-point predictions for the stencil tests                            */
/* ------------------------------------------------------------------------ */

double ora_predict_f64(const double* grid, const int64_t n[3], int levels, int level,
                       const int64_t g[3], int axis, int64_t t) {
  geom gg;
  for (int a = 0; a < 3; a++) { gg.n[a] = n[a]; gg.b[a] = 1; }
  gg.L = levels;
  int64_t m[3], s = stride_of(&gg, level);
  grid_ext(&gg, level, m);
  int64_t p[3] = {g[0] / s, g[1] / s, g[2] / s};
  if (level == 1) return base_pred_f64(grid, n, s, m, p, axis, t);
  return level_pred_f64(grid, n, s, m, p, ORA_PRED_CUBIC);
}

double ora_predict_mode_f64(const double* grid, const int64_t n[3], int levels, int level,
                            const int64_t g[3], int predictor) {
  geom gg;
  for (int a = 0; a < 3; a++) { gg.n[a] = n[a]; gg.b[a] = 1; }
  gg.L = levels;
  if (level < 2 || level > levels) return 0.0;
  int64_t m[3], s = stride_of(&gg, level);
  grid_ext(&gg, level, m);
  int64_t p[3] = {g[0] / s, g[1] / s, g[2] / s};
  return level_pred_f64(grid, n, s, m, p, predictor);
}

float ora_predict_f32(const float* grid, const int64_t n[3], int levels, int level,
                      const int64_t g[3], int axis, int64_t t) {
  geom gg;
  for (int a = 0; a < 3; a++) { gg.n[a] = n[a]; gg.b[a] = 1; }
  gg.L = levels;
  int64_t m[3], s = stride_of(&gg, level);
  grid_ext(&gg, level, m);
  int64_t p[3] = {g[0] / s, g[1] / s, g[2] / s};
  if (level == 1) return base_pred_f32(grid, n, s, m, p, axis, t);
  return level_pred_f32(grid, n, s, m, p, ORA_PRED_CUBIC);
}
