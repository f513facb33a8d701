/*
 * stz_oracle.h -- plain, slow, single-threaded CPU oracle of the STZ streaming
 * compressor (Sec. 3 of "STZ: A High Quality and High Speed Streaming Lossy
 * Compression Framework for Scientific Data", SC'25).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  The product path (the CUDA
 * library) shares no code, header, table or helper with it.
 *
 * What it computes, step by step in the paper's order:
 *   1. value range and error bounds (adaptive per-level bound, Sec. 3.1 opt. 5:
 *      a coarser level gets the bound of the next finer one divided by 2.5);
 *   2. hierarchical partition (Sec. 3.1 / 3.2): level l has stride
 *      s_l = 2^(L-l); level 1 is every point whose coordinates are all
 *      multiples of s_1; level l >= 2 is the points of the stride-s_l grid
 *      that are not on the stride-2*s_l grid, split into 7 (3D) or 3 (2D)
 *      sub-blocks by which coordinates are odd multiples of s_l;
 *   3. level 1 is coded by an SZ3-style 1D interpolation coder (Sec. 3.1
 *      opt. 3, Sec. 4.4) -- the base passes below;
 *   4. every finer level is predicted from the reconstructed coarser grid by
 *      multi-dimensional cubic interpolation (Eqs. 6, 7, 8), with linear
 *      interpolation (Eqs. 3-5) and one-sided rules at the field boundary
 *      (Sec. 3.1 opt. 2 "boundary points ... predicted directly");
 *   5. linear-scale quantization of the prediction error with outliers;
 *   6. Huffman coding of each sub-block's codes as one unit (Sec. 3.3), cut
 *      into independently decodable chunks (random access, Sec. 5 future
 *      work);
 *   7. full, progressive (Sec. 3.3 "progressive decompression") and region
 *      (Sec. 3.3 "random access decompression") decoding.
 *
 * Readings where the paper is silent are fixed here and listed in the design
 * notes: the base coder, the boundary rules, the quantizer formula, the
 * Huffman tie-breaks and length limit, the chunk/brick layout and the byte
 * format.  All arithmetic on field values is done in the field's precision P
 * (float for f32 fields, double for f64) with correctly rounded single
 * operations in a fixed order and no fused multiply-add, so that compressor
 * and decompressor predict identically.
 *
 * Parity status of each function is stated at its definition in
 * stz_oracle.c.
 */
#ifndef STZ_ORACLE_H
#define STZ_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORA_OK = 0,
  ORA_ERR_ARG = -1,
  ORA_ERR_CAPACITY = -2,
  ORA_ERR_CORRUPT = -3,
  ORA_ERR_NOMEM = -6
};

enum { ORA_F32 = 0, ORA_F64 = 1 };
enum { ORA_EB_ABS = 0, ORA_EB_REL = 1 };

/* Container constants (byte format, see stz_oracle.c "Byte format"). */
#define ORA_HEADER_BYTES 256
#define ORA_DIR_ENTRY_BYTES 48
#define ORA_MAX_LEVELS 6

/* Compression parameters.  dims are (nz, ny, nx), x fastest; a 2D field has
 * ndim = 2 and nz = 1. */
typedef struct {
  int dtype;          /* ORA_F32 or ORA_F64 */
  int ndim;           /* 2 or 3 */
  int64_t dims[3];    /* (nz, ny, nx) */
  int eb_mode;        /* ORA_EB_ABS or ORA_EB_REL */
  double eb;          /* > 0, finite */
  int levels;         /* L, 1..ORA_MAX_LEVELS */
  int radius;         /* quantization radius R, 2..32768 */
  int max_code_len;   /* Huffman length limit, 1..24 */
  int brick[3];       /* chunk brick (bz, by, bx) in sub-block cells */
  int nsub;           /* sub-chunks per chunk: 1, 2, 4 or 8 */
  /* Prediction of levels 2..L (the ablation of Sec. 3.1, Fig. 2):
   * ORA_PRED_CUBIC  = opt. 4, Eqs. 6-8 (the method; default),
   * ORA_PRED_LINEAR = opt. 2, multi-linear Eqs. 3-5,
   * ORA_PRED_DIRECT = opt. 1, Eq. 1 (the coarse point at the cell). */
  int predictor;
  /* Adaptive bound of Sec. 3.1 opt. 5: eb_l = eb_{l+1} / eb_ratio.  0 means
   * the paper's 2.5; 1 switches the adaptive bound off. */
  double eb_ratio;
} ora_params;

enum { ORA_PRED_CUBIC = 0, ORA_PRED_LINEAR = 1, ORA_PRED_DIRECT = 2 };

/* Upper bound on the container size for the given parameters. */
size_t ora_compress_bound(const ora_params* p);

/* Compress `field` (C order, dtype p->dtype).  Writes the container to
 * out[0..*out_bytes).  Returns ORA_OK, ORA_ERR_ARG or ORA_ERR_CAPACITY (then
 * *out_bytes holds the needed size). */
int ora_compress(const void* field, const ora_params* p, uint8_t* out,
                 size_t cap, size_t* out_bytes);

/* Quantization codes and reconstruction without the entropy stage: codes of
 * every stream concatenated in stream order (stream s occupies
 * codes[stream_off[s] .. stream_off[s+1])), outliers marked by symbol 0, and
 * the reconstructed field (what a full decode returns).  stream_off has
 * nstreams + 1 entries, nstreams = 1 + 7 (L - 1).  eb_out[0] = eb_abs,
 * eb_out[l] = bound of level l. */
int ora_quantize(const void* field, const ora_params* p, uint16_t* codes,
                 int64_t* stream_off, void* recon, double* eb_out);

/* Decode to level `level` (1..L; L = full resolution).  The output is the
 * stride-2^(L-level) grid, out_dims = ceil(n / 2^(L-level)) per axis (z, y,
 * x).  Returns ORA_ERR_CORRUPT on any inconsistency in the container. */
int ora_decompress(const uint8_t* comp, size_t comp_bytes, int level,
                   void* out, size_t out_cap_bytes, int64_t out_dims[3]);

/* Region [lo, hi) (field coordinates, z y x) at level `level`: the points of
 * the box whose coordinates are multiples of 2^(L-level), in C order. */
int ora_decompress_region(const uint8_t* comp, size_t comp_bytes,
                          const int64_t lo[3], const int64_t hi[3], int level,
                          void* out, size_t out_cap_bytes,
                          int64_t out_dims[3]);

/* Entropy-decode every stream of a container: symbols in stream order into
 * codes (stream s at stream_off[s]); no reconstruction. */
int ora_decode_streams(const uint8_t* comp, size_t comp_bytes,
                       uint16_t* codes, int64_t* stream_off);

/* Parsed header (subset) for tests. */
typedef struct {
  ora_params p;
  double eb_abs;
  double eb_level[ORA_MAX_LEVELS + 1];   /* index 1..L */
  double two_eb[ORA_MAX_LEVELS + 1];     /* 2*eb_l rounded to P */
  int nstreams;
  uint64_t total_bytes;
} ora_info;
int ora_parse_info(const uint8_t* comp, size_t comp_bytes, ora_info* info);

/* Huffman code lengths (two-queue construction, then length limiting):
 * freq[0..nsym), len[0..nsym) out (0 for absent symbols). */
int ora_huffman_lengths(const uint64_t* freq, int nsym, int max_len,
                        uint8_t* len);

/* Prediction of one point from a full-resolution grid `grid` (z y x, dims n)
 * treated as the reconstructed data: level >= 2 uses the multi-dimensional
 * stencils, level 1 with `axis` in 0..2 and `t` the pass stride uses the
 * base coder's 1D rule.  g is the point in field coordinates.  For tests. */
double ora_predict_f64(const double* grid, const int64_t n[3], int levels,
                       int level, const int64_t g[3], int axis, int64_t t);
/* The same for levels >= 2 with a chosen predictor (ORA_PRED_*). */
double ora_predict_mode_f64(const double* grid, const int64_t n[3], int levels,
                            int level, const int64_t g[3], int predictor);
float ora_predict_f32(const float* grid, const int64_t n[3], int levels,
                      int level, const int64_t g[3], int axis, int64_t t);

/* ROI selection module (Sec. 3.3, last paragraph; stz_oracle_roi.c): per
 * unit -- a block of block[3] points (z, y, x), clipped at the field's edge;
 * a slice along an axis is a block spanning the other two axes -- the value
 * range or the maximum of its finite values (-inf without one), then the
 * units with metric >= value (ORA_ROI_THRESHOLD) or the ceil(value * nunits)
 * largest, ties to the lower index (ORA_ROI_TOP, 0 < value <= 1).  sel
 * receives the selected unit indices ascending (room for nunits), metric_out
 * (may be NULL) every unit's metric. */
enum { ORA_ROI_RANGE = 0, ORA_ROI_MAX = 1 };
enum { ORA_ROI_THRESHOLD = 0, ORA_ROI_TOP = 1 };
int64_t ora_roi_units(const int64_t dims[3], const int64_t block[3]);
int ora_roi_select(const void* field, int dtype, const int64_t dims[3], const int64_t block[3],
                   int metric, int mode, double value, double* metric_out, int64_t* sel,
                   int64_t* nsel);

/* Stream position (brick-major order) of cell c in a sub-block of extent e
 * with brick b.  For tests. */
int64_t ora_stream_pos(const int64_t e[3], const int b[3], const int64_t c[3]);

#ifdef __cplusplus
}
#endif
#endif
