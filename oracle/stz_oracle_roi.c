/*
 * stz_oracle_roi.c -- the ROI selection module of Sec. 3.3 (last paragraph),
 * plainly: for each unit of a field (a block of bz x by x bx points, clipped
 * at the field's edge; a slice along an axis is the block that spans the
 * other two axes), the value range (max - min) or the maximum of its finite
 * values, then the units whose metric reaches a threshold, or the top x% of
 * units by metric.
 *
 * TEST INFRASTRUCTURE (see stz_oracle.h): only the tests, the smoke check and
 * the benchmark's CPU legs load it.
 *
 * Readings (the paper gives the idea, not the rules):
 *   - non-finite values are ignored (and -0 orders below +0); a unit without
 *     a finite value has the metric -infinity (never reaches a finite
 *     threshold, ranks last);
 *   - range = (double)max - (double)min, one correctly rounded subtraction;
 *   - threshold mode selects metric >= threshold;
 *   - top mode selects k = ceil(fraction * nunits) units (fraction in (0, 1],
 *     the product in double), the largest metrics first, equal metrics by
 *     lower unit index;
 *   - the selection is returned as ascending unit indices; units are
 *     numbered in raster order of (z / bz, y / by, x / bx).
 * Parity pins: closed forms on linear fields (the range of a slice of
 * f = a z + b y + c x is known exactly) and brute force with numpy on random
 * fields with ties and non-finite values (tests/test_oracle_roi.py).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "stz_oracle.h"

typedef struct {
  double m;
  int64_t i;
} ranked;

static int by_metric_desc(const void* pa, const void* pb) {
  const ranked* a = (const ranked*)pa;
  const ranked* b = (const ranked*)pb;
  if (a->m > b->m) return -1;
  if (a->m < b->m) return 1;
  return a->i < b->i ? -1 : (a->i > b->i ? 1 : 0);
}

static int by_index(const void* pa, const void* pb) {
  int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
  return a < b ? -1 : (a > b ? 1 : 0);
}

int64_t ora_roi_units(const int64_t dims[3], const int64_t block[3]) {
  int64_t n = 1;
  for (int a = 0; a < 3; a++) {
    if (dims[a] < 1 || block[a] < 1) return -1;
    n *= (dims[a] + block[a] - 1) / block[a];
  }
  return n;
}

int ora_roi_select(const void* field, int dtype, const int64_t dims[3], const int64_t block[3],
                   int metric, int mode, double value, double* metric_out, int64_t* sel,
                   int64_t* nsel) {
  if (dtype != ORA_F32 && dtype != ORA_F64) return ORA_ERR_ARG;
  if (metric != ORA_ROI_RANGE && metric != ORA_ROI_MAX) return ORA_ERR_ARG;
  if (mode != ORA_ROI_THRESHOLD && mode != ORA_ROI_TOP) return ORA_ERR_ARG;
  if (mode == ORA_ROI_TOP && !(value > 0.0 && value <= 1.0)) return ORA_ERR_ARG;
  int64_t nu = ora_roi_units(dims, block);
  if (nu < 1) return ORA_ERR_ARG;
  int64_t nb[3];
  for (int a = 0; a < 3; a++) nb[a] = (dims[a] + block[a] - 1) / block[a];
  double* lo = (double*)malloc(sizeof(double) * (size_t)nu);
  double* hi = (double*)malloc(sizeof(double) * (size_t)nu);
  char* any = (char*)calloc((size_t)nu, 1);
  ranked* r = (ranked*)malloc(sizeof(ranked) * (size_t)nu);
  if (!lo || !hi || !any || !r) {
    free(lo); free(hi); free(any); free(r);
    return ORA_ERR_NOMEM;
  }
  /* every point, in raster order, into its unit's minimum and maximum */
  for (int64_t z = 0; z < dims[0]; z++)
    for (int64_t y = 0; y < dims[1]; y++)
      for (int64_t x = 0; x < dims[2]; x++) {
        int64_t i = (z * dims[1] + y) * dims[2] + x;
        double v = dtype == ORA_F32 ? (double)((const float*)field)[i]
                                    : ((const double*)field)[i];
        if (!isfinite(v)) continue;
        int64_t u = ((z / block[0]) * nb[1] + y / block[1]) * nb[2] + x / block[2];
        /* ties between the zeros are broken as -0 < +0, so that the result
         * does not depend on the visiting order */
        if (!any[u]) {
          lo[u] = hi[u] = v;
          any[u] = 1;
        } else {
          if (v < lo[u] || (v == lo[u] && signbit(v) && !signbit(lo[u]))) lo[u] = v;
          if (v > hi[u] || (v == hi[u] && !signbit(v) && signbit(hi[u]))) hi[u] = v;
        }
      }
  for (int64_t u = 0; u < nu; u++) {
    double m = -INFINITY;
    if (any[u]) m = metric == ORA_ROI_MAX ? hi[u] : hi[u] - lo[u];
    if (metric_out) metric_out[u] = m;
    r[u].m = m;
    r[u].i = u;
  }
  int64_t k = 0;
  if (mode == ORA_ROI_THRESHOLD) {
    for (int64_t u = 0; u < nu; u++)
      if (r[u].m >= value) sel[k++] = u;
  } else {
    int64_t want = (int64_t)ceil(value * (double)nu);
    if (want > nu) want = nu;
    qsort(r, (size_t)nu, sizeof(ranked), by_metric_desc);
    for (int64_t j = 0; j < want; j++) sel[k++] = r[j].i;
    qsort(sel, (size_t)k, sizeof(int64_t), by_index);
  }
  *nsel = k;
  free(lo); free(hi); free(any); free(r);
  return ORA_OK;
}
