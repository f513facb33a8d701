// stz_common.cuh -- shared definitions of the STZ CUDA library (sm_103a).
//
// Geometry of the hierarchical partition (Sec. 3.1 Fig. 3, Sec. 3.2 three
// levels): level l of L has stride s_l = 2^(L-l); G_l is the grid of points
// whose coordinates are multiples of s_l.  Level 1 is G_1.  Level l >= 2 is
// G_l minus G_{l-1}, split into 7 sub-blocks by which G_l coordinates are odd
// (k = 4*(z odd) + 2*(y odd) + (x odd)); in 2D (nz = 1) the sub-blocks with
// an odd z are empty.  Sub-block k holds the points 2c + o_k of G_l, with c
// its "cell" (a point of G_{l-1}).
//
// Each stream (level 1, then level l sub-block k at index 1 + 7(l-2) + k-1)
// is stored brick-major: bricks of (bz, by, bx) cells in raster order, each
// brick one independently decodable chunk.  On the device a chunk's symbols
// live in a "slot" of bvol = bz*by*bx entries of the code buffer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "stz.h"

namespace stz {

constexpr int kMaxLevels = 6;
constexpr int kMaxStreams = 1 + 7 * (kMaxLevels - 1);
constexpr int kLevels = 3;              // L used by stz_compress
constexpr int kRadius = 1024;           // quantization radius R
constexpr int kAlphabet = 2 * kRadius;  // symbols 0 (outlier) .. 2R-1
constexpr int kMaxCodeLen = 12;         // Huffman length limit = decode table index bits
constexpr int kNSub = 8;                // sub-chunks per chunk (independent decode chains)
constexpr int kDecThreads = 256;        // threads per block of the chunk decoder
constexpr int kLutSize = 1 << kMaxCodeLen;
constexpr int kHeaderBytes = 256;
constexpr int kDirEntryBytes = 48;
constexpr int kBrick3D[3] = {8, 16, 16};
constexpr int kBrick2D[3] = {1, 32, 64};

// status bits written by kernels into DevParams::status
constexpr uint32_t kStatCorrupt = 1u;
constexpr uint32_t kStatCapacity = 2u;
constexpr uint32_t kStatTimeout = 4u;  // a bounded wait for an asynchronous copy ran out

#define STZ_HD __host__ __device__ __forceinline__

// Division of n in [0, 2^32) by a divisor d >= 1 fixed before the launch: a
// multiply-high, an add and a shift (the round-up method of Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994:
// with l = ceil(log2 d) and mul = floor(2^32 (2^l - d) / d) + 1,
// n / d = (mulhi(mul, n) + n) >> l exactly).
struct FastDiv {
  uint32_t d, mul, sh;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.sh = 0;
  while ((1ull << f.sh) < d) f.sh++;
  f.mul = (uint32_t)(((1ull << 32) * ((1ull << f.sh) - d)) / d + 1);
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return (uint32_t)(((unsigned long long)__umulhi(n, f.mul) + n) >> f.sh);
}

STZ_HD int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
STZ_HD int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
STZ_HD int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

struct StreamGeo {
  int64_t e[3];   // sub-block extent in cells
  int64_t nb[3];  // bricks per axis
  int64_t nsym;
  int64_t nchunks;
  int64_t chunk0;  // index of its first chunk among all streams' chunks
  int32_t o[3];    // odd offsets of the sub-block (0 for level 1)
  int32_t level;
};

struct Geo {
  int64_t n[3];  // field dims (z, y, x)
  int32_t b[3];  // brick
  int32_t L, ndim, dtype, nstreams;
  int64_t bvol;          // cells per brick = symbols per chunk slot
  int64_t total_chunks;  // over all streams
  StreamGeo s[kMaxStreams];
};

STZ_HD int64_t level_stride(int L, int l) { return (int64_t)1 << (L - l); }

STZ_HD void grid_extent(const int64_t n[3], int L, int l, int64_t m[3]) {
  int64_t s = level_stride(L, l);
  for (int a = 0; a < 3; a++) m[a] = cdiv(n[a], s);
}

// Which bricks of a stream a kernel touches, and where their slots start in
// the code buffer: ordinal of brick B = ((B0-lo0)*cnt1 + (B1-lo1))*cnt2 +
// (B2-lo2); slot of chunk = base + ordinal.
struct SlotMap {
  int64_t lo[3];
  int64_t cnt[3];
  int64_t base;
};

// Position of cell c in the stream (brick-major order), its local index in
// the brick and its slot entry in the code buffer.
struct CellAddr {
  int64_t pos;    // stream position (outlier indices refer to it)
  int64_t slot;   // code buffer entry
  int64_t chunk;  // chunk index within the stream
  int64_t sidx;   // chunk slot
  int local, cnt; // index within the chunk, symbols of the chunk
};

STZ_HD CellAddr cell_addr(const StreamGeo& sg, const int32_t b[3], int64_t bvol,
                          const SlotMap& sm, int64_t c0, int64_t c1, int64_t c2) {
  // cells per axis are below 2^30: 32-bit divisions
  int64_t B0 = (int32_t)c0 / b[0], B1 = (int32_t)c1 / b[1], B2 = (int32_t)c2 / b[2];
  int64_t l0 = imin(b[0], sg.e[0] - B0 * b[0]);
  int64_t l1 = imin(b[1], sg.e[1] - B1 * b[1]);
  int64_t l2 = imin(b[2], sg.e[2] - B2 * b[2]);
  int64_t local = ((c0 - B0 * b[0]) * l1 + (c1 - B1 * b[1])) * l2 + (c2 - B2 * b[2]);
  CellAddr r;
  r.pos = B0 * b[0] * sg.e[1] * sg.e[2] + B1 * b[1] * l0 * sg.e[2] + B2 * b[2] * l0 * l1 + local;
  r.chunk = (B0 * sg.nb[1] + B1) * sg.nb[2] + B2;
  int64_t ord = ((B0 - sm.lo[0]) * sm.cnt[1] + (B1 - sm.lo[1])) * sm.cnt[2] + (B2 - sm.lo[2]);
  r.sidx = sm.base + ord;
  r.slot = r.sidx * bvol + local;
  r.local = (int)local;
  r.cnt = (int)(l0 * l1 * l2);
  return r;
}

// Chunk j of a stream: brick coordinates, clipped extent, first position.
STZ_HD void chunk_brick(const StreamGeo& sg, const int32_t b[3], int64_t j, int64_t B[3],
                        int64_t l[3], int64_t* start) {
  B[0] = j / (sg.nb[1] * sg.nb[2]);
  B[1] = (j / sg.nb[2]) % sg.nb[1];
  B[2] = j % sg.nb[2];
  for (int a = 0; a < 3; a++) l[a] = imin(b[a], sg.e[a] - B[a] * b[a]);
  *start = B[0] * b[0] * sg.e[1] * sg.e[2] + B[1] * b[1] * l[0] * sg.e[2] + B[2] * b[2] * l[0] * l[1];
}

// Error-bound constants, computed on the device from the value range (or the
// absolute bound) so that no host round trip is needed.
struct DevParams {
  double eb;          // as given
  double eb_abs;      // finest-level bound
  double vmin, vmax;  // range of finite values (relative mode), else 0
  double eb_level[kMaxLevels + 1];  // index 1..L
  double two_eb_d[kMaxLevels + 1];  // 2 eb_l rounded to the field precision, as double
  float inv2eb_f[kMaxLevels + 1], two_eb_f[kMaxLevels + 1], ebc_f[kMaxLevels + 1];
  double inv2eb_d[kMaxLevels + 1], two_eb_dd[kMaxLevels + 1], ebc_d[kMaxLevels + 1];
  unsigned long long range_lo, range_hi;  // order-preserving keys of min / max
  double eb_ratio;    // eb_l = eb_{l+1} / eb_ratio (Sec. 3.1 opt. 5)
  uint32_t status;
  uint32_t pred;      // predictor of levels 2..L (kPred*)
};

// Predictor of levels 2..L (the ablation of Sec. 3.1): opt. 4 cubic Eqs. 6-8
// (the method), opt. 2 multi-linear Eqs. 3-5, opt. 1 direct Eq. 1.
constexpr int kPredCubic = 0, kPredLinear = 1, kPredDirect = 2;

// ---- correctly rounded single operations (no contraction into FMA) ----
__device__ __forceinline__ float op_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float op_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float op_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double op_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double op_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double op_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float op_abs(float a) { return fabsf(a); }
__device__ __forceinline__ double op_abs(double a) { return fabs(a); }
// Quantization integers (|v| < 2^22) to and from floating point with plain
// additions instead of conversion instructions: in [2^23, 2^24) the ulp of a
// float is 1, so adding 1.5 * 2^23 rounds v to an integer (to nearest, ties
// to even, as rint does) that sits in the low bits of the sum's encoding, and
// subtracting it back is exact.  The same holds for doubles with 1.5 * 2^52.
constexpr float kMagicF = 12582912.0f;              // 1.5 * 2^23
constexpr int kMagicFBits = 0x4B400000;             // its encoding
constexpr double kMagicD = 6755399441055744.0;      // 1.5 * 2^52
constexpr long long kMagicDBits = 0x4338000000000000LL;
// rint(v) as a value, and as an integer in q
__device__ __forceinline__ float round_q(float v, int& q) {
  const float t = __fadd_rn(v, kMagicF);
  q = __float_as_int(t) - kMagicFBits;
  return __fsub_rn(t, kMagicF);
}
__device__ __forceinline__ double round_q(double v, int& q) {
  const double t = __dadd_rn(v, kMagicD);
  q = (int)(__double_as_longlong(t) - kMagicDBits);
  return __dsub_rn(t, kMagicD);
}
// The integer add is opaque to the compiler: otherwise it folds the pair back
// into an int-to-float conversion instruction, which this GPU issues on its
// narrow FP64 pipe (the float decode kernels then spend half that pipe's
// issue rate on conversions).  The result is the same value either way.
__device__ __forceinline__ float from_int(int v, float) {
  int b;
  asm("add.s32 %0, %1, %2;" : "=r"(b) : "r"(v), "n"(kMagicFBits));
  return __fsub_rn(__int_as_float(b), kMagicF);
}
__device__ __forceinline__ double from_int(int v, double) {
  return __dsub_rn(__longlong_as_double(kMagicDBits + v), kMagicD);
}

template <typename T> struct QConst;
template <> struct QConst<float> {
  float inv2eb, two_eb, ebc, rlim;
  __device__ __forceinline__ void load(const DevParams* p, int l, int R) {
    inv2eb = p->inv2eb_f[l];
    two_eb = p->two_eb_f[l];
    ebc = p->ebc_f[l];
    rlim = (float)R - 0.5f;
  }
};
template <> struct QConst<double> {
  double inv2eb, two_eb, ebc, rlim;
  __device__ __forceinline__ void load(const DevParams* p, int l, int R) {
    inv2eb = p->inv2eb_d[l];
    two_eb = p->two_eb_dd[l];
    ebc = p->ebc_d[l];
    rlim = (double)R - 0.5;
  }
};

// Linear-scale quantization: q = round-half-even(d / 2eb) when |q| < R - 0.5,
// reconstruction pred + q * 2eb accepted when within ebc of x (ebc is below
// eb_l by at least one ulp, so the rounded test implies the exact bound).
// Returns the symbol q + R, or 0 (outlier, reconstruction = x).
template <typename T>
__device__ __forceinline__ int quantize(T x, T pred, const QConst<T>& q, int R, T& xr) {
  T d = op_sub(x, pred);
  T qf = op_mul(d, q.inv2eb);
  if (!(op_abs(qf) < q.rlim)) {
    xr = x;
    return 0;
  }
  int qi;
  const T qr = round_q(qf, qi);
  T rec = op_add(pred, op_mul(qr, q.two_eb));
  T e = op_sub(rec, x);
  if (!(op_abs(e) <= q.ebc)) {
    xr = x;
    return 0;
  }
  xr = rec;
  return qi + R;
}

// The same quantizer without branches (identical results): both tests are
// evaluated and the outcome selected at the end.
template <typename T>
__device__ __forceinline__ int quantize_sel(T x, T pred, const QConst<T>& q, int R, T& xr) {
  const T d = op_sub(x, pred);
  const T qf = op_mul(d, q.inv2eb);
  const bool in_range = op_abs(qf) < q.rlim;
  int qi;
  T qr = round_q(qf, qi);
  qi = in_range ? qi : 0;
  qr = in_range ? qr : T(0);
  const T rec = op_add(pred, op_mul(qr, q.two_eb));
  const bool ok = in_range && (op_abs(op_sub(rec, x)) <= q.ebc);
  xr = ok ? rec : x;
  return ok ? qi + R : 0;
}

template <typename T>
__device__ __forceinline__ T dequantize(int sym, T pred, T two_eb, int R) {
  return op_add(pred, op_mul(from_int(sym - R, T()), two_eb));
}

// Outliers when decoding.  A stream's outliers are listed by ascending
// stream position, and a chunk's positions are contiguous (brick-major
// order), so the outliers of each sub-chunk are a contiguous part of the
// list.  For streams dense in outliers (dense_outliers(): at least one per
// 2048 symbols) the chunk decoder records, per decoded chunk slot, where each
// of its sub-chunks starts in that list (sub_olo[slot * (kNSub + 1) + u],
// u = 0 .. nsub; entry nsub is the chunk's end), and an outlier's value is
// found by a binary search over its own sub-chunk's few entries; for sparse
// streams the search runs over the whole (short) list.  A symbol 0 whose
// position is not listed means a corrupt container.
inline bool dense_outliers(uint64_t nout, uint64_t nsym) { return nout > 0 && nout * 2048 >= nsym; }

template <typename T>
__device__ __forceinline__ bool outlier_value(const uint32_t* __restrict__ sub_olo, bool dense,
                                              int64_t sidx, int local, int cnt, int nsub,
                                              const uint32_t* opos, const T* oval, int64_t nout,
                                              int64_t pos, T& out) {
  if (nout <= 0 || cnt <= 0) return false;
  int64_t lo = 0, hi = nout;
  if (dense) {
    const int per = (cnt + nsub - 1) / nsub;
    const uint32_t* r = sub_olo + sidx * (kNSub + 1) + local / per;
    lo = imin((int64_t)r[0], nout);
    hi = imin((int64_t)r[1], nout);
  }
  const int64_t end = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)opos[mid] < pos) lo = mid + 1;
    else hi = mid;
  }
  if (lo < end && (int64_t)opos[lo] == pos) {
    out = oval[lo];
    return true;
  }
  return false;
}

// Per-stream decode-side pointers into a container on the device.
template <typename T>
struct StreamIn {
  const uint32_t* opos;  // outlier positions
  const T* oval;         // outlier values
  int64_t nout;
};

// ---- host helpers (stz_api.cu) ----
void make_geo(const int64_t n[3], int ndim, int dtype, int L, const int b[3], Geo* g);

// Symbols of all streams of a field.
inline int64_t total_symbols(const Geo& g) {
  int64_t n = 0;
  for (int s = 0; s < g.nstreams; s++) n += g.s[s].nsym;
  return n;
}
inline int cuda_ok(cudaError_t e) { return e == cudaSuccess ? STZ_OK : STZ_ERR_CUDA; }

}  // namespace stz
