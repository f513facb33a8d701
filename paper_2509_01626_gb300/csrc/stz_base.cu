// stz_base.cu -- level 1 (the coarsest grid, 1/64 of a 3D field) coded by an
// SZ3-style multilevel 1D interpolation coder (Sec. 3.1 opt. 3, Sec. 4.4):
// on the level-1 grid of extent m, T = smallest power of two >= max(m); the
// origin is predicted as 0; then for t = T/2 .. 1 and axis z, y, x one pass
// predicts every point whose pass-axis coordinate is an odd multiple of t,
// whose earlier coordinates are multiples of t and later ones multiples of
// 2t, from already reconstructed points.  A pass has no dependency inside
// itself, so each is one launch with a thread per point; the level-1 grid
// (8 MiB for a 512^3 field) stays resident in L2 across passes.
#include <cooperative_groups.h>
#include <string.h>

#include "stz_kernels.cuh"
#include "stz_prof.cuh"
#include "stz_predict.cuh"

namespace stz {

namespace cg = cooperative_groups;

struct PassGeo {
  int64_t start[3], step[3], cnt[3];
  int64_t total;
  int axis;
  int64_t t;
  int origin;      // the single point 0, predicted as 0
  FastDiv c2, c1;  // cnt[2], cnt[1]
};

// A coarse pass in units of the shared-memory subgrid (every ts-th point).
struct SubPass {
  int start[3], step[3];
  FastDiv c2, c1;  // cnt[2], cnt[1]
  int total, axis;
  int t, st, m;    // pass stride, element stride and extent along the axis, in subgrid units
  int origin;
};

template <typename T, bool DEC>
__global__ void __launch_bounds__(256) k_base_pass(BaseArgs a, PassGeo p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.total) return;
  const Geo& geo = a.geo;
  int64_t m[3];
  grid_extent(geo.n, geo.L, 1, m);
  const int64_t s1 = level_stride(geo.L, 1);
  int64_t i2 = i % p.cnt[2], r = i / p.cnt[2];
  int64_t i1 = r % p.cnt[1], i0 = r / p.cnt[1];
  int64_t g0 = p.start[0] + i0 * p.step[0];
  int64_t g1 = p.start[1] + i1 * p.step[1];
  int64_t g2 = p.start[2] + i2 * p.step[2];
  int64_t idx = (g0 * m[1] + g1) * m[2] + g2;
  T* grid = (T*)a.g1;
  T pred = T(0);
  if (!p.origin) {
    const int64_t st = p.axis == 0 ? m[1] * m[2] : (p.axis == 1 ? m[2] : 1);
    const int64_t c = p.axis == 0 ? g0 : (p.axis == 1 ? g1 : g2);
    pred = base_predict(grid, idx, st, c, p.t, m[p.axis]);
  }
  CellAddr ad = cell_addr(geo.s[0], geo.b, geo.bvol, a.sm, g0, g1, g2);
  if (!DEC) {
    QConst<T> q;
    q.load(a.dp, 1, kRadius);
    const T* f = (const T*)a.field;
    T x = f[((g0 * s1) * geo.n[1] + g1 * s1) * geo.n[2] + g2 * s1];
    T xr;
    int sym = quantize(x, pred, q, kRadius, xr);
    grid[idx] = xr;
    a.codes[ad.slot] = (uint16_t)sym;
    if (sym == 0) atomicAdd(&a.chunk_outliers[geo.s[0].chunk0 + ad.chunk], 1u);
  } else {
    int sym = a.codes[ad.slot];
    T v;
    if (sym == 0) {
      if (!outlier_value(a.sub_olo, a.dense != 0, ad.sidx, ad.local, ad.cnt, a.nsub, a.opos,
                         (const T*)a.oval, a.nout, ad.pos, v)) {
        v = T(0);
        atomicOr(a.status, kStatCorrupt);
      }
    } else {
      v = dequantize(sym, pred, (T)a.two_eb, kRadius);
    }
    grid[idx] = v;
  }
}

// All passes in one cooperative launch.  The first `nsmall` passes (the coarse
// strides, a few thousand points) run in block 0 alone with block barriers;
// the rest are spread over the grid with a grid-wide barrier between passes.
// Level-1 values written by other blocks are read with L2-only loads (__ldcg),
// never through a possibly stale L1 line.
constexpr int kMaxPasses = 64;
constexpr int64_t kLocalPoints = 32768;  // fine-pass points kept in the single block
#ifndef STZ_BASE_SUBGRID_KB
#define STZ_BASE_SUBGRID_KB 16
#endif
constexpr int64_t kBaseSubgridBytes = (int64_t)STZ_BASE_SUBGRID_KB * 1024;
struct PassList {
  PassGeo p[kMaxPasses];
  SubPass sp[kMaxPasses];  // the first nsmall passes in subgrid units
  int npass, nsmall;
  int nlocal;              // passes run by the single-block kernel (nsmall <= nlocal <= npass)
  int ts;                  // stride of the subgrid held in shared memory by the coarse phase
  int sm[3];               // subgrid extent
  FastDiv fsm2, fsm1;      // sm[2], sm[1]
  FastDiv bd[3];           // brick extents of stream 0
};

template <typename T>
__device__ __forceinline__ T base_predict_cg(const T* g1, int64_t idx, int64_t st, int64_t c,
                                             int64_t t, int64_t m) {
  const int64_t d = t * st;
  T vm1 = __ldcg(g1 + idx - d);
  bool p1 = c + t < m, m3 = c - 3 * t >= 0, p3 = c + 3 * t < m;
  if (m3 && p3)
    return cubic_1d(__ldcg(g1 + idx - 3 * d), vm1, __ldcg(g1 + idx + d), __ldcg(g1 + idx + 3 * d));
  if (p1) return op_mul(op_add(vm1, __ldcg(g1 + idx + d)), T(0.5));
  if (m3) return op_add(vm1, op_mul(op_sub(vm1, __ldcg(g1 + idx - 3 * d)), T(0.5)));
  return vm1;
}

// Address of level-1 grid point g in stream 0 (32-bit arithmetic: the level-1
// grid has fewer than 2^31 points).
struct Addr32 {
  int64_t slot, pos, sidx;
  int chunk, local, cnt;
};
__device__ __forceinline__ Addr32 addr0(const StreamGeo& sg, const int32_t b[3],
                                        const FastDiv bd[3], int bvol, const SlotMap& sm, int c0,
                                        int c1, int c2) {
  const int B0 = (int)fdiv(c0, bd[0]), B1 = (int)fdiv(c1, bd[1]), B2 = (int)fdiv(c2, bd[2]);
  const int e0 = (int)sg.e[0], e1 = (int)sg.e[1], e2 = (int)sg.e[2];
  const int l0 = min(b[0], e0 - B0 * b[0]), l1 = min(b[1], e1 - B1 * b[1]),
            l2 = min(b[2], e2 - B2 * b[2]);
  const int local = ((c0 - B0 * b[0]) * l1 + (c1 - B1 * b[1])) * l2 + (c2 - B2 * b[2]);
  Addr32 r;
  r.pos = (int64_t)B0 * b[0] * e1 * e2 + (int64_t)B1 * b[1] * l0 * e2 +
          (int64_t)B2 * b[2] * l0 * l1 + local;
  r.chunk = (B0 * (int)sg.nb[1] + B1) * (int)sg.nb[2] + B2;
  const int ord = ((B0 - (int)sm.lo[0]) * (int)sm.cnt[1] + (B1 - (int)sm.lo[1])) * (int)sm.cnt[2] +
                  (B2 - (int)sm.lo[2]);
  r.sidx = sm.base + ord;
  r.slot = r.sidx * (int64_t)bvol + local;
  r.local = local;
  r.cnt = l0 * l1 * l2;
  return r;
}

// The value of an outlier of stream 0 at address ad (a rare path, kept out of
// line so that it costs the passes no registers); a missing entry marks the
// container corrupt and gives 0.
template <typename T>
__device__ __noinline__ T base_outlier(const BaseArgs& a, const Addr32& ad) {
  T v;
  if (!outlier_value(a.sub_olo, a.dense != 0, ad.sidx, ad.local, ad.cnt, a.nsub, a.opos,
                     (const T*)a.oval, a.nout, ad.pos, v)) {
    v = T(0);
    atomicOr(a.status, kStatCorrupt);
  }
  return v;
}

template <typename T, bool DEC>
__device__ __forceinline__ void base_point(const BaseArgs& a, const PassGeo& p,
                                           const FastDiv bd[3], unsigned i, const int64_t m[3],
                                           int64_t s1, const QConst<T>& q) {
  const Geo& geo = a.geo;
  const unsigned r = fdiv(i, p.c2), i0 = fdiv(r, p.c1);
  const int i2 = (int)(i - r * p.c2.d), i1 = (int)(r - i0 * p.c1.d);
  const int g0 = (int)p.start[0] + i0 * (int)p.step[0];
  const int g1 = (int)p.start[1] + i1 * (int)p.step[1];
  const int g2 = (int)p.start[2] + i2 * (int)p.step[2];
  const int64_t idx = ((int64_t)g0 * m[1] + g1) * m[2] + g2;
  T* grid = (T*)a.g1;
  T pred = T(0);
  if (!p.origin) {
    const int64_t st = p.axis == 0 ? m[1] * m[2] : (p.axis == 1 ? m[2] : 1);
    const int64_t c = p.axis == 0 ? g0 : (p.axis == 1 ? g1 : g2);
    pred = base_predict_cg(grid, idx, st, c, p.t, m[p.axis]);
  }
  const Addr32 ad = addr0(geo.s[0], geo.b, bd, (int)geo.bvol, a.sm, g0, g1, g2);
  if (!DEC) {
    const T* f = (const T*)a.field;
    T x = f[(((int64_t)g0 * s1) * geo.n[1] + (int64_t)g1 * s1) * geo.n[2] + (int64_t)g2 * s1];
    T xr;
    int sym = quantize(x, pred, q, kRadius, xr);
    __stcg(grid + idx, xr);
    a.codes[ad.slot] = (uint16_t)sym;
    if (sym == 0) atomicAdd(&a.chunk_outliers[geo.s[0].chunk0 + ad.chunk], 1u);
  } else {
    int sym = a.codes[ad.slot];
    const T v = sym == 0 ? base_outlier<T>(a, ad) : dequantize(sym, pred, (T)a.two_eb, kRadius);
    __stcg(grid + idx, v);
  }
}

// Coarse phase in shared memory: every pass with stride t >= ts touches only
// points of the stride-ts subgrid (extent sm = ceil(m / ts)), which one block
// keeps in shared memory together with the points' codes; those passes run
// there with block barriers in 32-bit subgrid coordinates, and the subgrid
// (and, compressing, its codes) is then written out.  The remaining passes
// (t < ts) are spread over the grid with a grid barrier before each.
template <typename T, bool DEC>
__device__ void coarse_phase(const BaseArgs& a, const PassList& pl, T* sg, uint16_t* sc,
                             const int64_t m[3], int64_t s1, const QConst<T>& q) {
  const Geo& geo = a.geo;
  const int ts = pl.ts, sm1 = pl.sm[1], sm2 = pl.sm[2];
  const int nsg = pl.sm[0] * sm1 * sm2;
  // gather the subgrid's inputs, kGather independent loads in flight per
  // thread: the field values (compress) or the codes (decode); an outlier's
  // value is looked up here, off the passes' critical path
  constexpr int kGather = 8;
  for (int i0 = threadIdx.x; i0 < nsg; i0 += kGather * blockDim.x) {
    int64_t src[kGather];
#pragma unroll
    for (int u = 0; u < kGather; u++) {
      const int i = i0 + u * blockDim.x;
      const int ic = i < nsg ? i : 0;
      const unsigned r = fdiv((unsigned)ic, pl.fsm2), z = fdiv(r, pl.fsm1);
      const int x = ic - (int)r * sm2, y = (int)r - (int)z * sm1;
      const int g0 = (int)z * ts, g1 = y * ts, g2 = x * ts;
      if (!DEC) {
        src[u] = (((int64_t)g0 * s1) * geo.n[1] + (int64_t)g1 * s1) * geo.n[2] + (int64_t)g2 * s1;
      } else {
        src[u] = addr0(geo.s[0], geo.b, pl.bd, (int)geo.bvol, a.sm, g0, g1, g2).slot;
      }
    }
    if (!DEC) {
      T v[kGather];
#pragma unroll
      for (int u = 0; u < kGather; u++) v[u] = ((const T*)a.field)[src[u]];
#pragma unroll
      for (int u = 0; u < kGather; u++)
        if (i0 + u * (int)blockDim.x < nsg) sg[i0 + u * blockDim.x] = v[u];
    } else {
      uint16_t c[kGather];
#pragma unroll
      for (int u = 0; u < kGather; u++) c[u] = a.codes[src[u]];
#pragma unroll
      for (int u = 0; u < kGather; u++) {
        const int i = i0 + u * blockDim.x;
        if (i >= nsg) continue;
        sc[i] = c[u];
        if (c[u] == 0) {
          // the point's stream address again, on this rare path only (keeping
          // it for every gathered point costs registers the block has not got)
          const unsigned r = fdiv((unsigned)i, pl.fsm2), z = fdiv(r, pl.fsm1);
          const int x = i - (int)r * sm2, y = (int)r - (int)z * sm1;
          const Addr32 ad =
              addr0(geo.s[0], geo.b, pl.bd, (int)geo.bvol, a.sm, (int)z * ts, y * ts, x * ts);
          sg[i] = base_outlier<T>(a, ad);
        }
      }
    }
  }
  __syncthreads();
  for (int k = 0; k < pl.nsmall; k++) {
    const SubPass& p = pl.sp[k];
    for (int i = threadIdx.x; i < p.total; i += blockDim.x) {
      const unsigned r = fdiv((unsigned)i, p.c2), i0 = fdiv(r, p.c1);
      const int i2 = i - (int)(r * p.c2.d), i1 = (int)(r - i0 * p.c1.d);
      const int z = p.start[0] + (int)i0 * p.step[0], y = p.start[1] + i1 * p.step[1],
                x = p.start[2] + i2 * p.step[2];
      const int si = (z * sm1 + y) * sm2 + x;
      T pred = T(0);
      if (!p.origin) {
        const int c = p.axis == 0 ? z : (p.axis == 1 ? y : x);
        pred = base_predict<T, int>(sg, si, p.st, c, p.t, p.m);
      }
      if (!DEC) {
        T xr;
        const int sym = quantize(sg[si], pred, q, kRadius, xr);  // sg[si] is still the input
        sg[si] = xr;
        sc[si] = (uint16_t)sym;
      } else {
        const int sym = sc[si];
        if (sym != 0) sg[si] = dequantize(sym, pred, (T)a.two_eb, kRadius);
        // an outlier's value was placed by the gather
      }
    }
    __syncthreads();
  }
  // write the subgrid to the level-1 grid, and compressing its codes
  T* grid = (T*)a.g1;
  for (int i = threadIdx.x; i < nsg; i += blockDim.x) {
    const unsigned r = fdiv((unsigned)i, pl.fsm2), z = fdiv(r, pl.fsm1);
    const int x = i - (int)r * sm2, y = (int)r - (int)z * sm1;
    const int g0 = (int)z * ts, g1 = y * ts, g2 = x * ts;
    __stcg(grid + ((int64_t)g0 * m[1] + g1) * m[2] + g2, sg[i]);
    if (!DEC) {
      const Addr32 ad = addr0(geo.s[0], geo.b, pl.bd, (int)geo.bvol, a.sm, g0, g1, g2);
      const uint16_t sym = sc[i];
      a.codes[ad.slot] = sym;
      if (sym == 0) atomicAdd(&a.chunk_outliers[geo.s[0].chunk0 + ad.chunk], 1u);
    }
  }
}

template <typename T, bool DEC>
__global__ void __launch_bounds__(1024) k_base_coarse(const __grid_constant__ BaseArgs a,
                                                      const __grid_constant__ PassList pl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int64_t m[3];
  grid_extent(a.geo.n, a.geo.L, 1, m);
  const int64_t s1 = level_stride(a.geo.L, 1);
  QConst<T> q;
  if (!DEC) q.load(a.dp, 1, kRadius);
  const int nsg = pl.sm[0] * pl.sm[1] * pl.sm[2];
  T* sg = (T*)smem_raw;
  uint16_t* sc = (uint16_t*)(smem_raw + sizeof(T) * nsg);
  if (pl.nsmall > 0) coarse_phase<T, DEC>(a, pl, sg, sc, m, s1, q);
  // small remaining passes (a region's dependencies) in this block: global
  // writes are visible to the block after the barrier
  for (int k = pl.nsmall; k < pl.nlocal; k++) {
    __syncthreads();
    const PassGeo& p = pl.p[k];
    for (int i = threadIdx.x; i < (int)p.total; i += blockDim.x)
      base_point<T, DEC>(a, p, pl.bd, (unsigned)i, m, s1, q);
  }
}

template <typename T, bool DEC>
__global__ void __launch_bounds__(256) k_base_coop(const __grid_constant__ BaseArgs a,
                                                   const __grid_constant__ PassList pl) {
  cg::grid_group grid = cg::this_grid();
  int64_t m[3];
  grid_extent(a.geo.n, a.geo.L, 1, m);
  const int64_t s1 = level_stride(a.geo.L, 1);
  QConst<T> q;
  if (!DEC) q.load(a.dp, 1, kRadius);
  for (int k = pl.nlocal; k < pl.npass; k++) {
    if (k > pl.nlocal) grid.sync();
    const PassGeo& p = pl.p[k];
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.total; i += nth)
      base_point<T, DEC>(a, p, pl.bd, (unsigned)i, m, s1, q);
  }
}


template <typename T, bool DEC>
static int run_coop(const BaseArgs& a, cudaStream_t s, bool allow_coop = true) {
  int64_t m[3];
  grid_extent(a.geo.n, a.geo.L, 1, m);
  if (m[0] * m[1] * m[2] >= ((int64_t)1 << 31)) return STZ_ERR_ARG;  // 32-bit level-1 indexing
  int64_t mx = imax(m[0], imax(m[1], m[2]));
  int64_t T_ = 1;
  while (T_ < mx) T_ <<= 1;
  PassList pl;
  memset(&pl, 0, sizeof(pl));
  {
    PassGeo& p = pl.p[pl.npass++];
    for (int b = 0; b < 3; b++) {
      p.start[b] = 0;
      p.step[b] = 1;
      p.cnt[b] = 1;
    }
    p.total = 1;
    p.origin = 1;
    p.t = 1;
  }
  int64_t biggest = 1;
  for (int64_t t = T_ >> 1; t >= 1; t >>= 1) {
    for (int ax = 0; ax < 3; ax++) {
      PassGeo p;
      memset(&p, 0, sizeof(p));
      p.axis = ax;
      p.t = t;
      p.total = 1;
      for (int b = 0; b < 3; b++) {
        if (b == ax) {
          p.start[b] = t;
          p.step[b] = 2 * t;
          p.cnt[b] = m[b] > t ? (m[b] - t - 1) / (2 * t) + 1 : 0;
        } else if (b < ax) {
          p.start[b] = 0;
          p.step[b] = t;
          p.cnt[b] = cdiv(m[b], t);
        } else {
          p.start[b] = 0;
          p.step[b] = 2 * t;
          p.cnt[b] = cdiv(m[b], 2 * t);
        }
        p.total *= p.cnt[b];
      }
      if (p.total == 0) continue;
      if (pl.npass >= kMaxPasses) return STZ_ERR_ARG;
      pl.p[pl.npass++] = p;
      biggest = imax(biggest, p.total);
    }
  }
  // a region decode runs only what the box [rlo, rhi) depends on: walking the
  // passes backwards, pass k is cut to the current box, which then grows by
  // 3t along the pass axis (the reach of its predictor) for the passes before
  if (a.region) {
    int64_t lo[3], hi[3];
    for (int b = 0; b < 3; b++) {
      lo[b] = imax(0, a.rlo[b]);
      hi[b] = imin(m[b], a.rhi[b]);
    }
    for (int k = pl.npass - 1; k >= 0; k--) {
      PassGeo& p = pl.p[k];
      p.total = 1;
      for (int b = 0; b < 3; b++) {
        const int64_t i0 = lo[b] > p.start[b] ? cdiv(lo[b] - p.start[b], p.step[b]) : 0;
        const int64_t i1 =
            hi[b] > p.start[b] ? imin(p.cnt[b], cdiv(hi[b] - p.start[b], p.step[b])) : 0;
        p.start[b] += i0 * p.step[b];
        p.cnt[b] = imax(0, i1 - i0);
        p.total *= p.cnt[b];
      }
      if (!p.origin) {
        lo[p.axis] = imax(0, lo[p.axis] - 3 * p.t);
        hi[p.axis] = imin(m[p.axis], hi[p.axis] + 3 * p.t);
      }
    }
    int n = 0;
    biggest = 1;
    for (int k = 0; k < pl.npass; k++)
      if (pl.p[k].total > 0) {
        pl.p[n++] = pl.p[k];
        biggest = imax(biggest, pl.p[k].total);
      }
    pl.npass = n;
    if (n == 0) return STZ_OK;
  }
  // coarse phase: the passes with t >= ts, ts the smallest power of two whose
  // subgrid fits in kBaseSubgridBytes of shared memory
  const int64_t cap = kBaseSubgridBytes / (int64_t)sizeof(T);
  int64_t ts = 1;
  while (cdiv(m[0], ts) * cdiv(m[1], ts) * cdiv(m[2], ts) > cap) ts <<= 1;
  pl.ts = (int)ts;
  pl.nsmall = 0;
  while (pl.nsmall < pl.npass && (pl.p[pl.nsmall].origin || pl.p[pl.nsmall].t >= ts)) pl.nsmall++;
  for (int k = 0; k < pl.npass; k++) {
    pl.p[k].c2 = make_fastdiv((uint32_t)pl.p[k].cnt[2]);
    pl.p[k].c1 = make_fastdiv((uint32_t)pl.p[k].cnt[1]);
  }
  for (int b = 0; b < 3; b++) {
    pl.sm[b] = (int)cdiv(m[b], ts);
    pl.bd[b] = make_fastdiv((uint32_t)a.geo.b[b]);
  }
  pl.fsm2 = make_fastdiv((uint32_t)pl.sm[2]);
  pl.fsm1 = make_fastdiv((uint32_t)pl.sm[1]);
  for (int k = 0; k < pl.nsmall; k++) {
    const PassGeo& p = pl.p[k];
    SubPass& q = pl.sp[k];
    for (int b = 0; b < 3; b++) {
      q.start[b] = (int)(p.start[b] / ts);
      q.step[b] = (int)(p.step[b] / ts);  // 0 only for the origin, whose counts are 1
    }
    q.c2 = p.c2;
    q.c1 = p.c1;
    q.total = (int)p.total;
    q.axis = p.axis;
    q.t = (int)(p.t / ts);
    q.st = p.axis == 0 ? pl.sm[1] * pl.sm[2] : (p.axis == 1 ? pl.sm[2] : 1);
    q.m = pl.sm[p.axis];
    q.origin = p.origin;
  }
  // the passes after the coarse phase stay in the single block while they are
  // a few rounds of its threads each (a grid barrier costs more)
  pl.nlocal = pl.nsmall;
  {
    int64_t rest = 0;
    for (int k = pl.nsmall; k < pl.npass; k++) rest += pl.p[k].total;
    if (rest <= kLocalPoints) pl.nlocal = pl.npass;
  }
  // a region whose passes are small altogether runs them all on the level-1
  // grid in the single block: no subgrid is gathered and written back
  if (a.region) {
    int64_t all = 0;
    for (int k = 0; k < pl.npass; k++) all += pl.p[k].total;
    if (all <= kLocalPoints) {
      pl.nsmall = 0;
      pl.nlocal = pl.npass;
    }
  }
  const size_t nsg =
      pl.nsmall > 0 ? (size_t)pl.sm[0] * pl.sm[1] * pl.sm[2] : 0;  // no coarse phase: none
  const size_t smem = (sizeof(T) + sizeof(uint16_t)) * nsg;
  {
    auto ck = k_base_coarse<T, DEC>;
    if (allow_smem((const void*)ck, smem) != STZ_OK)
      return STZ_ERR_CUDA;
    ProfScope ps_(DEC ? "k_base_coarse_dec" : "k_base_coarse_enc", s);
    ck<<<1, 1024, smem, s>>>(a, pl);
    if (cudaGetLastError() != cudaSuccess) return STZ_ERR_CUDA;
  }
  if (pl.nlocal == pl.npass) return STZ_OK;
  biggest = 1;
  for (int k = pl.nlocal; k < pl.npass; k++) biggest = imax(biggest, pl.p[k].total);
  auto kern = k_base_coop<T, DEC>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
  if (per_sm < 1) return STZ_ERR_CUDA;
  int64_t blocks = imin((int64_t)sms * imin(per_sm, 4), imax(1, cdiv(biggest, 256)));
  void* args[] = {(void*)&a, (void*)&pl};
  cudaError_t e = cudaErrorNotSupported;
  if (allow_coop) {
    ProfScope ps_(DEC ? "k_base_coop_dec" : "k_base_coop_enc", s);
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)blocks), dim3(256), args, 0,
                                    s);
  }
  if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
    cudaGetLastError();  // clear, then one launch per remaining pass
    for (int k = pl.nlocal; k < pl.npass; k++) {
      const PassGeo& p = pl.p[k];
      ProfScope ps_(DEC ? "k_base_pass_dec" : "k_base_pass_enc", s);
      k_base_pass<T, DEC><<<(unsigned)cdiv(p.total, 256), 256, 0, s>>>(a, p);
    }
    return cuda_ok(cudaGetLastError());
  }
  return cuda_ok(e);
}

int launch_base(const BaseArgs& a, bool decode, cudaStream_t s) {
  if (a.geo.dtype == STZ_F32)
    return decode ? run_coop<float, true>(a, s) : run_coop<float, false>(a, s);
  return decode ? run_coop<double, true>(a, s) : run_coop<double, false>(a, s);
}

int launch_base_nocoop(const BaseArgs& a, bool decode, cudaStream_t s) {
  if (a.geo.dtype == STZ_F32)
    return decode ? run_coop<float, true>(a, s, false) : run_coop<float, false>(a, s, false);
  return decode ? run_coop<double, true>(a, s, false) : run_coop<double, false>(a, s, false);
}

}  // namespace stz
