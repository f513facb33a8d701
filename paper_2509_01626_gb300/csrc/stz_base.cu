// stz_base.cu -- level 1 (the coarsest grid, 1/64 of a 3D field) coded by an
// SZ3-style multilevel 1D interpolation coder (Sec. 3.1 opt. 3, Sec. 4.4):
// on the level-1 grid of extent m, T = smallest power of two >= max(m); the
// origin is predicted as 0; then for t = T/2 .. 1 and axis z, y, x one pass
// predicts every point whose pass-axis coordinate is an odd multiple of t,
// whose earlier coordinates are multiples of t and later ones multiples of
// 2t, from already reconstructed points.  A pass has no dependency inside
// itself, so each is one launch with a thread per point; the level-1 grid
// (8 MiB for a 512^3 field) stays resident in L2 across passes.
#include "stz_kernels.cuh"
#include "stz_prof.cuh"
#include "stz_predict.cuh"

namespace stz {

struct PassGeo {
  int64_t start[3], step[3], cnt[3];
  int64_t total;
  int axis;
  int64_t t;
  int origin;  // the single point 0, predicted as 0
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
      if (!find_outlier(a.opos, (const T*)a.oval, a.nout, ad.pos, v)) {
        v = T(0);
        atomicOr(a.status, kStatCorrupt);
      }
    } else {
      v = dequantize(sym, pred, (T)a.two_eb, kRadius);
    }
    grid[idx] = v;
  }
}

template <typename T, bool DEC>
static int run_passes(const BaseArgs& a, cudaStream_t s) {
  int64_t m[3];
  grid_extent(a.geo.n, a.geo.L, 1, m);
  int64_t mx = imax(m[0], imax(m[1], m[2]));
  int64_t T_ = 1;
  while (T_ < mx) T_ <<= 1;
  PassGeo p;
  for (int b = 0; b < 3; b++) {
    p.start[b] = 0;
    p.step[b] = 1;
    p.cnt[b] = 1;
  }
  p.total = 1;
  p.axis = 0;
  p.t = 1;
  p.origin = 1;
  const char* nm = DEC ? "k_base_pass_dec" : "k_base_pass_enc";
  {
    ProfScope ps_(nm, s);
    k_base_pass<T, DEC><<<1, 32, 0, s>>>(a, p);
  }
  p.origin = 0;
  for (int64_t t = T_ >> 1; t >= 1; t >>= 1) {
    for (int ax = 0; ax < 3; ax++) {
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
      int64_t blocks = cdiv(p.total, 256);
      ProfScope ps_(nm, s);
      k_base_pass<T, DEC><<<(unsigned)blocks, 256, 0, s>>>(a, p);
    }
  }
  return cuda_ok(cudaGetLastError());
}

int launch_base(const BaseArgs& a, bool decode, cudaStream_t s) {
  if (a.geo.dtype == STZ_F32)
    return decode ? run_passes<float, true>(a, s) : run_passes<float, false>(a, s);
  return decode ? run_passes<double, true>(a, s) : run_passes<double, false>(a, s);
}

}  // namespace stz
