// stz_level.cu -- levels 2..L: multi-dimensional cubic interpolation of each
// finer level from the reconstructed coarser grid (Sec. 3.1 opt. 2-5, Eqs.
// 6-8; Sec. 3.2), quantized with the level's bound (compress) or
// reconstructed from the decoded codes (decompress).
//
// Work unit = one brick of cells (bz x by x bx points of G_{l-1}), which is
// exactly one chunk of each of the 7 sub-block streams of the level, so the
// codes of a tile are 7 contiguous slot ranges.  The coarse grid of the tile
// plus a halo of 1 below and 2 above (the cubic stencils' reach) is staged in
// shared memory; each thread owns cells and computes their up-to-7 fine
// points, reading x (compress) and writing G_l (next level's coarse grid, or
// the output) with coalesced accesses along x.  Persistent grid: blocks loop
// over tiles; compress accumulates per-stream histograms in shared memory
// (16-bit counters packed in pairs, flushed before they can overflow).
#include "stz_kernels.cuh"
#include "stz_prof.cuh"
#include "stz_predict.cuh"

#include <stdio.h>

namespace stz {

constexpr int kLevelThreads = 256;
constexpr int kHistWords = kAlphabet / 2;  // per stream, 2 counters per word
constexpr int kFlushTiles = 31;            // 31 * 2048 < 65536

struct TileCtx {
  int64_t m[3];   // G_l extent
  int64_t c[3];   // cell
  int base;       // tile index of the cell
  int lz, ly, lx; // cell within the brick
  bool cv;        // cell exists
};

template <int K, typename T, bool DEC>
__device__ __forceinline__ void do_point(const LevelArgs& a, const TileCtx& tc, const T* tile,
                                         const int st[3], const QConst<T>& q, T two_eb,
                                         uint32_t* hist, const int64_t* s_slot,
                                         const int64_t* s_pos, const int64_t* s_chunk,
                                         const int (*s_l)[3], int lane) {
  constexpr int oz = (K >> 2) & 1, oy = (K >> 1) & 1, ox = K & 1;
  const int* ll = s_l[K];
  bool v = tc.cv && tc.lz < ll[0] && tc.ly < ll[1] && tc.lx < ll[2];
  const int64_t g[3] = {2 * tc.c[0] + oz, 2 * tc.c[1] + oy, 2 * tc.c[2] + ox};
  const bool in_fine = g[0] >= a.flo[0] && g[0] < a.fhi[0] && g[1] >= a.flo[1] &&
                       g[1] < a.fhi[1] && g[2] >= a.flo[2] && g[2] < a.fhi[2];
  if (DEC) v = v && in_fine;
  const int64_t local = ((int64_t)tc.lz * ll[1] + tc.ly) * ll[2] + tc.lx;
  const Geo& geo = a.geo;
  int64_t fidx = 0;
  if (a.fine) {
    const int64_t fe1 = a.fhi[1] - a.flo[1], fe2 = a.fhi[2] - a.flo[2];
    fidx = ((g[0] - a.flo[0]) * fe1 + (g[1] - a.flo[1])) * fe2 + (g[2] - a.flo[2]);
  }
  if (!DEC) {
    int sym = 0;
    if (v) {
      T pred = level_predict<K>(tile, tc.base, st, g, tc.m);
      const int64_t s = level_stride(geo.L, a.level);
      const T* f = (const T*)a.field;
      T x = f[((g[0] * s) * geo.n[1] + g[1] * s) * geo.n[2] + g[2] * s];
      T xr;
      sym = quantize(x, pred, q, kRadius, xr);
      a.codes[s_slot[K] + local] = (uint16_t)sym;
      if (a.fine) ((T*)a.fine)[fidx] = xr;
      if (sym == 0) atomicAdd(&a.chunk_outliers[s_chunk[K]], 1u);
    }
    const bool isR = v && sym == kRadius;
    const unsigned bm = __ballot_sync(0xffffffffu, isR);
    uint32_t* h = hist + (K - 1) * kHistWords;
    if (bm != 0u && lane == __ffs(bm) - 1) atomicAdd(&h[kRadius >> 1], (uint32_t)__popc(bm));
    if (v && !isR) atomicAdd(&h[sym >> 1], 1u << ((sym & 1) * 16));
  } else {
    if (v) {
      int sym = a.codes[s_slot[K] + local];
      T val;
      if (sym == 0) {
        if (!find_outlier(a.opos[K], (const T*)a.oval[K], a.nout[K], s_pos[K] + local, val)) {
          val = T(0);
          atomicOr(a.status, kStatCorrupt);
        }
      } else {
        T pred = level_predict<K>(tile, tc.base, st, g, tc.m);
        val = dequantize(sym, pred, two_eb, kRadius);
      }
      ((T*)a.fine)[fidx] = val;
    }
  }
}

template <typename T>
__device__ void flush_hist(uint32_t* hist, uint32_t* gh, int level) {
  for (int w = threadIdx.x; w < 7 * kHistWords; w += blockDim.x) {
    uint32_t v = hist[w];
    if (v) {
      int K = w / kHistWords + 1;
      int sym = (w % kHistWords) * 2;
      int sid = 1 + 7 * (level - 2) + (K - 1);
      uint32_t* dst = gh + (int64_t)sid * kAlphabet + sym;
      if (v & 0xFFFFu) atomicAdd(dst, v & 0xFFFFu);
      if (v >> 16) atomicAdd(dst + 1, v >> 16);
      hist[w] = 0;
    }
  }
}

template <typename T, bool DEC>
__global__ void __launch_bounds__(kLevelThreads) k_level(const __grid_constant__ LevelArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int64_t s_slot[8], s_pos[8], s_chunk[8];
  __shared__ int s_l[8][3];
  const Geo& geo = a.geo;
  const int l = a.level;
  TileCtx tc;
  int64_t M[3];
  grid_extent(geo.n, geo.L, l, tc.m);
  grid_extent(geo.n, geo.L, l - 1, M);
  const int b0 = geo.b[0], b1 = geo.b[1], b2 = geo.b[2];
  int ext[3], org[3];
  for (int d = 0; d < 3; d++) {
    ext[d] = M[d] > 1 ? geo.b[d] + 3 : 1;
    org[d] = M[d] > 1 ? -1 : 0;
  }
  const int tvol = ext[0] * ext[1] * ext[2];
  T* tile = (T*)smem;
  uint32_t* hist = (uint32_t*)(smem + (((size_t)tvol * sizeof(T) + 15) & ~(size_t)15));
  const int st[3] = {ext[1] * ext[2], ext[2], 1};
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31;
  QConst<T> q;
  if (!DEC) {
    q.load(a.dp, l, kRadius);
    for (int w = tid; w < 7 * kHistWords; w += nth) hist[w] = 0;
  }
  const T two_eb = (T)a.two_eb;
  const T* coarse = (const T*)a.coarse;
  const int64_t ce1 = a.chi[1] - a.clo[1], ce2 = a.chi[2] - a.clo[2];
  const int64_t ntiles = a.tcnt[0] * a.tcnt[1] * a.tcnt[2];
  const int bvol = b0 * b1 * b2;
  const int iters = (bvol + nth - 1) / nth;
  int since_flush = 0;
  for (int64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
    const int64_t Tb[3] = {a.tlo[0] + tt / (a.tcnt[1] * a.tcnt[2]),
                           a.tlo[1] + (tt / a.tcnt[2]) % a.tcnt[1], a.tlo[2] + tt % a.tcnt[2]};
    const int64_t c0[3] = {Tb[0] * b0, Tb[1] * b1, Tb[2] * b2};
    __syncthreads();
    if (tid < 7) {
      const int K = tid + 1;
      const StreamGeo& sg = geo.s[1 + 7 * (l - 2) + (K - 1)];
      const SlotMap& sm = a.sm[K];
      bool ok = Tb[0] < sg.nb[0] && Tb[1] < sg.nb[1] && Tb[2] < sg.nb[2];
      if (ok) {
        int64_t l0 = imin(b0, sg.e[0] - c0[0]), l1 = imin(b1, sg.e[1] - c0[1]),
                l2 = imin(b2, sg.e[2] - c0[2]);
        s_l[K][0] = (int)l0;
        s_l[K][1] = (int)l1;
        s_l[K][2] = (int)l2;
        s_chunk[K] = sg.chunk0 + (Tb[0] * sg.nb[1] + Tb[1]) * sg.nb[2] + Tb[2];
        s_pos[K] = c0[0] * sg.e[1] * sg.e[2] + c0[1] * l0 * sg.e[2] + c0[2] * l0 * l1;
        int64_t ord = ((Tb[0] - sm.lo[0]) * sm.cnt[1] + (Tb[1] - sm.lo[1])) * sm.cnt[2] +
                      (Tb[2] - sm.lo[2]);
        s_slot[K] = (sm.base + ord) * geo.bvol;
      } else {
        s_l[K][0] = s_l[K][1] = s_l[K][2] = 0;
        s_chunk[K] = s_pos[K] = s_slot[K] = 0;
      }
    }
    for (int i = tid; i < tvol; i += nth) {
      const int iz = i / (ext[1] * ext[2]), iy = (i / ext[2]) % ext[1], ix = i % ext[2];
      const int64_t cz = c0[0] + org[0] + iz, cy = c0[1] + org[1] + iy, cx = c0[2] + org[2] + ix;
      T v = T(0);
      if (cz >= a.clo[0] && cz < a.chi[0] && cy >= a.clo[1] && cy < a.chi[1] && cx >= a.clo[2] &&
          cx < a.chi[2])
        v = coarse[((cz - a.clo[0]) * ce1 + (cy - a.clo[1])) * ce2 + (cx - a.clo[2])];
      tile[i] = v;
    }
    __syncthreads();
    for (int it = 0; it < iters; it++) {
      const int ci = tid + it * nth;
      tc.lz = ci / (b1 * b2);
      tc.ly = (ci / b2) % b1;
      tc.lx = ci % b2;
      tc.c[0] = c0[0] + tc.lz;
      tc.c[1] = c0[1] + tc.ly;
      tc.c[2] = c0[2] + tc.lx;
      tc.cv = ci < bvol && tc.c[0] < M[0] && tc.c[1] < M[1] && tc.c[2] < M[2];
      tc.base = ((tc.lz - org[0]) * ext[1] + (tc.ly - org[1])) * ext[2] + (tc.lx - org[2]);
      if (tc.cv && a.fine) {
        const int64_t g0 = 2 * tc.c[0], g1 = 2 * tc.c[1], g2 = 2 * tc.c[2];
        if (g0 >= a.flo[0] && g0 < a.fhi[0] && g1 >= a.flo[1] && g1 < a.fhi[1] &&
            g2 >= a.flo[2] && g2 < a.fhi[2]) {
          const int64_t fe1 = a.fhi[1] - a.flo[1], fe2 = a.fhi[2] - a.flo[2];
          ((T*)a.fine)[((g0 - a.flo[0]) * fe1 + (g1 - a.flo[1])) * fe2 + (g2 - a.flo[2])] =
              tile[tc.base];
        }
      }
      do_point<1, T, DEC>(a, tc, tile, st, q, two_eb, hist, s_slot, s_pos, s_chunk, s_l, lane);
      do_point<2, T, DEC>(a, tc, tile, st, q, two_eb, hist, s_slot, s_pos, s_chunk, s_l, lane);
      do_point<3, T, DEC>(a, tc, tile, st, q, two_eb, hist, s_slot, s_pos, s_chunk, s_l, lane);
      do_point<4, T, DEC>(a, tc, tile, st, q, two_eb, hist, s_slot, s_pos, s_chunk, s_l, lane);
      do_point<5, T, DEC>(a, tc, tile, st, q, two_eb, hist, s_slot, s_pos, s_chunk, s_l, lane);
      do_point<6, T, DEC>(a, tc, tile, st, q, two_eb, hist, s_slot, s_pos, s_chunk, s_l, lane);
      do_point<7, T, DEC>(a, tc, tile, st, q, two_eb, hist, s_slot, s_pos, s_chunk, s_l, lane);
    }
    if (!DEC && ++since_flush == kFlushTiles) {
      __syncthreads();
      flush_hist<T>(hist, a.hist, l);
      since_flush = 0;
    }
  }
  if (!DEC) {
    __syncthreads();
    flush_hist<T>(hist, a.hist, l);
  }
}

template <typename T, bool DEC>
static int run_level(const LevelArgs& a, cudaStream_t s) {
  int64_t M[3];
  grid_extent(a.geo.n, a.geo.L, a.level - 1, M);
  int tvol = 1;
  for (int d = 0; d < 3; d++) tvol *= M[d] > 1 ? a.geo.b[d] + 3 : 1;
  size_t smem = (((size_t)tvol * sizeof(T) + 15) & ~(size_t)15);
  if (!DEC) smem += sizeof(uint32_t) * 7 * kHistWords;
  auto kern = k_level<T, DEC>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return STZ_ERR_CUDA;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLevelThreads, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t ntiles = a.tcnt[0] * a.tcnt[1] * a.tcnt[2];
  if (ntiles == 0) return STZ_OK;
  int64_t grid = imin(ntiles, (int64_t)sms * per_sm);
  char nm[48];
  snprintf(nm, sizeof(nm), "k_level%d_%s_%s", a.level, DEC ? "dec" : "enc",
           sizeof(T) == 4 ? "f32" : "f64");
  ProfScope ps_(nm, s);
  kern<<<(unsigned)grid, kLevelThreads, smem, s>>>(a);
  return cuda_ok(cudaGetLastError());
}

int launch_level(const LevelArgs& a, bool decode, cudaStream_t s) {
  if (a.geo.dtype == STZ_F32)
    return decode ? run_level<float, true>(a, s) : run_level<float, false>(a, s);
  return decode ? run_level<double, true>(a, s) : run_level<double, false>(a, s);
}

}  // namespace stz
