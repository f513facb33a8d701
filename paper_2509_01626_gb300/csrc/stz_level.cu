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
// (one 32-bit counter per symbol), added to the global ones at the end.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "stz_kernels.cuh"
#include "stz_prof.cuh"
#include "stz_predict.cuh"

#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

namespace stz {

constexpr int kLevelThreads = 256;
constexpr int kHistWords = kAlphabet;  // shared-memory counters per stream

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
      T pred = level_predict<K>(tile, tc.base, st, g, tc.m, a.pred);
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
    if (bm != 0u && lane == __ffs(bm) - 1) atomicAdd(&h[kRadius], (uint32_t)__popc(bm));
    if (v && !isR) atomicAdd(&h[sym], 1u);
  } else {
    if (v) {
      int sym = a.codes[s_slot[K] + local];
      T val;
      if (sym == 0) {
        if (!outlier_value(a.sub_olo, a.dense[K] != 0, s_slot[K] / geo.bvol, (int)local,
                           ll[0] * ll[1] * ll[2], a.nsub, a.opos[K], (const T*)a.oval[K],
                           a.nout[K], s_pos[K] + local, val)) {
          val = T(0);
          atomicOr(a.status, kStatCorrupt);
        }
      } else {
        T pred = level_predict<K>(tile, tc.base, st, g, tc.m, a.pred);
        val = dequantize(sym, pred, two_eb, kRadius);
      }
      ((T*)a.fine)[fidx] = val;
    }
  }
}

template <typename T>
__device__ void flush_hist(uint32_t* hist, uint32_t* gh, int level) {
  for (int w = threadIdx.x; w < 7 * kHistWords; w += blockDim.x) {
    const uint32_t v = hist[w];
    if (v) {
      const int K = w / kHistWords + 1;
      const int sid = 1 + 7 * (level - 2) + (K - 1);
      atomicAdd(gh + (int64_t)sid * kAlphabet + (w % kHistWords), v);
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
  for (int64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
    const int64_t Tb[3] = {a.tlo[0] + tt / (a.tcnt[1] * a.tcnt[2]),
                           a.tlo[1] + (tt / a.tcnt[2]) % a.tcnt[1], a.tlo[2] + tt % a.tcnt[2]};
    const int64_t c0[3] = {Tb[0] * b0, Tb[1] * b1, Tb[2] * b2};
    __syncthreads();
    if (tid < 7) {
      const int K = tid + 1;
      const StreamGeo& sg = geo.s[1 + 7 * (l - 2) + (K - 1)];
      const SlotMap& sm = a.sm[K];
      // the brick holds points of this stream that the call needs (a region
      // decode gives each stream its own brick range)
      bool ok = Tb[0] >= sm.lo[0] && Tb[0] < sm.lo[0] + sm.cnt[0] && Tb[1] >= sm.lo[1] &&
                Tb[1] < sm.lo[1] + sm.cnt[1] && Tb[2] >= sm.lo[2] && Tb[2] < sm.lo[2] + sm.cnt[2];
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
  }
  if (!DEC) {
    __syncthreads();
    flush_hist<T>(hist, a.hist, l);
  }
}

// ---------------------------------------------------------------- fast path
// Interior cells of 3D fields with the 8 x 16 x 16 brick.  Thread (ly, lx)
// walks the 8 cells of its column along z and keeps the coarse values it
// needs in a register window of 4 planes (dz = -1, 0, 1, 2) x 12 points,
// loading one new plane of 12 values per cell.  Pattern of (dy, dx) offsets:
//   0 (0,-1)  1 (0,0)  2 (0,1)  3 (0,2)  4 (-1,0)  5 (1,0)  6 (2,0)  7 (1,1)
//   8 (-1,-1) 9 (-1,2) 10 (2,-1) 11 (2,2)
// which covers every tap of Eqs. 6-8 for the 7 sub-blocks of a cell.  Only
// cells with 1 <= c <= M-3 on every axis are handled here (all stencils cubic,
// all points present); the others belong to the shell kernel below.
constexpr int kFBZ = 8, kFBY = 16, kFBX = 16;
// A tile row holds coarse x = c0x - 4 .. c0x + 19 (kFEX = 24 elements; the
// stencils read c0x - 1 .. c0x + 17), so that rows start on 16-byte
// boundaries when the coarse box does and copy as 16-byte chunks.
constexpr int kFEY = kFBY + 3, kFEX = kFBX + 8, kFEZY = kFEY * kFEX;
constexpr int kFX0 = 3;  // tile x index of coarse x = c0x - 1

template <typename T>
__device__ __forceinline__ void load_plane(T (&w)[12], const T* __restrict__ t, int b) {
  w[0] = t[b - 1];
  w[1] = t[b];
  w[2] = t[b + 1];
  w[3] = t[b + 2];
  w[4] = t[b - kFEX];
  w[5] = t[b + kFEX];
  w[6] = t[b + 2 * kFEX];
  w[7] = t[b + kFEX + 1];
  w[8] = t[b - kFEX - 1];
  w[9] = t[b - kFEX + 2];
  w[10] = t[b + 2 * kFEX - 1];
  w[11] = t[b + 2 * kFEX + 2];
}

// the 7 interior predictions of a cell (index K-1), with the operand order of
// level_predict's cubic branch
template <typename T>
__device__ __forceinline__ void cell_predict(const T (&w0)[12], const T (&w1)[12],
                                             const T (&w2)[12], const T (&w3)[12], T (&p)[7]) {
  p[0] = cubic_1d(w1[0], w1[1], w1[2], w1[3]);  // K=1 (x)
  p[1] = cubic_1d(w1[4], w1[1], w1[5], w1[6]);  // K=2 (y)
  {                                             // K=3 (y, x)
    T si = op_add(op_add(w1[1], w1[2]), op_add(w1[5], w1[7]));
    T so = op_add(op_add(w1[8], w1[9]), op_add(w1[10], w1[11]));
    p[2] = op_add(op_mul(si, T(0.25)), op_mul(op_sub(si, so), T(0.03125)));
  }
  p[3] = cubic_1d(w0[1], w1[1], w2[1], w3[1]);  // K=4 (z)
  {                                             // K=5 (z, x)
    T si = op_add(op_add(w1[1], w1[2]), op_add(w2[1], w2[2]));
    T so = op_add(op_add(w0[0], w0[3]), op_add(w3[0], w3[3]));
    p[4] = op_add(op_mul(si, T(0.25)), op_mul(op_sub(si, so), T(0.03125)));
  }
  {                                             // K=6 (z, y)
    T si = op_add(op_add(w1[1], w1[5]), op_add(w2[1], w2[5]));
    T so = op_add(op_add(w0[4], w0[6]), op_add(w3[4], w3[6]));
    p[5] = op_add(op_mul(si, T(0.25)), op_mul(op_sub(si, so), T(0.03125)));
  }
  {                                             // K=7 (z, y, x)
    T si = op_add(op_add(op_add(w1[1], w1[2]), op_add(w1[5], w1[7])),
                  op_add(op_add(w2[1], w2[2]), op_add(w2[5], w2[7])));
    T so = op_add(op_add(op_add(w0[8], w0[9]), op_add(w0[10], w0[11])),
                  op_add(op_add(w3[8], w3[9]), op_add(w3[10], w3[11])));
    p[6] = op_add(op_mul(si, T(0.125)), op_mul(op_sub(si, so), T(0.015625)));
  }
}

// ---- asynchronous copies into shared memory (cp.async, zero fill) ----
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? BYTES : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES),
               "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Per-tile stream information, computed by threads 0..6 (one per sub-block).
struct TileInfo {
  int64_t slot[8], pos[8], chunk[8];
  int l[8][3];
  int c0[3];
};

__device__ __forceinline__ void tile_info(const LevelArgs& a, int64_t tt, TileInfo& ti) {
  const Geo& geo = a.geo;
  const int l = a.level;
  // tile counts and brick coordinates fit in 32 bits (cells per axis < 2^30)
  const int t32 = (int)tt, n2 = (int)a.tcnt[2], n12 = (int)a.tcnt[1] * n2;
  const int64_t Tb[3] = {a.tlo[0] + t32 / n12, a.tlo[1] + (t32 % n12) / n2, a.tlo[2] + t32 % n2};
  const int c0[3] = {(int)Tb[0] * kFBZ, (int)Tb[1] * kFBY, (int)Tb[2] * kFBX};
  const int tid = threadIdx.x;
  if (tid < 3) ti.c0[tid] = c0[tid];
  if (tid < 7) {
    const int K = tid + 1;
    const StreamGeo& sg = geo.s[1 + 7 * (l - 2) + (K - 1)];
    const SlotMap& sm = a.sm[K];
    // the brick holds points of this stream that the call needs (a region
    // decode gives each stream its own brick range, within the stream's own)
    if (Tb[0] >= sm.lo[0] && Tb[0] < sm.lo[0] + sm.cnt[0] && Tb[1] >= sm.lo[1] &&
        Tb[1] < sm.lo[1] + sm.cnt[1] && Tb[2] >= sm.lo[2] && Tb[2] < sm.lo[2] + sm.cnt[2]) {
      const int64_t l0 = imin(kFBZ, sg.e[0] - c0[0]), l1 = imin(kFBY, sg.e[1] - c0[1]),
                    l2 = imin(kFBX, sg.e[2] - c0[2]);
      ti.l[K][0] = (int)l0;
      ti.l[K][1] = (int)l1;
      ti.l[K][2] = (int)l2;
      ti.chunk[K] = sg.chunk0 + (Tb[0] * sg.nb[1] + Tb[1]) * sg.nb[2] + Tb[2];
      ti.pos[K] = (int64_t)c0[0] * sg.e[1] * sg.e[2] + c0[1] * l0 * sg.e[2] + c0[2] * l0 * l1;
      const int64_t ord =
          ((Tb[0] - sm.lo[0]) * sm.cnt[1] + (Tb[1] - sm.lo[1])) * sm.cnt[2] + (Tb[2] - sm.lo[2]);
      ti.slot[K] = (sm.base + ord) * geo.bvol;
    } else {
      ti.l[K][0] = ti.l[K][1] = ti.l[K][2] = 0;
      ti.chunk[K] = ti.pos[K] = ti.slot[K] = 0;
    }
  }
}

// Issue the copies of tile tt's coarse grid (with halo) into `tile`.  VEC:
// the coarse box's base, row pitch and x origin are 16-byte aligned, so every
// 16-byte chunk of a tile row lies wholly inside or wholly outside the box
// (zero-filled); otherwise element by element.
template <typename T, bool VEC>
__device__ __noinline__ void tile_prefetch(const LevelArgs& a, int64_t tt, T* tile) {
  // tile counts and brick coordinates fit in 32 bits (cells per axis < 2^30)
  const int t32 = (int)tt, n2 = (int)a.tcnt[2], n12 = (int)a.tcnt[1] * n2;
  const int64_t Tb[3] = {a.tlo[0] + t32 / n12, a.tlo[1] + (t32 % n12) / n2, a.tlo[2] + t32 % n2};
  const T* coarse = (const T*)a.coarse;
  const int clo0 = (int)a.clo[0], clo1 = (int)a.clo[1], clo2 = (int)a.clo[2];
  const int ce0 = (int)(a.chi[0] - a.clo[0]), ce1 = (int)(a.chi[1] - a.clo[1]),
            ce2 = (int)(a.chi[2] - a.clo[2]);
  // local coarse coordinates of tile element (0, 0, 0)
  const int z0 = (int)Tb[0] * kFBZ - 1 - clo0, y0 = (int)Tb[1] * kFBY - 1 - clo1,
            x0 = (int)Tb[2] * kFBX - 1 - kFX0 - clo2;
  if (VEC) {
    constexpr int epc = 16 / sizeof(T);  // elements per chunk
    constexpr int cpr = kFEX / epc;      // chunks per row
    constexpr int nchunk = (kFBZ + 3) * kFEY * cpr;
    for (int q = threadIdx.x; q < nchunk; q += blockDim.x) {
      const int row = q / cpr, j = q - row * cpr;
      const int iz = row / kFEY, iy = row - iz * kFEY;
      const int cz = z0 + iz, cy = y0 + iy, cx = x0 + j * epc;
      const bool in = (unsigned)cz < (unsigned)ce0 && (unsigned)cy < (unsigned)ce1 &&
                      (unsigned)cx < (unsigned)ce2;
      const T* src = in ? coarse + ((int64_t)cz * ce1 + cy) * ce2 + cx : coarse;
      cp_async<16>(tile + row * kFEX + j * epc, src, in);
    }
  } else {
    constexpr int tvol = (kFBZ + 3) * kFEY * (kFBX + 3);
    for (int i = threadIdx.x; i < tvol; i += blockDim.x) {
      const int row = i / (kFBX + 3), ix = i - row * (kFBX + 3);
      const int iz = row / kFEY, iy = row - iz * kFEY;
      const int cz = z0 + iz, cy = y0 + iy, cx = x0 + kFX0 + ix;
      const bool in = (unsigned)cz < (unsigned)ce0 && (unsigned)cy < (unsigned)ce1 &&
                      (unsigned)cx < (unsigned)ce2;
      const T* src = in ? coarse + ((int64_t)cz * ce1 + cy) * ce2 + cx : coarse;
      cp_async<sizeof(T)>(tile + row * kFEX + kFX0 + ix, src, in);
    }
  }
  cp_async_commit();
}

// Two consecutive values as one 8- or 16-byte access.
// A tile takes fast_tile's FULL form when all 7 of its sub-block bricks are
// whole and, when decoding, all its fine points lie inside the fine box.
__device__ __forceinline__ bool tile_full(const LevelArgs& a, const TileInfo& ti, bool dec) {
  bool full = true;
#pragma unroll
  for (int K = 1; K <= 7; K++)
    full = full && ti.l[K][0] == kFBZ && ti.l[K][1] == kFBY && ti.l[K][2] == kFBX;
  if (!dec) return full;
  return full && 2 * ti.c0[0] >= a.flo[0] && 2 * (ti.c0[0] + kFBZ) <= a.fhi[0] &&
         2 * ti.c0[1] >= a.flo[1] && 2 * (ti.c0[1] + kFBY) <= a.fhi[1] &&
         2 * ti.c0[2] >= a.flo[2] && 2 * (ti.c0[2] + kFBX) <= a.fhi[2];
}

template <typename T> struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };

// One tile of the fast path.  FULL: all 7 sub-block bricks of the tile are
// whole, so a cell has the same local code index lz*256 + tid in every stream,
// and (when decoding) all the tile's fine points lie inside the fine box.
// The 7 global loads of a cell (x when compressing, codes when decoding) are
// issued one cell ahead of their use.  PAIR: the fine box and (at stride 1)
// the field have even, aligned rows, so the x-neighbour points of a cell
// (ox = 0, 1) are read and written as pairs.
// SC (decoding): the tile's codes were staged in shared memory, stream K's
// chunk at scodes + (K - 1) * kTileSlot, and are read from there.
constexpr int kTileSlot = kFBZ * kFBY * kFBX;  // symbols of a brick (one chunk)
template <typename T, bool DEC, bool FULL, bool PAIR, bool SC = false>
__device__ __forceinline__ void fast_tile(const LevelArgs& a, const T* __restrict__ tile,
                                          const TileInfo& ti, const int M[3], const QConst<T>& q,
                                          T two_eb, uint32_t* hist, int xdz, int xdy, int xdx,
                                          int fe2, int fdz, const uint16_t* scodes = nullptr) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int ly = tid >> 4, lx = tid & 15;
  const int c0z = ti.c0[0], cy = ti.c0[1] + ly, cx = ti.c0[2] + lx;
  const bool in_yx = (unsigned)(cy - 1) <= (unsigned)(M[1] - 4) &&
                     (unsigned)(cx - 1) <= (unsigned)(M[2] - 4);
  const int flo0 = (int)a.flo[0], flo1 = (int)a.flo[1], flo2 = (int)a.flo[2];
  const int fhi0 = (int)a.fhi[0], fhi1 = (int)a.fhi[1], fhi2 = (int)a.fhi[2];
  const bool fy0 = 2 * cy >= flo1 && 2 * cy < fhi1, fy1 = 2 * cy + 1 >= flo1 && 2 * cy + 1 < fhi1;
  const bool fx0 = 2 * cx >= flo2 && 2 * cx < fhi2, fx1 = 2 * cx + 1 >= flo2 && 2 * cx + 1 < fhi2;
  const int tb = (kFEY + ly + 1) * kFEX + (lx + 1 + kFX0);
  uint16_t* cp[7];
  int cstep[7];
#pragma unroll
  for (int K = 1; K <= 7; K++) {
    const int l1 = FULL ? kFBY : ti.l[K][1], l2 = FULL ? kFBX : ti.l[K][2];
    uint16_t* base = SC ? (uint16_t*)scodes + (K - 1) * kTileSlot : a.codes + ti.slot[K];
    cp[K - 1] = base + (FULL ? tid : ly * l2 + lx);
    cstep[K - 1] = l1 * l2;
  }
  const T* xp = DEC ? nullptr
                    : (const T*)a.field + (int64_t)(2 * c0z) * xdz + (int64_t)(2 * cy) * xdy +
                          (int64_t)(2 * cx) * xdx;
  T* fp = a.fine ? (T*)a.fine + ((int64_t)(2 * c0z - flo0) * (fhi1 - flo1) + (2 * cy - flo1)) *
                                    (int64_t)fe2 +
                       (2 * cx - flo2)
                 : nullptr;
  // the tile's fine points all inside the fine box (every tile of a full
  // decode): its cells need no per-point box test
  const bool tile_in = FULL || !DEC || (2 * c0z >= flo0 && 2 * (c0z + kFBZ) <= fhi0 &&
                                2 * ti.c0[1] >= flo1 && 2 * (ti.c0[1] + kFBY) <= fhi1 &&
                                2 * ti.c0[2] >= flo2 && 2 * (ti.c0[2] + kFBX) <= fhi2);
  // cell lz is "on" for sub-block K if interior (and its point inside the box)
  auto cell_on = [&](int lz, int K) -> bool {
    const int cz = c0z + lz;
    const bool interior = in_yx && (unsigned)(cz - 1) <= (unsigned)(M[0] - 4);
    if (tile_in) return interior;
    const int oz = (K >> 2) & 1, oy = (K >> 1) & 1, ox = K & 1;
    const int gz = 2 * cz + oz;
    return interior && gz >= flo0 && gz < fhi0 && (oy ? fy1 : fy0) && (ox ? fx1 : fx0);
  };
  using P2 = typename Pair2<T>::type;
  const bool xpair = PAIR && !DEC && xdx == 1;
  // the 7 field values of cell lz at x pointer p (compress; one "on" for all)
  auto load_x = [&](const T* p, bool on, T (&dst)[7]) {
    if (xpair) {
      dst[0] = on ? p[1] : T(0);  // K = 1; the even point is the coarse copy
      const P2 zero = {T(0), T(0)};
      const P2 v2 = on ? *(const P2*)(p + xdy) : zero;
      const P2 v4 = on ? *(const P2*)(p + xdz) : zero;
      const P2 v6 = on ? *(const P2*)(p + xdz + xdy) : zero;
      dst[1] = v2.x;
      dst[2] = v2.y;
      dst[3] = v4.x;
      dst[4] = v4.y;
      dst[5] = v6.x;
      dst[6] = v6.y;
    } else {
#pragma unroll
      for (int K = 1; K <= 7; K++) {
        const int oz = (K >> 2) & 1, oy = (K >> 1) & 1, ox = K & 1;
        dst[K - 1] = on ? p[oz * xdz + oy * xdy + ox * xdx] : T(0);
      }
    }
  };
  // the copied coarse value (index 0) and the 7 points of a cell, stored to
  // the fine box where on; x-neighbour pairs as one access when PAIR
  auto store8 = [&](const T (&v)[8], const bool (&o)[8]) {
#pragma unroll
    for (int pr = 0; pr < 4; pr++) {
      T* dst = fp + (pr >> 1) * fdz + (pr & 1) * fe2;
      const bool a0 = o[2 * pr], a1 = o[2 * pr + 1];
      if (PAIR && a0 && a1) {
        P2 w;
        w.x = v[2 * pr];
        w.y = v[2 * pr + 1];
        *(P2*)dst = w;
      } else {
        if (a0) dst[0] = v[2 * pr];
        if (a1) dst[1] = v[2 * pr + 1];
      }
    }
  };
  // all 8 points of a cell, unconditionally (whole tiles)
  auto store8_all = [&](const T (&v)[8]) {
#pragma unroll
    for (int pr = 0; pr < 4; pr++) {
      T* dst = fp + (pr >> 1) * fdz + (pr & 1) * fe2;
      if (PAIR) {
        P2 w;
        w.x = v[2 * pr];
        w.y = v[2 * pr + 1];
        *(P2*)dst = w;
      } else {
        dst[0] = v[2 * pr];
        dst[1] = v[2 * pr + 1];
      }
    }
  };
  // loads of cell 0
  T xv[7];
  int cv[7];
  if (!DEC) load_x(xp, cell_on(0, 1), xv);
#pragma unroll
  for (int K = 1; K <= 7; K++) {
    const bool on = cell_on(0, K);
    if (DEC) cv[K - 1] = on ? (int)*cp[K - 1] : 1;
  }
  // counts of the zero-error symbol R per stream, kept in registers over the
  // tile and added to the shared histogram once per warp at its end
  uint32_t nR[7];
#pragma unroll
  for (int K = 0; K < 7; K++) nR[K] = 0;
  T w0[12], w1[12], w2[12], w3[12];
  load_plane(w0, tile, tb - kFEZY);
  load_plane(w1, tile, tb);
  load_plane(w2, tile, tb + kFEZY);
  // whole tiles, decoding: two cells per iteration, so that half the plane
  // copies become register renames (level 3 decode 0.395 -> 0.341 ms at
  // 512^3; encoding, whose cells carry more live values, runs slower unrolled)
  static_assert(kFBZ % 2 == 0, "the unrolled z loop takes two cells at a time");
#pragma unroll((FULL && DEC) ? 2 : 1)
  for (int lz = 0; lz < kFBZ; lz++) {
    load_plane(w3, tile, tb + (lz + 2) * kFEZY);
    const int cz = c0z + lz;
    const bool interior = in_yx && (unsigned)(cz - 1) <= (unsigned)(M[0] - 4);
    const bool fz0 = 2 * cz >= flo0 && 2 * cz < fhi0;
    // issue the next cell's loads before this cell's arithmetic
    T xn[7];
    int cn[7];
    const bool more = lz + 1 < kFBZ;
    if (!DEC) load_x(xp + 2 * xdz, more && cell_on(lz + 1, 1), xn);
#pragma unroll
    for (int K = 1; K <= 7; K++) {
      const bool on = more && cell_on(lz + 1, K);
      if (DEC) cn[K - 1] = on ? (int)*(cp[K - 1] + cstep[K - 1]) : 1;
    }
    T p[7];
    cell_predict(w0, w1, w2, w3, p);
    const bool copy_on = interior && (tile_in || (fz0 && fy0 && fx0));  // the coarse point
    // in phases over the cell's 7 points: the arithmetic of all 7 first (7
    // independent chains to interleave), then the stores, then the counts
    bool on[7];
#pragma unroll
    for (int K = 1; K <= 7; K++) on[K - 1] = cell_on(lz, K);
    if (!DEC) {
      int sym[7];
      T xq[7];
#pragma unroll
      for (int K = 0; K < 7; K++) sym[K] = quantize_sel(xv[K], p[K], q, kRadius, xq[K]);
      if (FULL) {
        // a whole tile: a cell's 7 codes and 8 points are all written or
        // none (interior), under one test; outliers counted under another
        if (interior) {
          bool anyout = false;
#pragma unroll
          for (int K = 1; K <= 7; K++) {
            *cp[K - 1] = (uint16_t)sym[K - 1];
            anyout = anyout || sym[K - 1] == 0;
          }
          if (anyout) {
#pragma unroll
            for (int K = 1; K <= 7; K++)
              if (sym[K - 1] == 0) atomicAdd(&a.chunk_outliers[ti.chunk[K]], 1u);
          }
          if (fp) {
            const T v8[8] = {w1[1], xq[0], xq[1], xq[2], xq[3], xq[4], xq[5], xq[6]};
            store8_all(v8);
          }
        } else {
#pragma unroll
          for (int K = 0; K < 7; K++) sym[K] = -1;
        }
      } else {
#pragma unroll
        for (int K = 1; K <= 7; K++) {
          if (!on[K - 1]) {
            sym[K - 1] = -1;
            continue;
          }
          *cp[K - 1] = (uint16_t)sym[K - 1];
          if (sym[K - 1] == 0) atomicAdd(&a.chunk_outliers[ti.chunk[K]], 1u);
        }
        if (fp) {
          const T v8[8] = {w1[1], xq[0], xq[1], xq[2], xq[3], xq[4], xq[5], xq[6]};
          const bool o8[8] = {copy_on, on[0], on[1], on[2], on[3], on[4], on[5], on[6]};
          store8(v8, o8);
        }
      }
#pragma unroll
      for (int K = 1; K <= 7; K++) {
        const int sk = sym[K - 1];
        nR[K - 1] += sk == kRadius;
        if (sk >= 0 && sk != kRadius)
          atomicAdd(&hist[(K - 1) * kHistWords + sk], 1u);
      }
    } else {
      T val[7];
#pragma unroll
      for (int K = 0; K < 7; K++) val[K] = dequantize(cv[K], p[K], two_eb, kRadius);
      // one test for the cell's 7 codes; the rare outliers point by point
      bool anyout = false;
#pragma unroll
      for (int K = 0; K < 7; K++) anyout = anyout || (on[K] && cv[K] == 0);
      if (anyout) {
#pragma unroll
        for (int K = 1; K <= 7; K++) {
          if (on[K - 1] && cv[K - 1] == 0) {  // outlier: its value from the list
            const int64_t local =
                cp[K - 1] - (SC ? (uint16_t*)scodes + (K - 1) * kTileSlot : a.codes + ti.slot[K]);
            if (!outlier_value(a.sub_olo, a.dense[K] != 0, ti.slot[K] / a.geo.bvol, (int)local,
                               ti.l[K][0] * ti.l[K][1] * ti.l[K][2], a.nsub, a.opos[K],
                               (const T*)a.oval[K], a.nout[K], ti.pos[K] + local, val[K - 1])) {
              val[K - 1] = T(0);
              atomicOr(a.status, kStatCorrupt);
            }
          }
        }
      }
      const T v8[8] = {w1[1], val[0], val[1], val[2], val[3], val[4], val[5], val[6]};
      if (FULL) {
        // a whole tile inside the box: a cell's 8 points are all stored or
        // none (interior), under one test
        if (interior) store8_all(v8);
      } else {
        const bool o8[8] = {copy_on, on[0], on[1], on[2], on[3], on[4], on[5], on[6]};
        store8(v8, o8);
      }
    }
    if (!DEC) xp += 2 * xdz;
    if (fp) fp += 2 * fdz;
#pragma unroll
    for (int K = 0; K < 7; K++) {
      cp[K] += cstep[K];
      if (!DEC) xv[K] = xn[K];
      else cv[K] = cn[K];
    }
#pragma unroll
    for (int j = 0; j < 12; j++) {
      w0[j] = w1[j];
      w1[j] = w2[j];
      w2[j] = w3[j];
    }
  }
  if (!DEC) {
#pragma unroll
    for (int K = 0; K < 7; K++) {
      const uint32_t n = __reduce_add_sync(0xffffffffu, nR[K]);
      if (lane == 0 && n) atomicAdd(&hist[K * kHistWords + kRadius], n);
    }
  }
}

// ---- the coarse tile by one TMA tensor copy (cp.async.bulk.tensor) ----
// The tensor map describes the coarse box [clo, chi) (x fastest); a tile's
// box of (kFBZ + 3, kFEY, kFEX) elements starts at the same local coordinates
// as tile_prefetch's, outside the box it reads zeros.  One thread issues the
// copy, which completes on an mbarrier that the block then waits on.
constexpr int kTmaWaitIters = 1 << 20;  // a bound on every wait (about a second)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
// waits for the phase of parity `parity` to complete; false when the bound ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (int it = 0; it < kTmaWaitIters; it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <typename T>
__device__ __forceinline__ void tma_tile(const CUtensorMap& m, const LevelArgs& a, int64_t tt,
                                         T* tile, unsigned long long* bar) {
  const int t32 = (int)tt, n2 = (int)a.tcnt[2], n12 = (int)a.tcnt[1] * n2;
  const int Tb0 = (int)a.tlo[0] + t32 / n12, Tb1 = (int)a.tlo[1] + (t32 % n12) / n2,
            Tb2 = (int)a.tlo[2] + t32 % n2;
  const int z0 = Tb0 * kFBZ - 1 - (int)a.clo[0], y0 = Tb1 * kFBY - 1 - (int)a.clo[1],
            x0 = Tb2 * kFBX - 1 - kFX0 - (int)a.clo[2];
  constexpr uint32_t bytes = (uint32_t)((kFBZ + 3) * kFEZY * sizeof(T));
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(tile)),
      "l"((unsigned long long)(uintptr_t)&m), "r"(x0), "r"(y0), "r"(z0), "r"(smem_u32(bar))
      : "memory");
}

// Decoding f32, the interior kernel also stages a tile's codes in shared
// memory: the 7 chunks (one per stream) of the tile's brick, copied with the
// coarse tile one tile ahead, so that a cell's 7 code reads wait on shared
// memory instead of global memory (2 x 28 KiB beside the 2 x 20 KiB tiles).
template <typename T, bool DEC>
__host__ __device__ constexpr bool stage_codes() { return DEC && sizeof(T) == 4; }
constexpr size_t kTileCodeBytes = 7 * (size_t)kTileSlot * sizeof(uint16_t);

// the chunks of tile ti's 7 streams into dst (stream K at (K - 1) * kTileSlot):
// each brick's symbols, rounded up to whole 16-byte units (a slot holds a
// whole brick's worth of symbols, so the rounding stays inside it)
__device__ __forceinline__ void codes_prefetch(const LevelArgs& a, const TileInfo& ti,
                                               uint16_t* dst) {
  constexpr int kUnits = kTileSlot / 8;  // 16-byte units per chunk
  for (int q = threadIdx.x; q < 7 * kUnits; q += blockDim.x) {
    const int K = q / kUnits + 1, j = q - (K - 1) * kUnits;
    const int cnt = ti.l[K][0] * ti.l[K][1] * ti.l[K][2];
    if (j * 8 < cnt)
      cp_async<16>(dst + (K - 1) * kTileSlot + j * 8, a.codes + ti.slot[K] + j * 8, true);
  }
  cp_async_commit();
}

template <typename T, bool TMA>
__host__ __device__ constexpr size_t fast_tile_bytes() {
  return TMA ? (((size_t)(kFBZ + 3) * kFEZY * sizeof(T) + 127) & ~(size_t)127)
             : (((size_t)(kFBZ + 3) * kFEZY * sizeof(T) + 15) & ~(size_t)15);
}

template <typename T, bool DEC, bool PAIR, bool TMA>
__global__ void __launch_bounds__(kLevelThreads, 2)
    k_level_fast(const __grid_constant__ LevelArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ TileInfo s_ti[2];
  __shared__ __align__(8) unsigned long long s_bar[2];
  // TMA destinations are 128-byte aligned (the launch adds 128 bytes of slack)
  unsigned char* smem =
      TMA ? (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127) : smem_raw;
  const Geo& geo = a.geo;
  const int l = a.level;
  int64_t M64[3];
  grid_extent(geo.n, geo.L, l - 1, M64);
  const int M[3] = {(int)M64[0], (int)M64[1], (int)M64[2]};
  constexpr size_t tbytes = fast_tile_bytes<T, TMA>();
  T* tiles[2] = {(T*)smem, (T*)(smem + tbytes)};
  uint32_t* hist = (uint32_t*)(smem + 2 * tbytes);
  constexpr bool SC = stage_codes<T, DEC>() && !TMA;
  uint16_t* scodes[2] = {(uint16_t*)(smem + 2 * tbytes),
                         (uint16_t*)(smem + 2 * tbytes + kTileCodeBytes)};
  const int tid = threadIdx.x;
  if (TMA) {
    if (tid == 0) {
      mbar_init(&s_bar[0]);
      mbar_init(&s_bar[1]);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
  }
  QConst<T> q;
  if (!DEC) {
    q.load(a.dp, l, kRadius);
    for (int w = tid; w < 7 * kHistWords; w += blockDim.x) hist[w] = 0;
  }
  const T two_eb = (T)a.two_eb;
  const int64_t ntiles = a.tcnt[0] * a.tcnt[1] * a.tcnt[2];
  const int64_t s = level_stride(geo.L, l);
  const int xdz = (int)(s * geo.n[1] * geo.n[2]), xdy = (int)(s * geo.n[2]), xdx = (int)s;
  const int fe2 = (int)(a.fhi[2] - a.flo[2]);
  const int fdz = (int)((a.fhi[1] - a.flo[1]) * fe2);
  constexpr int epc = 16 / sizeof(T);
  const bool vec = ((uintptr_t)a.coarse & 15) == 0 && (a.chi[2] - a.clo[2]) % epc == 0 &&
                   a.clo[2] % epc == 0;
  auto prefetch = [&](int64_t t, int buf) {
    if (TMA) {
      if (tid == 0) tma_tile(tmap, a, t, tiles[buf], &s_bar[buf]);
    } else if (vec) {
      tile_prefetch<T, true>(a, t, tiles[buf]);
    } else {
      tile_prefetch<T, false>(a, t, tiles[buf]);
    }
  };
  uint32_t phase = 0u;  // bit b: parity of buffer b's next completion
  int64_t tt = blockIdx.x;
  int b = 0;
  if (tt < ntiles) {
    tile_info(a, tt, s_ti[0]);
    prefetch(tt, 0);
    if (SC) {
      __syncthreads();  // the tile's slots, from threads 0..6
      codes_prefetch(a, s_ti[0], scodes[0]);
    }
  }
  for (; tt < ntiles; tt += gridDim.x, b ^= 1) {
    if (TMA) {
      const bool ok = mbar_wait(&s_bar[b], (phase >> b) & 1u);
      phase ^= 1u << b;
      if (__syncthreads_or(!ok)) {
        // the copy did not complete in time: report it, give it one more
        // bounded wait so that no copy is in flight at exit, and stop
        if (tid == 0) atomicOr(a.status, kStatTimeout);
        mbar_wait(&s_bar[b], ((phase >> b) & 1u) ^ 1u);
        break;
      }
    } else {
      cp_async_wait_all();
      __syncthreads();
    }
    const int64_t nt = tt + gridDim.x;
    if (nt < ntiles) {
      tile_info(a, nt, s_ti[b ^ 1]);
      prefetch(nt, b ^ 1);
      if (SC) {
        __syncthreads();  // the next tile's slots, from threads 0..6
        codes_prefetch(a, s_ti[b ^ 1], scodes[b ^ 1]);
      }
    }
    const TileInfo& ti = s_ti[b];
    if (tile_full(a, ti, DEC))
      fast_tile<T, DEC, true, PAIR, SC>(a, tiles[b], ti, M, q, two_eb, hist, xdz, xdy, xdx, fe2,
                                        fdz, scodes[b]);
    else
      fast_tile<T, DEC, false, PAIR, SC>(a, tiles[b], ti, M, q, two_eb, hist, xdz, xdy, xdx, fe2,
                                         fdz, scodes[b]);
  }
  if (!TMA) cp_async_wait_all();
  if (!DEC) {
    __syncthreads();
    flush_hist<T>(hist, a.hist, l);
  }
}

// ---------------------------------------------------------------- shell
// Cells on the field boundary (c = 0 or c >= M-2 on some axis) of the needed
// cell range, one thread per cell, generic per-point rules read straight from
// the coarse grid.  Enumerated as three disjoint slabs: boundary z; interior z
// with boundary y; interior z and y with boundary x.
struct ShellGeo {
  int64_t lo[3], hi[3];  // needed cell range
  int64_t bv[3][3];      // boundary values per axis
  int nb[3];
  int64_t ilo[3], ihi[3];  // interior range per axis (may be empty)
  int64_t nA, nB, nC;
};

// Prediction of the sub-block-K point of a boundary cell, the rules of
// level_predict with the taps read through per-axis offsets: tap(dz, dy, dx)
// is the coarse value at cell + (dz, dy, dx), d in -1..2, clamped into the
// coarse box (a clamped tap is never one a chosen rule uses).  cub[a]: the
// cubic stencil fits along axis a at the odd point; rule[a]: the one-axis
// rule there otherwise; every value has the operation order of level_predict.
template <typename T>
struct ShellTaps {
  const T* __restrict__ cb;  // coarse value of the cell
  int oz[4], oy[4], ox[4];   // element offsets of d = -1, 0, 1, 2 per axis
  __device__ __forceinline__ T operator()(int dz, int dy, int dx) const {
    return __ldg(cb + (oz[dz + 1] + oy[dy + 1] + ox[dx + 1]));
  }
};

// One one-axis rule r over the slots w(q) of its axis (q = 0: the -1 point,
// 1: the +1 point, 2: the -3 point): the midpoint, the extrapolation or the
// copy; only the slots the rule uses are read.
// LAZY (decoding, where the kernel waits on these loads): branch on the
// rule and read only its slots; otherwise (compressing, bound by issue) read
// all three and select, without branches.
template <typename T, bool LAZY, typename W>
__device__ __forceinline__ T rule_apply(int r, const W& w) {
  const T w0 = w(0);
  if (LAZY) {
    if (r == kMid) return op_mul(op_add(w0, w(1)), T(0.5));
    if (r == kExt) return op_add(w0, op_mul(op_sub(w0, w(2)), T(0.5)));
    return w0;
  }
  const T mid = op_mul(op_add(w0, w(1)), T(0.5));
  const T ext = op_add(w0, op_mul(op_sub(w0, w(2)), T(0.5)));
  return r == kMid ? mid : (r == kExt ? ext : w0);
}

// coarse offset of slot q of a one-axis rule: 0 -> 0, 1 -> +1, 2 -> -1
__device__ __forceinline__ constexpr int sd(int q) { return q == 0 ? 0 : (q == 1 ? 1 : -1); }

template <int K, typename T, bool LAZY>
__device__ __forceinline__ T shell_predict(const ShellTaps<T>& t, const bool cub[3],
                                           const int rule[3]) {
  constexpr int oz = (K >> 2) & 1, oy = (K >> 1) & 1, ox = K & 1;
  constexpr int nodd = oz + oy + ox;
  constexpr int a0 = oz ? 0 : (oy ? 1 : 2);
  constexpr int a1 = nodd >= 2 ? (oz ? (oy ? 1 : 2) : 2) : 2;
  // tap at offsets (u along a0, v along a1, w along a2) -> (dz, dy, dx)
  auto at = [&](int u, int v, int w) -> T {
    int d[3] = {0, 0, 0};
    d[a0] += u;
    if (nodd >= 2) d[a1] += v;
    if (nodd == 3) d[2] += w;
    return t(d[0], d[1], d[2]);
  };
  bool cubic = cub[a0];
  if (nodd >= 2) cubic = cubic && cub[a1];
  if (nodd == 3) cubic = cubic && cub[2];
  if (cubic) {
    if (nodd == 1) return cubic_1d(at(-1, 0, 0), at(0, 0, 0), at(1, 0, 0), at(2, 0, 0));
    if (nodd == 2) {
      const T si = op_add(op_add(at(0, 0, 0), at(0, 1, 0)), op_add(at(1, 0, 0), at(1, 1, 0)));
      const T so = op_add(op_add(at(-1, -1, 0), at(-1, 2, 0)), op_add(at(2, -1, 0), at(2, 2, 0)));
      return op_add(op_mul(si, T(0.25)), op_mul(op_sub(si, so), T(0.03125)));
    }
    const T si = op_add(op_add(op_add(at(0, 0, 0), at(0, 0, 1)), op_add(at(0, 1, 0), at(0, 1, 1))),
                        op_add(op_add(at(1, 0, 0), at(1, 0, 1)), op_add(at(1, 1, 0), at(1, 1, 1))));
    const T so =
        op_add(op_add(op_add(at(-1, -1, -1), at(-1, -1, 2)), op_add(at(-1, 2, -1), at(-1, 2, 2))),
               op_add(op_add(at(2, -1, -1), at(2, -1, 2)), op_add(at(2, 2, -1), at(2, 2, 2))));
    return op_add(op_mul(si, T(0.125)), op_mul(op_sub(si, so), T(0.015625)));
  }
  const int r0 = rule[a0], r1 = rule[a1], r2 = rule[2];
  // the separable rules, innermost along a0: each rule reads only its slots
  if constexpr (nodd == 1) {
    return rule_apply<T, LAZY>(r0, [&](int q0) { return at(sd(q0), 0, 0); });
  } else if constexpr (nodd == 2) {
    return rule_apply<T, LAZY>(r1, [&](int q1) {
      return rule_apply<T, LAZY>(r0, [&](int q0) { return at(sd(q0), sd(q1), 0); });
    });
  } else {
    return rule_apply<T, LAZY>(r2, [&](int q2) {
      return rule_apply<T, LAZY>(r1, [&](int q1) {
        return rule_apply<T, LAZY>(r0, [&](int q0) { return at(sd(q0), sd(q1), sd(q2)); });
      });
    });
  }
}

// One cell of the boundary shell: cell i of the shell's enumeration (cv:
// i is inside it), its 7 fine points predicted with the per-axis rules and
// quantized (compress) or reconstructed (decode).
template <typename T, bool DEC>
__device__ __forceinline__ void shell_cell(const LevelArgs& a, const ShellGeo& sh, int64_t i,
                                           bool cv, const QConst<T>& q, uint32_t* hist,
                                           uint32_t (&nR)[7]) {
  const Geo& geo = a.geo;
  const int l = a.level;
  int64_t m64[3];
  grid_extent(geo.n, geo.L, l, m64);
  const int m[3] = {(int)m64[0], (int)m64[1], (int)m64[2]};
  const T two_eb = (T)a.two_eb;
  const int ce[3] = {(int)(a.chi[0] - a.clo[0]), (int)(a.chi[1] - a.clo[1]),
                     (int)(a.chi[2] - a.clo[2])};
  const int cst[3] = {ce[1] * ce[2], ce[2], 1};  // coarse box strides (elements)
  const int64_t fe1 = a.fhi[1] - a.flo[1], fe2 = a.fhi[2] - a.flo[2];
  const int64_t s = level_stride(geo.L, l);
  const int64_t xst[3] = {s * geo.n[1] * geo.n[2], s * geo.n[2], s};  // field strides
  const int64_t fst[3] = {fe1 * fe2, fe2, 1};                        // fine box strides
  int c[3] = {0, 0, 0};
  if (cv) {
    // 32-bit index arithmetic: a shell has fewer than 2^31 cells (checked at
    // launch), and 32-bit divisions cost a fraction of 64-bit ones
    const uint32_t nx = (uint32_t)(sh.hi[2] - sh.lo[2]), ny = (uint32_t)(sh.hi[1] - sh.lo[1]);
    const uint32_t nA = (uint32_t)sh.nA, nB = (uint32_t)sh.nB, ii = (uint32_t)i;
    if (ii < nA) {
      const uint32_t r = ii / nx, p = r / ny;
      c[0] = (int)sh.bv[0][p];
      c[1] = (int)sh.lo[1] + (int)(r - p * ny);
      c[2] = (int)sh.lo[2] + (int)(ii - r * nx);
    } else if (ii < nA + nB) {
      const uint32_t k = ii - nA, nb1 = (uint32_t)sh.nb[1];
      const uint32_t r = k / nx, p = r / nb1;
      c[0] = (int)sh.ilo[0] + (int)p;
      c[1] = (int)sh.bv[1][r - p * nb1];
      c[2] = (int)sh.lo[2] + (int)(k - r * nx);
    } else {
      const uint32_t k = ii - nA - nB, iyn = (uint32_t)(sh.ihi[1] - sh.ilo[1]);
      const uint32_t nb2 = (uint32_t)sh.nb[2];
      const uint32_t r = k / nb2, p = r / iyn;
      c[0] = (int)sh.ilo[0] + (int)p;
      c[1] = (int)sh.ilo[1] + (int)(r - p * iyn);
      c[2] = (int)sh.bv[2][k - r * nb2];
    }
  }
  // per axis: the odd point's existence, stencil and rule; clamped taps
  ShellTaps<T> tp;
  bool odd_in[3], cub[3];
  int rule[3];
  int64_t cbase = 0;
#pragma unroll
  for (int ax = 0; ax < 3; ax++) {
    const int lc = c[ax] - (int)a.clo[ax];
    cbase += (int64_t)lc * cst[ax];
    int* o = ax == 0 ? tp.oz : (ax == 1 ? tp.oy : tp.ox);
#pragma unroll
    for (int d = -1; d <= 2; d++) o[d + 1] = (min(max(lc + d, 0), ce[ax] - 1) - lc) * cst[ax];
    const int go = 2 * c[ax] + 1;
    odd_in[ax] = go < m[ax];
    cub[ax] = go >= 3 && go + 3 < m[ax];
    rule[ax] = go + 1 < m[ax] ? kMid : (go >= 3 ? kExt : kCopy);
  }
  tp.cb = (const T*)a.coarse + cbase;
  const int64_t g0[3] = {2 * (int64_t)c[0], 2 * (int64_t)c[1], 2 * (int64_t)c[2]};
  bool ev_box = true;  // the even point (copied coarse value) inside the fine box
#pragma unroll
  for (int ax = 0; ax < 3; ax++) ev_box = ev_box && g0[ax] >= a.flo[ax] && g0[ax] < a.fhi[ax];
  const int64_t fidx0 = ((g0[0] - a.flo[0]) * fe1 + (g0[1] - a.flo[1])) * fe2 + (g0[2] - a.flo[2]);
  if (cv && a.fine && ev_box) ((T*)a.fine)[fidx0] = tp(0, 0, 0);
  // the cell's brick and place in it (the same for the 7 sub-blocks); the
  // shell runs only beside the interior kernel, with its brick
  constexpr int kB[3] = {kFBZ, kFBY, kFBX};
  const int Bc[3] = {c[0] / kB[0], c[1] / kB[1], c[2] / kB[2]};
  const int rc[3] = {c[0] - Bc[0] * kB[0], c[1] - Bc[1] * kB[1], c[2] - Bc[2] * kB[2]};
  const int64_t xbase = DEC ? 0 : g0[0] * xst[0] + g0[1] * xst[1] + g0[2] * xst[2];
#pragma unroll
  for (int K = 1; K <= 7; K++) {
    const int o[3] = {(K >> 2) & 1, (K >> 1) & 1, K & 1};
    bool v = cv;
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
      if (o[ax]) v = v && odd_in[ax];
      if (DEC) {
        const int64_t g = g0[ax] + o[ax];
        v = v && g >= a.flo[ax] && g < a.fhi[ax];
      }
    }
    const int sid = 1 + 7 * (l - 2) + (K - 1);
    int sym = -1;
    if (v) {
      const StreamGeo& sg = geo.s[sid];
      const SlotMap& sm = a.sm[K];
      const int l0 = min(kB[0], (int)sg.e[0] - Bc[0] * kB[0]);
      const int l1 = min(kB[1], (int)sg.e[1] - Bc[1] * kB[1]);
      const int l2 = min(kB[2], (int)sg.e[2] - Bc[2] * kB[2]);
      const int local = (rc[0] * l1 + rc[1]) * l2 + rc[2];
      const int64_t ord = ((Bc[0] - sm.lo[0]) * sm.cnt[1] + (Bc[1] - sm.lo[1])) * sm.cnt[2] +
                          (Bc[2] - sm.lo[2]);
      const int64_t slot = (sm.base + ord) * (int64_t)kTileSlot + local;
      const int64_t fidx = fidx0 + o[0] * fst[0] + o[1] * fst[1] + o[2] * fst[2];
      T pred;
      switch (K) {
        case 1: pred = shell_predict<1, T, DEC>(tp, cub, rule); break;
        case 2: pred = shell_predict<2, T, DEC>(tp, cub, rule); break;
        case 3: pred = shell_predict<3, T, DEC>(tp, cub, rule); break;
        case 4: pred = shell_predict<4, T, DEC>(tp, cub, rule); break;
        case 5: pred = shell_predict<5, T, DEC>(tp, cub, rule); break;
        case 6: pred = shell_predict<6, T, DEC>(tp, cub, rule); break;
        default: pred = shell_predict<7, T, DEC>(tp, cub, rule); break;
      }
      if (!DEC) {
        const T x = __ldg((const T*)a.field + xbase + o[0] * xst[0] + o[1] * xst[1] +
                          o[2] * xst[2]);
        T xq;
        sym = quantize_sel(x, pred, q, kRadius, xq);
        a.codes[slot] = (uint16_t)sym;
        if (a.fine) ((T*)a.fine)[fidx] = xq;
        if (sym == 0) {
          const int64_t chunk = ((int64_t)Bc[0] * sg.nb[1] + Bc[1]) * sg.nb[2] + Bc[2];
          atomicAdd(&a.chunk_outliers[sg.chunk0 + chunk], 1u);
        }
      } else {
        const int sy = a.codes[slot];
        T val = dequantize(sy, pred, two_eb, kRadius);
        if (sy == 0) {
          const int64_t pos = (int64_t)Bc[0] * kB[0] * sg.e[1] * sg.e[2] +
                              (int64_t)Bc[1] * kB[1] * l0 * sg.e[2] +
                              (int64_t)Bc[2] * kB[2] * l0 * l1 + local;
          if (!outlier_value(a.sub_olo, a.dense[K] != 0, sm.base + ord, local, l0 * l1 * l2,
                             a.nsub, a.opos[K], (const T*)a.oval[K], a.nout[K], pos, val)) {
            val = T(0);
            atomicOr(a.status, kStatCorrupt);
          }
        }
        ((T*)a.fine)[fidx] = val;
      }
    }
    if (!DEC) {
      nR[K - 1] += sym == kRadius;
      if (sym >= 0 && sym != kRadius)
        atomicAdd(&hist[(K - 1) * kHistWords + sym], 1u);
    }
  }
}

// 4 blocks per SM when decoding: the loads of a cell's taps and codes are its
// latency.  Compressing, the shared histograms leave room for 3 at most, and
// the registers that 3 would cost spill more than the extra warps hide.
template <typename T, bool DEC>
__global__ void __launch_bounds__(256, DEC ? 4 : 2)
    k_level_shell(const __grid_constant__ LevelArgs a, const __grid_constant__ ShellGeo sh) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* hist = (uint32_t*)smem;
  const int l = a.level;
  const int lane = threadIdx.x & 31;
  QConst<T> q;
  if (!DEC) {
    q.load(a.dp, l, kRadius);
    for (int w = threadIdx.x; w < 7 * kHistWords; w += blockDim.x) hist[w] = 0;
    __syncthreads();
  }
  const int64_t total = sh.nA + sh.nB + sh.nC;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = cdiv(total, nth);
  uint32_t nR[7] = {0, 0, 0, 0, 0, 0, 0};  // zero-error symbols per stream, added at the end
  for (int64_t it = 0; it < iters; it++) {
    const int64_t i = it * nth + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    shell_cell<T, DEC>(a, sh, i, i < total, q, hist, nR);
  }
  if (!DEC) {
#pragma unroll
    for (int K = 0; K < 7; K++) {
      const uint32_t n = __reduce_add_sync(0xffffffffu, nR[K]);
      if (lane == 0 && n) atomicAdd(&hist[K * kHistWords + kRadius], n);
    }
    __syncthreads();
    flush_hist<T>(hist, a.hist, l);
  }
}

// ------------------------------------------------------ many decodes at once
// The batched served form: the level-l decode of many region requests in one
// launch.  args[r] (device memory) is request r's LevelArgs; its tiles
// (shell cells) are the global indices [tile0[r], tile0[r + 1]).  Every tile
// runs exactly as in k_level_fast (k_level_shell) with its own request's
// arguments, so each output is bitwise the single-request decode.
__device__ __forceinline__ int request_of(const int64_t* __restrict__ first, int n, int64_t t) {
  int lo = 0, hi = n - 1;  // the last r with first[r] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T, bool PAIR>
__global__ void __launch_bounds__(kLevelThreads, 2)
    k_level_fast_multi(const LevelArgs* __restrict__ args, const int64_t* __restrict__ tile0,
                       int n) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TileInfo s_ti[2];
  constexpr int tvol = (kFBZ + 3) * kFEZY;
  constexpr size_t tbytes = ((size_t)tvol * sizeof(T) + 15) & ~(size_t)15;
  T* tiles[2] = {(T*)smem, (T*)(smem + tbytes)};
  const int64_t ntiles = tile0[n];
  constexpr int epc = 16 / sizeof(T);
  auto prefetch = [&](const LevelArgs& a, int64_t t, T* tile) {
    const bool vec = ((uintptr_t)a.coarse & 15) == 0 && (a.chi[2] - a.clo[2]) % epc == 0 &&
                     a.clo[2] % epc == 0;
    if (vec) tile_prefetch<T, true>(a, t, tile);
    else tile_prefetch<T, false>(a, t, tile);
  };
  QConst<T> q;  // unused when decoding
  int64_t tt = blockIdx.x;
  int b = 0;
  if (tt < ntiles) {
    const int r = request_of(tile0, n, tt);
    tile_info(args[r], tt - tile0[r], s_ti[0]);
    prefetch(args[r], tt - tile0[r], tiles[0]);
  }
  for (; tt < ntiles; tt += gridDim.x, b ^= 1) {
    cp_async_wait_all();
    __syncthreads();
    const int r = request_of(tile0, n, tt);
    const LevelArgs& a = args[r];
    const int64_t nt = tt + gridDim.x;
    if (nt < ntiles) {
      const int r2 = request_of(tile0, n, nt);
      tile_info(args[r2], nt - tile0[r2], s_ti[b ^ 1]);
      prefetch(args[r2], nt - tile0[r2], tiles[b ^ 1]);
    }
    const Geo& geo = a.geo;
    int64_t M64[3];
    grid_extent(geo.n, geo.L, a.level - 1, M64);
    const int M[3] = {(int)M64[0], (int)M64[1], (int)M64[2]};
    const int64_t sl = level_stride(geo.L, a.level);
    const int xdz = (int)(sl * geo.n[1] * geo.n[2]), xdy = (int)(sl * geo.n[2]), xdx = (int)sl;
    const int fe2 = (int)(a.fhi[2] - a.flo[2]);
    const int fdz = (int)((a.fhi[1] - a.flo[1]) * fe2);
    const T two_eb = (T)a.two_eb;
    const TileInfo& ti = s_ti[b];
    if (tile_full(a, ti, true))
      fast_tile<T, true, true, PAIR>(a, tiles[b], ti, M, q, two_eb, nullptr, xdz, xdy, xdx, fe2,
                                     fdz);
    else
      fast_tile<T, true, false, PAIR>(a, tiles[b], ti, M, q, two_eb, nullptr, xdz, xdy, xdx, fe2,
                                      fdz);
  }
  cp_async_wait_all();
}

template <typename T>
__global__ void __launch_bounds__(256, 4)
    k_level_shell_multi(const LevelArgs* __restrict__ args, const ShellGeo* __restrict__ shs,
                        const int64_t* __restrict__ cell0, int n) {
  QConst<T> q;  // unused when decoding
  uint32_t nR[7] = {0, 0, 0, 0, 0, 0, 0};
  const int64_t total = cell0[n];
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = cdiv(total, nth);
  for (int64_t it = 0; it < iters; it++) {
    const int64_t i = it * nth + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool cv = i < total;
    const int r = cv ? request_of(cell0, n, i) : 0;
    shell_cell<T, true>(args[r], shs[r], cv ? i - cell0[r] : 0, cv, q, nullptr, nR);
  }
}

// ---------------------------------------------------------------- launchers
static int sm_count() { return launch_sms(); }

template <typename T, bool DEC>
static int run_level_generic(const LevelArgs& a, double bytes, cudaStream_t s) {
  int64_t M[3];
  grid_extent(a.geo.n, a.geo.L, a.level - 1, M);
  int tvol = 1;
  for (int d = 0; d < 3; d++) tvol *= M[d] > 1 ? a.geo.b[d] + 3 : 1;
  size_t smem = (((size_t)tvol * sizeof(T) + 15) & ~(size_t)15);
  if (!DEC) smem += sizeof(uint32_t) * 7 * kHistWords;
  auto kern = k_level<T, DEC>;
  if (allow_smem((const void*)kern, smem) != STZ_OK)
    return STZ_ERR_CUDA;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLevelThreads, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t ntiles = a.tcnt[0] * a.tcnt[1] * a.tcnt[2];
  if (ntiles == 0) return STZ_OK;
  int64_t grid = imin(ntiles, (int64_t)sm_count() * per_sm);
  char nm[48];
  snprintf(nm, sizeof(nm), "k_level%d_%s_%s", a.level, DEC ? "dec" : "enc",
           sizeof(T) == 4 ? "f32" : "f64");
  ProfScope ps_(nm, s, bytes);
  kern<<<(unsigned)grid, kLevelThreads, smem, s>>>(a);
  return cuda_ok(cudaGetLastError());
}

// cuTensorMapEncodeTiled, from the driver through the runtime (no link
// against the driver library); null if unavailable
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  }();
  return fn;
}

// The tensor map of the coarse box of a level launch for the interior
// kernel's tile copies.  Needs a 16-byte aligned base, rows a multiple of 16
// bytes and an x origin on a 16-byte boundary (then every tile's x
// coordinate, c0x - 4 - clo_x, is one too); false otherwise.
template <typename T>
static bool coarse_tensor_map(const LevelArgs& a, CUtensorMap* m) {
  constexpr int epc = 16 / sizeof(T);
  const int64_t ce[3] = {a.chi[0] - a.clo[0], a.chi[1] - a.clo[1], a.chi[2] - a.clo[2]};
  if (((uintptr_t)a.coarse & 15) || ce[2] % epc || a.clo[2] % epc) return false;
  for (int d = 0; d < 3; d++)
    if (ce[d] < 1 || ce[d] >= ((int64_t)1 << 31)) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dim[3] = {(cuuint64_t)ce[2], (cuuint64_t)ce[1], (cuuint64_t)ce[0]};
  const cuuint64_t stride[2] = {(cuuint64_t)(ce[2] * sizeof(T)),
                                (cuuint64_t)(ce[1] * ce[2] * sizeof(T))};
  const cuuint32_t box[3] = {(cuuint32_t)kFEX, (cuuint32_t)kFEY, (cuuint32_t)(kFBZ + 3)};
  const cuuint32_t es[3] = {1, 1, 1};
  memset(m, 0, sizeof(*m));
  return enc(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
             3, (void*)a.coarse, dim, stride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, bool DEC>
static int run_level_fast(const LevelArgs& a, const int64_t M[3], double bytes, cudaStream_t s) {
  // interior cells exist only with M >= 4 on every axis
  if (M[0] < 4 || M[1] < 4 || M[2] < 4) return STZ_OK;
  // the coarse tile by TMA when compressing (measured: level 3 encode 0.387 ->
  // 0.357 ms at 512^3); decoding keeps cp.async, as the TMA variant of the
  // decode kernel spills at 128 registers and ran slower (0.413 -> 0.499 ms)
  CUtensorMap tmap;
  const bool tma = !DEC && coarse_tensor_map<T>(a, &tmap);
  if (!tma) memset(&tmap, 0, sizeof(tmap));
  size_t smem = tma ? 2 * fast_tile_bytes<T, true>() + 128 : 2 * fast_tile_bytes<T, false>();
  if (!DEC) smem += sizeof(uint32_t) * 7 * kHistWords;
  if (stage_codes<T, DEC>()) smem += 2 * kTileCodeBytes;
  // x-neighbour pairs as one access: the fine box's rows (and, reading the
  // field at stride 1, the field's rows) even and 2-element aligned
  const uintptr_t a2 = 2 * sizeof(T);
  bool pair = true;
  if (a.fine)
    pair = pair && (uintptr_t)a.fine % a2 == 0 && (a.fhi[2] - a.flo[2]) % 2 == 0 &&
           a.flo[2] % 2 == 0;
  if (!DEC && level_stride(a.geo.L, a.level) == 1)
    pair = pair && (uintptr_t)a.field % a2 == 0 && a.geo.n[2] % 2 == 0;
  constexpr bool kTma = !DEC;  // the decode kernels are not built with TMA tiles
  auto kern = pair ? (tma ? k_level_fast<T, DEC, true, kTma> : k_level_fast<T, DEC, true, false>)
                   : (tma ? k_level_fast<T, DEC, false, kTma> : k_level_fast<T, DEC, false, false>);
  if (allow_smem((const void*)kern, smem) != STZ_OK)
    return STZ_ERR_CUDA;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLevelThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t ntiles = a.tcnt[0] * a.tcnt[1] * a.tcnt[2];
  if (ntiles == 0) return STZ_OK;
  const int64_t grid = imin(ntiles, (int64_t)sm_count() * per_sm);
  char nm[48];
  snprintf(nm, sizeof(nm), "k_level%d_%s_%s", a.level, DEC ? "dec" : "enc",
           sizeof(T) == 4 ? "f32" : "f64");
  ProfScope ps_(nm, s, bytes);
  kern<<<(unsigned)grid, kLevelThreads, smem, s>>>(a, tmap);
  return cuda_ok(cudaGetLastError());
}

// The cells of G_{l-1} whose fine points can fall in the fine box, and the
// boundary cells among them (the shell kernel's).  Returns the box's cell
// count (0: nothing to do); sh->nA + nB + nC is the shell's.
static int64_t shell_geo(const LevelArgs& a, const int64_t M[3], ShellGeo* sh) {
  memset(sh, 0, sizeof(*sh));
  int64_t cells = 1;
  for (int d = 0; d < 3; d++) {
    sh->lo[d] = imax(0, a.flo[d] / 2);
    sh->hi[d] = imin(M[d], cdiv(a.fhi[d], 2));
    if (sh->hi[d] <= sh->lo[d]) return 0;
    cells *= sh->hi[d] - sh->lo[d];
    const int64_t cand[3] = {0, M[d] - 2, M[d] - 1};
    sh->nb[d] = 0;
    for (int k = 0; k < 3; k++) {
      const int64_t v = cand[k];
      bool dup = false;
      for (int j = 0; j < sh->nb[d]; j++) dup = dup || sh->bv[d][j] == v;
      const bool boundary = !(v >= 1 && v <= M[d] - 3);
      if (!dup && boundary && v >= sh->lo[d] && v < sh->hi[d]) sh->bv[d][sh->nb[d]++] = v;
    }
    sh->ilo[d] = imax(1, sh->lo[d]);
    sh->ihi[d] = imax(sh->ilo[d], imin(M[d] - 2, sh->hi[d]));
  }
  const int64_t ny = sh->hi[1] - sh->lo[1], nx = sh->hi[2] - sh->lo[2];
  const int64_t iz = sh->ihi[0] - sh->ilo[0], iy = sh->ihi[1] - sh->ilo[1];
  sh->nA = sh->nb[0] * ny * nx;
  sh->nB = iz * sh->nb[1] * nx;
  sh->nC = iz * iy * sh->nb[2];
  return cells;
}

// shell_cell's index arithmetic is 32-bit
static bool shell_fits(const ShellGeo& sh) {
  return sh.nA + sh.nB + sh.nC < ((int64_t)1 << 31);
}

template <typename T, bool DEC>
static int run_level_shell(const LevelArgs& a, const ShellGeo& sh, double bytes, cudaStream_t s) {
  const int64_t total = sh.nA + sh.nB + sh.nC;
  if (total == 0) return STZ_OK;
  const size_t smem = DEC ? 0 : sizeof(uint32_t) * 7 * kHistWords;
  auto kern = k_level_shell<T, DEC>;
  if (smem > 48 * 1024 &&
      allow_smem((const void*)kern, smem) != STZ_OK)
    return STZ_ERR_CUDA;
  int64_t grid = imin(cdiv(total, 256), (int64_t)sm_count() * 4);
  char nm[48];
  snprintf(nm, sizeof(nm), "k_level%d_shell_%s_%s", a.level, DEC ? "dec" : "enc",
           sizeof(T) == 4 ? "f32" : "f64");
  ProfScope ps_(nm, s, bytes);
  kern<<<(unsigned)grid, 256, smem, s>>>(a, sh);
  return cuda_ok(cudaGetLastError());
}

// Algorithmic bytes of one coarse cell (its 7 new points and the copied
// coarse point): decoding reads 7 codes and the coarse value and writes 8
// fine values; compressing reads 7 field values and the coarse value, writes
// 7 codes and, below the finest level, 8 reconstructed values.
template <typename T, bool DEC>
static double cell_bytes(const LevelArgs& a) {
  const double P = (double)sizeof(T);
  return DEC ? 7 * 2 + P + 8 * P : 7 * P + P + 7 * 2 + (a.fine ? 8 * P : 0.0);
}

template <typename T, bool DEC>
static int run_level(const LevelArgs& a, cudaStream_t s) {
  int64_t M[3];
  grid_extent(a.geo.n, a.geo.L, a.level - 1, M);
  const int64_t sl = level_stride(a.geo.L, a.level);
  const int64_t fe = (a.fhi[1] - a.flo[1]) * (a.fhi[2] - a.flo[2]);
  // the fast interior and boundary kernels implement the cubic predictor;
  // the ablation predictors run in the generic kernel
  const bool fast = a.pred == kPredCubic && a.geo.b[0] == kFBZ && a.geo.b[1] == kFBY &&
                    a.geo.b[2] == kFBX &&
                    2 * kFBZ * sl * a.geo.n[1] * a.geo.n[2] < ((int64_t)1 << 31) &&
                    2 * kFBZ * fe < ((int64_t)1 << 31);
  ShellGeo sh;
  const int64_t cells = shell_geo(a, M, &sh);
  if (!shell_fits(sh)) return STZ_ERR_ARG;
  const double bpc = cell_bytes<T, DEC>(a);
  if (!fast) return run_level_generic<T, DEC>(a, (double)cells * bpc, s);
  const int64_t nshell = sh.nA + sh.nB + sh.nC;
  int rc = run_level_fast<T, DEC>(a, M, (double)(cells - nshell) * bpc, s);
  if (rc != STZ_OK) return rc;
  return run_level_shell<T, DEC>(a, sh, (double)nshell * bpc, s);
}

// ---- the batched served form: one level of many region decodes ----
bool level_multi_ok(const LevelArgs& a) {
  const int64_t sl = level_stride(a.geo.L, a.level);
  const int64_t fe = (a.fhi[1] - a.flo[1]) * (a.fhi[2] - a.flo[2]);
  return a.pred == kPredCubic && a.geo.b[0] == kFBZ && a.geo.b[1] == kFBY &&
         a.geo.b[2] == kFBX && 2 * kFBZ * sl * a.geo.n[1] * a.geo.n[2] < ((int64_t)1 << 31) &&
         2 * kFBZ * fe < ((int64_t)1 << 31);
}

static size_t al256l(size_t v) { return (v + 255) & ~(size_t)255; }

size_t level_multi_arena_bytes(int n) {
  return al256l(sizeof(LevelArgs) * (size_t)n) + al256l(sizeof(ShellGeo) * (size_t)n) +
         2 * al256l(sizeof(int64_t) * (size_t)(n + 1));
}

template <typename T>
static int run_level_multi(const LevelArgs* h, int n, uint8_t* arena, cudaStream_t s) {
  std::vector<uint8_t> buf(level_multi_arena_bytes(n), 0);
  const size_t o_sh = al256l(sizeof(LevelArgs) * (size_t)n);
  const size_t o_t0 = o_sh + al256l(sizeof(ShellGeo) * (size_t)n);
  const size_t o_c0 = o_t0 + al256l(sizeof(int64_t) * (size_t)(n + 1));
  ShellGeo* shs = (ShellGeo*)(buf.data() + o_sh);
  int64_t* tile0 = (int64_t*)(buf.data() + o_t0);
  int64_t* cell0 = (int64_t*)(buf.data() + o_c0);
  memcpy(buf.data(), h, sizeof(LevelArgs) * (size_t)n);
  bool pair = true;
  double fast_bytes = 0.0, shell_bytes = 0.0;
  tile0[0] = cell0[0] = 0;
  for (int r = 0; r < n; r++) {
    const LevelArgs& a = h[r];
    int64_t M[3];
    grid_extent(a.geo.n, a.geo.L, a.level - 1, M);
    const int64_t cells = shell_geo(a, M, &shs[r]);
    if (!shell_fits(shs[r])) return STZ_ERR_ARG;
    const int64_t nshell = shs[r].nA + shs[r].nB + shs[r].nC;
    // interior cells exist only with M >= 4 on every axis
    const bool interior = M[0] >= 4 && M[1] >= 4 && M[2] >= 4 && cells > 0;
    tile0[r + 1] = tile0[r] + (interior ? a.tcnt[0] * a.tcnt[1] * a.tcnt[2] : 0);
    cell0[r + 1] = cell0[r] + nshell;
    const uintptr_t a2 = 2 * sizeof(T);
    pair = pair && (uintptr_t)a.fine % a2 == 0 && (a.fhi[2] - a.flo[2]) % 2 == 0 &&
           a.flo[2] % 2 == 0;
    const double bpc = cell_bytes<T, true>(a);
    fast_bytes += (double)(cells - nshell) * bpc;
    shell_bytes += (double)nshell * bpc;
  }
  if (cudaMemcpyAsync(arena, buf.data(), buf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return STZ_ERR_CUDA;
  const LevelArgs* args = (const LevelArgs*)arena;
  const ShellGeo* dsh = (const ShellGeo*)(arena + o_sh);
  const int64_t* dt0 = (const int64_t*)(arena + o_t0);
  const int64_t* dc0 = (const int64_t*)(arena + o_c0);
  char nm[48];
  if (tile0[n] > 0) {
    const size_t smem = 2 * (((size_t)(kFBZ + 3) * kFEZY * sizeof(T) + 15) & ~(size_t)15);
    auto kern = pair ? k_level_fast_multi<T, true> : k_level_fast_multi<T, false>;
    if (allow_smem((const void*)kern, smem) != STZ_OK)
      return STZ_ERR_CUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLevelThreads, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = imin(tile0[n], (int64_t)sm_count() * per_sm);
    snprintf(nm, sizeof(nm), "k_level%d_dec_%s", h[0].level, sizeof(T) == 4 ? "f32" : "f64");
    ProfScope ps_(nm, s, fast_bytes);
    kern<<<(unsigned)grid, kLevelThreads, smem, s>>>(args, dt0, n);
    if (cudaGetLastError() != cudaSuccess) return STZ_ERR_CUDA;
  }
  if (cell0[n] > 0) {
    const int64_t grid = imin(cdiv(cell0[n], 256), (int64_t)sm_count() * 4);
    snprintf(nm, sizeof(nm), "k_level%d_shell_dec_%s", h[0].level,
             sizeof(T) == 4 ? "f32" : "f64");
    ProfScope ps_(nm, s, shell_bytes);
    k_level_shell_multi<T><<<(unsigned)grid, 256, 0, s>>>(args, dsh, dc0, n);
    if (cudaGetLastError() != cudaSuccess) return STZ_ERR_CUDA;
  }
  return STZ_OK;
}

int launch_level_multi(const LevelArgs* h, int n, uint8_t* arena_dev, cudaStream_t s) {
  if (n <= 0) return STZ_OK;
  for (int r = 0; r < n; r++)
    if (!level_multi_ok(h[r]) || h[r].level != h[0].level || h[r].geo.dtype != h[0].geo.dtype)
      return STZ_ERR_ARG;
  return h[0].geo.dtype == STZ_F32 ? run_level_multi<float>(h, n, arena_dev, s)
                                   : run_level_multi<double>(h, n, arena_dev, s);
}

// ---- the batched form: the level stages of many fields in one launch ----
// Work items are (field, level, tile): `gran` consecutive interior brick
// tiles of k_level_fast, or 256 boundary cells of k_level_shell, of one
// (field, level) group.  The host lists them in a schedule order (all fields'
// level 2, then all level 3, ...; or field by field) and every block claims
// the next item from one counter.  An item of level l > 2 first waits until
// every item of level l-1 of its field is done (a count per group, released
// after the block's writes, read with acquire).  Items are claimed in order
// and wait only on earlier ones, so the earliest unfinished item can always
// proceed: no residency assumption is needed.  Each item runs the code of the
// single-field kernels with its field's arguments; histogram counts of a group
// gather in shared memory and go to the group's global histograms when the
// block moves to another group, so every field's codes, grids and histograms
// are those of its own launches.
constexpr int kQueueWaitIters = 1 << 24;  // a bound on every wait (about a second)

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// waits until *done >= need; false when the bound ran out or another block
// gave up (*abort set)
__device__ bool queue_wait(const uint32_t* done, uint32_t need, const uint32_t* abort) {
  for (int it = 0; it < kQueueWaitIters; it++) {
    if (ld_acquire_u32(done) >= need) return true;
    if (*(volatile const uint32_t*)abort) return false;
    __nanosleep(64);
  }
  return false;
}

// Tile buffers of the queue kernel: two for f32 (the next tile of an item
// loads while the current one is computed), one for f64 (two would leave
// room for one block per SM beside the histograms).
template <typename T>
__host__ __device__ constexpr int queue_bufs() { return sizeof(T) == 4 ? 2 : 1; }
template <typename T>
__host__ __device__ constexpr size_t queue_smem() {
  return 128 + queue_bufs<T>() * fast_tile_bytes<T, true>() + sizeof(uint32_t) * 7 * kHistWords;
}

template <typename T>
__global__ void __launch_bounds__(kLevelThreads, 2) k_level_queue(const __grid_constant__ LevelQueue qa) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ TileInfo s_ti[2];
  __shared__ __align__(8) unsigned long long s_bar[2];
  __shared__ long long s_item;
  __shared__ int s_ok;
  constexpr int NB = queue_bufs<T>();
  constexpr size_t tbytes = fast_tile_bytes<T, true>();
  // TMA destinations are 128-byte aligned (the launch adds 128 bytes of slack)
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  T* tiles[2] = {(T*)smem, (T*)(smem + (NB - 1) * tbytes)};
  uint32_t* hist = (uint32_t*)(smem + NB * tbytes);
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&s_bar[0]);
    mbar_init(&s_bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int w = tid; w < 7 * kHistWords; w += blockDim.x) hist[w] = 0;
  __syncthreads();
  uint32_t phase = 0u;  // bit b: parity of buffer b's next completion
  int b = 0;            // the buffer of the next tile
  int cur = -1;         // the group whose counts are in the shared histograms
  bool stop = false;
  QConst<T> q;
  while (!stop) {
    if (tid == 0) s_item = (long long)atomicAdd(qa.claim, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= qa.total) break;
    int lo = 0, hi = qa.nseg - 1;  // the last segment whose first item is <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (qa.segs[mid].first <= item) lo = mid;
      else hi = mid - 1;
    }
    const QueueSeg sg = qa.segs[lo];
    const int g = sg.group;
    const LevelArgs& a = qa.args[g];
    const QueueGroup& G = qa.groups[g];
    if (g != cur) {
      if (cur >= 0) {
        flush_hist<T>(hist, qa.args[cur].hist, qa.args[cur].level);
        __syncthreads();
      }
      cur = g;
      q.load(a.dp, a.level, kRadius);
    }
    if (tid == 0) {
      int ok = 1;
      if (G.dep >= 0) ok = queue_wait(qa.done + G.dep, qa.groups[G.dep].items, qa.abort);
      if (!ok) {
        atomicOr(a.status, kStatTimeout);
        atomicExch(qa.abort, 1u);
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    const int64_t k = item - sg.first;
    if (sg.kind == 0) {
      int64_t M64[3];
      grid_extent(a.geo.n, a.geo.L, a.level - 1, M64);
      const int M[3] = {(int)M64[0], (int)M64[1], (int)M64[2]};
      const int64_t sl = level_stride(a.geo.L, a.level);
      const int xdz = (int)(sl * a.geo.n[1] * a.geo.n[2]), xdy = (int)(sl * a.geo.n[2]),
                xdx = (int)sl;
      const int fe2 = (int)(a.fhi[2] - a.flo[2]);
      const int fdz = (int)((a.fhi[1] - a.flo[1]) * fe2);
      const bool tma = G.tma != 0;
      const CUtensorMap* tm = qa.tmaps + g;
      // tile t of the item into buffer bb: its stream information, and its
      // coarse grid with halo by one TMA copy or per-thread copies
      auto issue = [&](int64_t t, int bb) {
        tile_info(a, t, s_ti[bb]);
        if (tma) {
          if (tid == 0) tma_tile<T>(*tm, a, t, tiles[bb], &s_bar[bb]);
        } else if (G.vec) {
          tile_prefetch<T, true>(a, t, tiles[bb]);
        } else {
          tile_prefetch<T, false>(a, t, tiles[bb]);
        }
      };
      const int64_t t0 = k * (int64_t)qa.gran, t1 = min(t0 + (int64_t)qa.gran, G.ntile);
      issue(t0, b);
      for (int64_t t = t0; t < t1; t++) {
        if (tma) {
          const bool ok = mbar_wait(&s_bar[b], (phase >> b) & 1u);
          phase ^= 1u << b;
          if (__syncthreads_or(!ok)) {
            // the copy did not complete in time: report it, give it one more
            // bounded wait so that no copy is in flight at exit, and stop
            if (tid == 0) {
              atomicOr(a.status, kStatTimeout);
              atomicExch(qa.abort, 1u);
            }
            mbar_wait(&s_bar[b], ((phase >> b) & 1u) ^ 1u);
            stop = true;
            break;
          }
        } else {
          cp_async_wait_all();
          __syncthreads();
        }
        const int nb = NB == 2 ? b ^ 1 : b;
        if (NB == 2 && t + 1 < t1) issue(t + 1, nb);
        const TileInfo& ti = s_ti[b];
        const bool full = tile_full(a, ti, false);
        if (G.pair) {
          if (full)
            fast_tile<T, false, true, true>(a, tiles[b], ti, M, q, T(0), hist, xdz, xdy, xdx, fe2,
                                            fdz);
          else
            fast_tile<T, false, false, true>(a, tiles[b], ti, M, q, T(0), hist, xdz, xdy, xdx,
                                             fe2, fdz);
        } else {
          if (full)
            fast_tile<T, false, true, false>(a, tiles[b], ti, M, q, T(0), hist, xdz, xdy, xdx,
                                             fe2, fdz);
          else
            fast_tile<T, false, false, false>(a, tiles[b], ti, M, q, T(0), hist, xdz, xdy, xdx,
                                              fe2, fdz);
        }
        __syncthreads();  // the buffer and its tile information are reused
        if (NB == 1 && t + 1 < t1) issue(t + 1, b);
        b = nb;
      }
      if (stop) break;
    } else {
      uint32_t nR[7] = {0, 0, 0, 0, 0, 0, 0};
      const int64_t i = k * kLevelThreads + tid;
      shell_cell<T, false>(a, qa.shs[g], i, i < G.nshell, q, hist, nR);
#pragma unroll
      for (int K = 0; K < 7; K++) {
        const uint32_t n = __reduce_add_sync(0xffffffffu, nR[K]);
        if (lane == 0 && n) atomicAdd(&hist[K * kHistWords + kRadius], n);
      }
      __syncthreads();
    }
    // the item's grid points, codes and outlier counts, then its completion
    if (tid == 0) {
      __threadfence();
      atomicAdd(qa.done + g, 1u);
    }
  }
  __syncthreads();
  if (cur >= 0) flush_hist<T>(hist, qa.args[cur].hist, qa.args[cur].level);
}

// A group of the queue: the level stage of one field, its interior tiles and
// boundary cells.  False when the group does not suit the fast kernels.
bool level_queue_ok(const LevelArgs& a) { return level_multi_ok(a) && a.geo.ndim == 3; }

static size_t queue_layout(int n, int nseg, size_t off[8]) {
  size_t o = 0;
  off[0] = o;  // LevelArgs[n]
  o += al256l(sizeof(LevelArgs) * (size_t)n);
  off[1] = o;  // ShellGeo[n]
  o += al256l(sizeof(ShellGeo) * (size_t)n);
  off[2] = o;  // QueueGroup[n]
  o += al256l(sizeof(QueueGroup) * (size_t)n);
  off[3] = o;  // QueueSeg[nseg]
  o += al256l(sizeof(QueueSeg) * (size_t)nseg);
  off[5] = o;  // CUtensorMap[n] (64-byte aligned)
  o += al256l(sizeof(CUtensorMap) * (size_t)n);
  off[4] = o;  // done[n], claim, abort: the words the host zeroes
  o += al256l(sizeof(uint32_t) * (size_t)n + 16);
  return o;
}

size_t level_queue_arena_bytes(int n) {
  size_t off[8];
  return queue_layout(n, 2 * n, off);
}

template <typename T>
static int plan_queue(const LevelArgs* h, int n, int schedule, int gran, int blocks_per_sm,
                      uint8_t* arena, LevelQueuePlan* P) {
  // the groups' order: level-major (every field's level 2, then level 3, ...)
  // or field-major (the caller's order: a field's levels ascending); a
  // group's dependency is its own field's previous level
  std::vector<int> order((size_t)n);
  for (int r = 0; r < n; r++) order[(size_t)r] = r;
  if (schedule == 0)
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return h[x].level < h[y].level; });
  size_t off[8];
  const size_t bytes = queue_layout(n, 2 * n, off);
  P->buf.assign(bytes, 0);
  memcpy(P->buf.data() + off[0], h, sizeof(LevelArgs) * (size_t)n);
  ShellGeo* shs = (ShellGeo*)(P->buf.data() + off[1]);
  QueueGroup* grp = (QueueGroup*)(P->buf.data() + off[2]);
  QueueSeg* seg = (QueueSeg*)(P->buf.data() + off[3]);
  constexpr int epc = 16 / sizeof(T);
  double fast_bytes = 0.0, shell_bytes = 0.0;
  for (int r = 0; r < n; r++) {
    const LevelArgs& a = h[r];
    int64_t M[3];
    grid_extent(a.geo.n, a.geo.L, a.level - 1, M);
    const int64_t cells = shell_geo(a, M, &shs[r]);
    if (!shell_fits(shs[r])) return STZ_ERR_ARG;
    const int64_t nshell = shs[r].nA + shs[r].nB + shs[r].nC;
    const bool interior = M[0] >= 4 && M[1] >= 4 && M[2] >= 4 && cells > 0;
    QueueGroup& G = grp[r];
    G.ntile = interior ? a.tcnt[0] * a.tcnt[1] * a.tcnt[2] : 0;
    G.nshell = nshell;
    const int64_t items = cdiv(G.ntile, gran) + cdiv(nshell, kLevelThreads);
    if (items >= ((int64_t)1 << 31)) return STZ_ERR_ARG;
    G.items = (uint32_t)items;
    G.dep = -1;  // level 2 follows level 1, which precedes the launch
    for (int p = 0; p < n; p++)
      if (p != r && h[p].codes == a.codes && h[p].level == a.level - 1) G.dep = p;
    if (a.level > 2 && G.dep < 0) return STZ_ERR_ARG;  // its level below is not queued
    const uintptr_t a2 = 2 * sizeof(T);
    bool pair = a.fine == nullptr || ((uintptr_t)a.fine % a2 == 0 &&
                                      (a.fhi[2] - a.flo[2]) % 2 == 0 && a.flo[2] % 2 == 0);
    if (level_stride(a.geo.L, a.level) == 1)
      pair = pair && (uintptr_t)a.field % a2 == 0 && a.geo.n[2] % 2 == 0;
    G.pair = pair ? 1 : 0;
    G.vec = ((uintptr_t)a.coarse & 15) == 0 && (a.chi[2] - a.clo[2]) % epc == 0 &&
            a.clo[2] % epc == 0;
    // the coarse tile by one TMA copy where the coarse box allows a tensor map
    CUtensorMap* tm = (CUtensorMap*)(P->buf.data() + off[5]) + r;
    G.tma = coarse_tensor_map<T>(a, tm) ? 1 : 0;
    if (!G.tma) memset(tm, 0, sizeof(*tm));
    const double bpc = cell_bytes<T, false>(a);
    fast_bytes += (double)(cells - nshell) * bpc;
    shell_bytes += (double)nshell * bpc;
  }
  // a group's level below must come earlier in the order
  std::vector<int> pos((size_t)n);
  for (int i = 0; i < n; i++) pos[(size_t)order[(size_t)i]] = i;
  for (int r = 0; r < n; r++)
    if (grp[r].dep >= 0 && pos[(size_t)grp[r].dep] > pos[(size_t)r]) return STZ_ERR_ARG;
  int nseg = 0;
  int64_t total = 0;
  for (int r : order) {
    const QueueGroup& G = grp[r];
    if (G.ntile > 0) {
      seg[nseg] = QueueSeg{total, r, 0};
      total += cdiv(G.ntile, gran);
      nseg++;
    }
    if (G.nshell > 0) {
      seg[nseg] = QueueSeg{total, r, 1};
      total += cdiv(G.nshell, kLevelThreads);
      nseg++;
    }
  }
  LevelQueue& qa = P->qa;
  qa.args = (const LevelArgs*)(arena + off[0]);
  qa.shs = (const ShellGeo*)(arena + off[1]);
  qa.groups = (const QueueGroup*)(arena + off[2]);
  qa.segs = (const QueueSeg*)(arena + off[3]);
  qa.tmaps = (const CUtensorMap*)(arena + off[5]);
  qa.nseg = nseg;
  qa.done = (uint32_t*)(arena + off[4]);
  qa.claim =
      (unsigned long long*)(arena + off[4] + ((sizeof(uint32_t) * (size_t)n + 7) & ~(size_t)7));
  qa.abort = (uint32_t*)(qa.claim + 1);
  qa.total = total;
  qa.gran = gran;
  P->arena = arena;
  P->counters = arena + off[4];
  P->counter_words = (int64_t)((bytes - off[4]) / 4);
  P->f64 = sizeof(T) == 8;
  P->bytes = fast_bytes + shell_bytes;
  P->smem = queue_smem<T>();
  auto kern = k_level_queue<T>;
  if (allow_smem((const void*)kern, P->smem) != STZ_OK) return STZ_ERR_CUDA;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLevelThreads, P->smem);
  if (per_sm < 1) per_sm = 1;
  if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
  P->grid = imin(total, (int64_t)sm_count() * per_sm);
  return STZ_OK;
}

int plan_level_queue(const LevelArgs* h, int n, int schedule, int gran, int blocks_per_sm,
                     uint8_t* arena_dev, LevelQueuePlan* P) {
  P->buf.clear();
  P->grid = 0;
  if (n <= 0) return STZ_OK;
  if (gran < 1 || gran > 64 || (schedule != 0 && schedule != 1) || ((uintptr_t)arena_dev & 255))
    return STZ_ERR_ARG;
  for (int r = 0; r < n; r++)
    if (!level_queue_ok(h[r]) || h[r].geo.dtype != h[0].geo.dtype) return STZ_ERR_ARG;
  return h[0].geo.dtype == STZ_F32
             ? plan_queue<float>(h, n, schedule, gran, blocks_per_sm, arena_dev, P)
             : plan_queue<double>(h, n, schedule, gran, blocks_per_sm, arena_dev, P);
}

int write_level_queue(const LevelQueuePlan& P, cudaStream_t s) {
  if (P.grid == 0) return STZ_OK;
  // from pageable memory: staged before the call returns
  return cuda_ok(cudaMemcpyAsync(P.arena, P.buf.data(), P.buf.size(), cudaMemcpyHostToDevice, s));
}

int run_level_queue(const LevelQueuePlan& P, cudaStream_t s) {
  if (P.grid == 0) return STZ_OK;
  int rc = launch_zero_words((uint32_t*)P.counters, P.counter_words, s);
  if (rc != STZ_OK) return rc;
  ProfScope ps_(P.f64 ? "k_level_queue_f64" : "k_level_queue_f32", s, P.bytes);
  if (P.f64)
    k_level_queue<double><<<(unsigned)P.grid, kLevelThreads, P.smem, s>>>(P.qa);
  else
    k_level_queue<float><<<(unsigned)P.grid, kLevelThreads, P.smem, s>>>(P.qa);
  return cuda_ok(cudaGetLastError());
}

int launch_level(const LevelArgs& a, bool decode, cudaStream_t s) {
  if (a.geo.dtype == STZ_F32)
    return decode ? run_level<float, true>(a, s) : run_level<float, false>(a, s);
  return decode ? run_level<double, true>(a, s) : run_level<double, false>(a, s);
}

}  // namespace stz
