// stz_roi.cu -- the ROI selection module of Sec. 3.3 (last paragraph): the
// value range or the maximum of each slice or block of a field, then the
// units whose metric reaches a threshold, or the top x% of them, as input to
// random-access decompression (stz_decompress_region).  Typically run on a
// progressive (coarse) decode of a field: the coarse grid is 1/64 of the
// points and locates the regions worth decoding at full resolution.
//
// Unit u = ((z / bz) * nby + y / by) * nbx + x / bx over blocks of
// (bz, by, bx) points clipped at the field's edge; a slice along an axis is
// the block that spans the other two axes.
//
//   k_roi_reduce: one point per thread in raster order (coalesced loads);
//     each value becomes an order-preserving 64-bit key of its double value
//     (non-finite values contribute nothing; -0 orders below +0); a warp
//     reduces runs of lanes that share a unit (units are contiguous along
//     x) with a segmented shuffle reduction, and each run's first lane
//     updates the unit's minimum and maximum keys with 64-bit atomics.
//   k_roi_select: one block.  Per unit the metric (max, or max - min as one
//     correctly rounded double subtraction; -inf without a finite value);
//     threshold: metric >= value; top k = ceil(fraction * nunits): the k-th
//     largest metric key is found by an 8-pass radix select (8 bits a pass,
//     from the top), then the units above it and the lowest-index units equal
//     to it are kept.  The selection is written in ascending unit order by
//     block-wide prefix sums.
#include "stz_kernels.cuh"
#include "stz_prof.cuh"

#include <math.h>

namespace stz {

constexpr int kRoiSelectThreads = 1024;

__device__ __forceinline__ unsigned long long okey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double okey_val(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}

struct RoiGeo {
  int64_t n[3];
  int64_t b[3];
  int64_t nb[3];
  int64_t npts;
  int64_t nunits;
};

template <typename T>
__global__ void __launch_bounds__(256) k_roi_reduce(const T* __restrict__ x, RoiGeo g,
                                                    unsigned long long* __restrict__ kmin,
                                                    unsigned long long* __restrict__ kmax) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // every lane runs the same number of iterations (full-warp shuffles)
  const int64_t base0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  for (int64_t base = base0; base < g.npts; base += stride) {
    const int64_t i = base + lane;
    const bool in = i < g.npts;
    unsigned long long lo = ~0ull, hi = 0ull;
    long long u = -1 - lane;  // distinct for lanes past the end
    if (in) {
      const int64_t xx = i % g.n[2], r = i / g.n[2];
      const int64_t yy = r % g.n[1], zz = r / g.n[1];
      u = (long long)(((zz / g.b[0]) * g.nb[1] + yy / g.b[1]) * g.nb[2] + xx / g.b[2]);
      const double v = (double)x[i];
      if (isfinite(v)) lo = hi = okey(v);
    }
    // segmented suffix reduction: lane l combines lanes l .. 31 of its run
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const long long u2 = __shfl_down_sync(0xffffffffu, u, off);
      const unsigned long long lo2 = __shfl_down_sync(0xffffffffu, lo, off);
      const unsigned long long hi2 = __shfl_down_sync(0xffffffffu, hi, off);
      if (lane + off < 32 && u2 == u) {
        lo = lo2 < lo ? lo2 : lo;
        hi = hi2 > hi ? hi2 : hi;
      }
    }
    const long long up = __shfl_up_sync(0xffffffffu, u, 1);
    const bool head = in && (lane == 0 || up != u);
    if (head && hi != 0ull) {
      atomicMin(&kmin[u], lo);
      atomicMax(&kmax[u], hi);
    }
  }
}

__global__ void k_roi_init(unsigned long long* __restrict__ kmin, unsigned long long* __restrict__ kmax,
                           int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    kmin[i] = ~0ull;
    kmax[i] = 0ull;
  }
}

// exclusive prefix sum of v over the 1024 threads of the block; *total the sum
__device__ __forceinline__ uint32_t block_scan_1024(uint32_t v, uint32_t* wsum, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t s = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, s, off);
    if (lane >= off) s += t;
  }
  if (lane == 31) wsum[w] = s;
  __syncthreads();
  if (w == 0) {
    uint32_t t = wsum[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t q = __shfl_up_sync(0xffffffffu, t, off);
      if (lane >= off) t += q;
    }
    wsum[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const uint32_t before = (w > 0 ? wsum[w - 1] : 0u) + (s - v);
  *total = wsum[31];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kRoiSelectThreads) k_roi_select(
    const unsigned long long* __restrict__ kmin, const unsigned long long* __restrict__ kmax,
    unsigned long long* __restrict__ mkey, int64_t n, int metric, int mode, double value,
    int64_t k, double* __restrict__ metric_out, int64_t* __restrict__ sel,
    unsigned long long* __restrict__ nsel) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t wsum[32];
  __shared__ unsigned long long s_prefix, s_mask;
  __shared__ int64_t s_need;
  const int tid = threadIdx.x;
  // metrics and their keys
  for (int64_t u = tid; u < n; u += blockDim.x) {
    const unsigned long long hk = kmax[u];
    double m = -INFINITY;
    if (hk != 0ull) {
      const double hv = okey_val(hk);
      m = metric == STZ_ROI_MAX ? hv : __dsub_rn(hv, okey_val(kmin[u]));
    }
    if (metric_out) metric_out[u] = m;
    mkey[u] = okey(m);
  }
  __syncthreads();
  // top mode: the key T of the k-th largest metric; need = how many units
  // with key == T are kept (the lowest-index ones)
  unsigned long long T = 0ull;
  int64_t need = 0;
  if (mode == STZ_ROI_TOP) {
    if (tid == 0) {
      s_prefix = 0ull;
      s_mask = 0ull;
      s_need = k;
    }
    for (int pass = 7; pass >= 0; pass--) {
      for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0u;
      __syncthreads();
      const unsigned long long pre = s_prefix, msk = s_mask;
      for (int64_t u = tid; u < n; u += blockDim.x) {
        const unsigned long long key = mkey[u];
        if ((key & msk) == pre) atomicAdd(&hist[(key >> (8 * pass)) & 255u], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        int64_t rem = s_need;
        int d = 255;
        for (; d > 0; d--) {
          if ((int64_t)hist[d] >= rem) break;
          rem -= hist[d];
        }
        s_prefix = pre | ((unsigned long long)d << (8 * pass));
        s_mask = msk | (255ull << (8 * pass));
        s_need = rem;
      }
      __syncthreads();
    }
    T = s_prefix;
    need = s_need;
  }
  // compaction in unit order
  uint32_t kept = 0u, eq_before = 0u;
  for (int64_t u0 = 0; u0 < n; u0 += blockDim.x) {
    const int64_t u = u0 + tid;
    bool take = false, eq = false;
    if (u < n) {
      const unsigned long long key = mkey[u];
      if (mode == STZ_ROI_THRESHOLD) {
        take = okey_val(key) >= value;
      } else {
        eq = key == T;
        take = key > T;
      }
    }
    uint32_t eq_total;
    const uint32_t eq_rank = eq_before + block_scan_1024(eq ? 1u : 0u, wsum, &eq_total);
    if (eq && (int64_t)eq_rank < need) take = true;
    eq_before += eq_total;
    uint32_t tot;
    const uint32_t pos = kept + block_scan_1024(take ? 1u : 0u, wsum, &tot);
    if (take) sel[pos] = u;
    kept += tot;
  }
  if (tid == 0) *nsel = kept;
}

int launch_roi(const void* field, int dtype, const int64_t n[3], const int64_t b[3], int metric,
               int mode, double value, int64_t k, unsigned long long* kmin,
               unsigned long long* kmax, unsigned long long* mkey, double* metric_out,
               int64_t* sel, unsigned long long* nsel, cudaStream_t s) {
  RoiGeo g;
  g.npts = 1;
  g.nunits = 1;
  for (int a = 0; a < 3; a++) {
    g.n[a] = n[a];
    g.b[a] = b[a];
    g.nb[a] = cdiv(n[a], b[a]);
    g.npts *= n[a];
    g.nunits *= g.nb[a];
  }
  const int sms = launch_sms();
  {
    const int blocks = (int)imin(imax(cdiv(g.nunits, 256), 1), (int64_t)sms * 4);
    ProfScope ps_("k_roi_init", s);
    k_roi_init<<<blocks, 256, 0, s>>>(kmin, kmax, g.nunits);
    if (cudaGetLastError() != cudaSuccess) return STZ_ERR_CUDA;
  }
  {
    const int blocks = (int)imin(imax(cdiv(g.npts, 256), 1), (int64_t)sms * 8);
    const double bytes = (double)g.npts * (dtype == STZ_F32 ? 4 : 8);
    ProfScope ps_("k_roi_reduce", s, bytes);
    if (dtype == STZ_F32)
      k_roi_reduce<float><<<blocks, 256, 0, s>>>((const float*)field, g, kmin, kmax);
    else
      k_roi_reduce<double><<<blocks, 256, 0, s>>>((const double*)field, g, kmin, kmax);
    if (cudaGetLastError() != cudaSuccess) return STZ_ERR_CUDA;
  }
  ProfScope ps_("k_roi_select", s);
  k_roi_select<<<1, kRoiSelectThreads, 0, s>>>(kmin, kmax, mkey, g.nunits, metric, mode, value, k,
                                               metric_out, sel, nsel);
  return cuda_ok(cudaGetLastError());
}

}  // namespace stz
