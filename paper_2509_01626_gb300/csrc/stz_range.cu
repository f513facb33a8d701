// stz_range.cu -- value range of the finite values and the error-bound
// constants (absolute or value-range-relative bound; per-level bounds
// eb_l = eb_{l+1} / 2.5, Sec. 3.1 opt. 5, applied level by level as in the
// three-level scheme of Sec. 3.2).
#include "stz_kernels.cuh"
#include "stz_prof.cuh"

namespace stz {

// Order-preserving 64-bit keys: -0 sorts below +0, finite values only.
__device__ __forceinline__ unsigned long long key_f32(uint32_t u) {
  return (u & 0x80000000u) ? (unsigned long long)(~u) : (unsigned long long)(u | 0x80000000u);
}
__device__ __forceinline__ unsigned long long key_f64(unsigned long long u) {
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double val_f32(unsigned long long k) {
  uint32_t u = (uint32_t)k;
  u = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
  return (double)__uint_as_float(u);
}
__device__ __forceinline__ double val_f64(unsigned long long k) {
  unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)u);
}

__device__ __forceinline__ void upd(unsigned long long k, unsigned long long& lo,
                                    unsigned long long& hi) {
  lo = k < lo ? k : lo;
  hi = k > hi ? k : hi;
}

template <int DT>
__global__ void __launch_bounds__(256) k_range(const void* __restrict__ field, int64_t n,
                                               unsigned long long* __restrict__ part,
                                               uint32_t* __restrict__ z0, int64_t nz0,
                                               uint32_t* __restrict__ z1, int64_t nz1) {
  unsigned long long lo = ~0ull, hi = 0ull;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < nz0; i += nth) z0[i] = 0u;
  for (int64_t i = tid; i < nz1; i += nth) z1[i] = 0u;
  if (DT == STZ_F32) {
    // 32-bit keys (a float's key fits 32 bits; 0 and 0xFFFFFFFF are no key of
    // a finite value, so they serve as the empty bounds)
    uint32_t lo32 = 0xFFFFFFFFu, hi32 = 0u;
    auto upd32 = [&](uint32_t u) {
      if ((u & 0x7F800000u) != 0x7F800000u) {
        const uint32_t k = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        lo32 = min(lo32, k);
        hi32 = max(hi32, k);
      }
    };
    const uint32_t* f = (const uint32_t*)field;
    const int64_t n4 = n >> 2;
    const uint4* f4 = (const uint4*)field;
    int64_t i = tid;
    for (; i + 7 * nth < n4; i += 8 * nth) {  // eight 16-byte loads in flight per thread
      uint4 v[8];
#pragma unroll
      for (int k = 0; k < 8; k++) v[k] = __ldcs(f4 + i + k * nth);
#pragma unroll
      for (int k = 0; k < 8; k++) {
        upd32(v[k].x);
        upd32(v[k].y);
        upd32(v[k].z);
        upd32(v[k].w);
      }
    }
    for (; i < n4; i += nth) {
      const uint4 v = __ldg(f4 + i);
      upd32(v.x);
      upd32(v.y);
      upd32(v.z);
      upd32(v.w);
    }
    for (int64_t j = (n4 << 2) + tid; j < n; j += nth) upd32(f[j]);
    lo = lo32 == 0xFFFFFFFFu ? ~0ull : (unsigned long long)lo32;
    hi = (unsigned long long)hi32;
  } else {
    const unsigned long long* f = (const unsigned long long*)field;
    const int64_t n2 = n >> 1;
    const ulonglong2* f2 = (const ulonglong2*)field;
    const unsigned long long em = 0x7FF0000000000000ull;
    for (int64_t i = tid; i < n2; i += nth) {
      ulonglong2 v = __ldg(f2 + i);
      if ((v.x & em) != em) upd(key_f64(v.x), lo, hi);
      if ((v.y & em) != em) upd(key_f64(v.y), lo, hi);
    }
    for (int64_t i = (n2 << 1) + tid; i < n; i += nth) {
      unsigned long long u = f[i];
      if ((u & em) != em) upd(key_f64(u), lo, hi);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, off);
    unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, off);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  __shared__ unsigned long long slo[8], shi[8];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    slo[w] = lo;
    shi[w] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
      lo = slo[i] < lo ? slo[i] : lo;
      hi = shi[i] > hi ? shi[i] : hi;
    }
    part[2 * blockIdx.x] = lo;
    part[2 * blockIdx.x + 1] = hi;
  }
}

// largest float <= v (v > 0)
__device__ __forceinline__ float rz_float(double v) { return __double2float_rz(v); }

__global__ void __launch_bounds__(256) k_params(DevParams* dp,
                                                const unsigned long long* __restrict__ part,
                                                int nparts, int dtype, int eb_mode, double eb,
                                                int L, int R, double ratio, int pred) {
  unsigned long long lo = ~0ull, hi = 0ull;
  if (eb_mode == STZ_EB_REL) {
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
      const unsigned long long l = part[2 * b], h = part[2 * b + 1];
      lo = l < lo ? l : lo;
      hi = h > hi ? h : hi;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, off);
    const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, off);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  __shared__ unsigned long long slo[8], shi[8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    slo[w] = lo;
    shi[w] = hi;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
    lo = slo[i] < lo ? slo[i] : lo;
    hi = shi[i] > hi ? shi[i] : hi;
  }
  dp->range_lo = lo;
  dp->range_hi = hi;
  dp->status = 0;
  double vmin = 0.0, vmax = 0.0;
  bool any = false;
  if (eb_mode == STZ_EB_REL && dp->range_lo != ~0ull) {
    any = true;
    vmin = dtype == STZ_F32 ? val_f32(dp->range_lo) : val_f64(dp->range_lo);
    vmax = dtype == STZ_F32 ? val_f32(dp->range_hi) : val_f64(dp->range_hi);
  }
  double ea = eb;
  if (eb_mode == STZ_EB_REL) {
    double range = any ? __dsub_rn(vmax, vmin) : 0.0;
    ea = __dmul_rn(eb, range);
    if (!(ea > 0.0) || !isfinite(ea)) ea = eb;
  }
  dp->eb = eb;
  dp->eb_abs = ea;
  dp->eb_ratio = ratio;
  dp->pred = (uint32_t)pred;
  dp->vmin = vmin;
  dp->vmax = vmax;
  for (int l = 0; l <= kMaxLevels; l++) {
    dp->eb_level[l] = dp->two_eb_d[l] = 0.0;
    dp->inv2eb_f[l] = dp->two_eb_f[l] = dp->ebc_f[l] = 0.f;
    dp->inv2eb_d[l] = dp->two_eb_dd[l] = dp->ebc_d[l] = 0.0;
  }
  for (int l = 1; l <= L; l++) {
    double r = 1.0;
    for (int k = 0; k < L - l; k++) r = __dmul_rn(r, ratio);
    double ebl = __ddiv_rn(ea, r);
    dp->eb_level[l] = ebl;
    double two = __dmul_rn(2.0, ebl);
    double inv = __ddiv_rn(1.0, two);
    if (dtype == STZ_F32) {
      dp->two_eb_f[l] = __double2float_rn(two);
      dp->inv2eb_f[l] = __double2float_rn(inv);
      dp->ebc_f[l] = nextafterf(rz_float(ebl), 0.0f);
      dp->two_eb_d[l] = (double)dp->two_eb_f[l];
    } else {
      dp->two_eb_dd[l] = two;
      dp->inv2eb_d[l] = inv;
      dp->ebc_d[l] = nextafter(ebl, 0.0);
      dp->two_eb_d[l] = two;
    }
  }
  (void)R;
}

int launch_range(const void* field, int dtype, int64_t n, unsigned long long* part, int* nparts,
                 uint32_t* z0, int64_t nz0, uint32_t* z1, int64_t nz1, cudaStream_t s) {
  const int sms = launch_sms();
  const int64_t per = dtype == STZ_F32 ? 4 : 2;
  const int64_t want = imax(cdiv(cdiv(n, per), 256), cdiv(imax(nz0, nz1), 256));
  // 12 blocks per SM measured fastest (0.088 ms at 512^3, against 0.101 at 8)
  const int blocks = (int)imin(imax(want, 1), imin((int64_t)sms * 12, kRangeMaxBlocks));
  *nparts = blocks;
  ProfScope ps_("k_range", s, (double)n * (dtype == STZ_F32 ? 4 : 8));  // one read of the field
  if (dtype == STZ_F32) k_range<STZ_F32><<<blocks, 256, 0, s>>>(field, n, part, z0, nz0, z1, nz1);
  else k_range<STZ_F64><<<blocks, 256, 0, s>>>(field, n, part, z0, nz0, z1, nz1);
  return cuda_ok(cudaGetLastError());
}

int launch_params(DevParams* dp, const unsigned long long* part, int nparts, int dtype,
                  int eb_mode, double eb, int L, int R, double ratio, int pred, cudaStream_t s) {
  ProfScope ps_("k_params", s);
  k_params<<<1, 256, 0, s>>>(dp, part, nparts, dtype, eb_mode, eb, L, R, ratio, pred);
  return cuda_ok(cudaGetLastError());
}

}  // namespace stz
