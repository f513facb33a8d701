// stz_huffman.cu -- Huffman coding of each sub-block's quantization codes as
// one unit (Sec. 2.1 step 3, Sec. 3.3), cut into brick chunks that decode
// independently (the random-access decoding the paper leaves to future work,
// Sec. 5).
//
// Code construction (one thread block per stream, all streams at once):
// live symbols sorted by (frequency, symbol); two-queue Huffman merge with a
// leaf winning ties; code counts per length; if the longest exceeds 12 the
// counts are repaired as in ITU-T T.81 Annex K.3; lengths handed out by
// frequency rank; canonical codes by (length, symbol), MSB-first.
// Decoding: 4096-entry table indexed by the next 12 bits, one thread per
// chunk.
#include "stz_kernels.cuh"
#include "stz_prof.cuh"

namespace stz {

// ---------------------------------------------------------------- histograms
__global__ void __launch_bounds__(256) k_stream_hist(const __grid_constant__ Geo g, int sid,
                                                     const uint16_t* __restrict__ codes,
                                                     uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kAlphabet];
  for (int i = threadIdx.x; i < kAlphabet; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const StreamGeo& sg = g.s[sid];
  for (int64_t j = blockIdx.x; j < sg.nchunks; j += gridDim.x) {
    int64_t B[3], l[3], start;
    chunk_brick(sg, g.b, j, B, l, &start);
    const int64_t cnt = l[0] * l[1] * l[2];
    const uint16_t* c = codes + (sg.chunk0 + j) * g.bvol;
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) atomicAdd(&h[c[i]], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kAlphabet; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[(int64_t)sid * kAlphabet + i], h[i]);
}

int launch_stream_hist(const Geo& g, int sid, const uint16_t* codes, uint32_t* hist,
                       cudaStream_t s) {
  if (g.s[sid].nchunks == 0) return STZ_OK;
  int blocks = (int)imin(g.s[sid].nchunks, 304);
  ProfScope ps_("k_stream_hist", s);
  k_stream_hist<<<blocks, 256, 0, s>>>(g, sid, codes, hist);
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------- codebook
constexpr int kBookThreads = 1024;

__device__ void bitonic_sort_u64(unsigned long long* k, int n /* power of 2 */) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
        int lo = 2 * i - (i & (stride - 1));
        int hi = lo + stride;
        bool asc = (lo & size) == 0;
        unsigned long long a = k[lo], b = k[hi];
        if ((a > b) == asc) {
          k[lo] = b;
          k[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kBookThreads) k_codebook(const uint32_t* __restrict__ hist,
                                                           uint16_t* __restrict__ enc,
                                                           BookDev* __restrict__ books) {
  __shared__ unsigned long long key[kAlphabet];
  __shared__ unsigned long long iw[kAlphabet];
  __shared__ uint16_t par_leaf[kAlphabet];
  __shared__ uint16_t par_int[kAlphabet];
  __shared__ uint8_t dep[kAlphabet];
  __shared__ uint8_t len_of[kAlphabet];
  __shared__ int bl[64];
  __shared__ uint32_t first_code[32];
  __shared__ int first_index[32];
  __shared__ int s_n;
  const int s = blockIdx.x;
  const int tid = threadIdx.x;
  const uint32_t* h = hist + (int64_t)s * kAlphabet;
  if (tid == 0) s_n = 0;
  if (tid < 64) bl[tid] = 0;
  __syncthreads();
  int live = 0;
  for (int i = tid; i < kAlphabet; i += blockDim.x) {
    uint32_t f = h[i];
    key[i] = f ? (((unsigned long long)f << 11) | (unsigned long long)i) : ~0ull;
    len_of[i] = 0;
    live += f != 0;
  }
  if (live) atomicAdd(&s_n, live);
  __syncthreads();
  bitonic_sort_u64(key, kAlphabet);  // ends with a barrier
  const int nl = s_n;
  BookDev* bk = books + s;
  uint16_t* e = enc + (int64_t)s * kAlphabet;
  if (nl == 0) {
    for (int i = tid; i < kAlphabet; i += blockDim.x) e[i] = 0;
    if (tid == 0) bk->nlive = 0;
    return;
  }
  if (nl == 1) {
    const int sym = (int)(key[0] & 2047ull);
    for (int i = tid; i < kAlphabet; i += blockDim.x) e[i] = (i == sym) ? (uint16_t)1 : 0;
    if (tid == 0) {
      bk->nlive = 1;
      bk->sym[0] = (uint16_t)sym;
      bk->len[0] = 1;
    }
    return;
  }
  // two-queue merge (sequential, one thread)
  if (tid == 0) {
    int i = 0, j = 0;
    unsigned long long lw = key[0] >> 11;
    unsigned long long jw = 0;
    for (int k = 0; k < nl - 1; k++) {
      unsigned long long w = 0;
#pragma unroll
      for (int pick = 0; pick < 2; pick++) {
        const bool take_leaf = i < nl && (j >= k || lw <= jw);
        if (take_leaf) {
          w += lw;
          par_leaf[i] = (uint16_t)k;
          i++;
          lw = i < nl ? (key[i] >> 11) : 0ull;
        } else {
          w += jw;
          par_int[j] = (uint16_t)k;
          j++;
          jw = j < k ? iw[j] : 0ull;
        }
      }
      iw[k] = w;
      if (j == k) jw = w;  // the queue was empty: its head is the new node
    }
    dep[nl - 2] = 0;
    for (int k = nl - 3; k >= 0; k--) dep[k] = (uint8_t)(dep[par_int[k]] + 1);
  }
  __syncthreads();
  for (int i = tid; i < nl; i += blockDim.x) atomicAdd(&bl[min(dep[par_leaf[i]] + 1, 63)], 1);
  __syncthreads();
  if (tid == 0) {
    int maxd = 0;
    for (int d = 1; d < 64; d++)
      if (bl[d]) maxd = d;
    for (int L = maxd; L > kMaxCodeLen; L--) {
      while (bl[L] > 0) {
        int jj = L - 2;
        while (jj > 0 && bl[jj] == 0) jj--;
        bl[L] -= 2;
        bl[L - 1] += 1;
        bl[jj + 1] += 2;
        bl[jj] -= 1;
      }
    }
    uint32_t code = 0;
    int idx = 0;
    for (int L = 1; L <= kMaxCodeLen; L++) {
      first_code[L] = code;
      first_index[L] = idx;
      code = (code + (uint32_t)bl[L]) << 1;
      idx += bl[L];
    }
  }
  __syncthreads();
  // lengths by rank: sorted index i (ascending frequency) has rank nl-1-i
  for (int i = tid; i < nl; i += blockDim.x) {
    int r = nl - 1 - i;
    int L = 1, cum = bl[1];
    while (r >= cum) {
      L++;
      cum += bl[L];
    }
    len_of[key[i] & 2047ull] = (uint8_t)L;
  }
  __syncthreads();
  // canonical order: sort (length, symbol)
  for (int i = tid; i < kAlphabet; i += blockDim.x)
    key[i] = len_of[i] ? (((unsigned long long)len_of[i] << 11) | (unsigned long long)i) : ~0ull;
  __syncthreads();
  bitonic_sort_u64(key, kAlphabet);
  for (int i = tid; i < kAlphabet; i += blockDim.x) e[i] = 0;
  __syncthreads();
  for (int k = tid; k < nl; k += blockDim.x) {
    const int L = (int)(key[k] >> 11);
    const int sym = (int)(key[k] & 2047ull);
    const uint32_t code = first_code[L] + (uint32_t)(k - first_index[L]);
    e[sym] = (uint16_t)((code << 4) | (uint32_t)L);
    bk->sym[k] = (uint16_t)sym;
    bk->len[k] = (uint8_t)L;
  }
  if (tid == 0) bk->nlive = (uint32_t)nl;
}

int launch_codebook(const Geo& g, const uint32_t* hist, uint16_t* enc, BookDev* books,
                    cudaStream_t s) {
  ProfScope ps_("k_codebook", s);
  k_codebook<<<g.nstreams, kBookThreads, 0, s>>>(hist, enc, books);
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------- chunk sizes
__device__ __forceinline__ int stream_of_chunk(const Geo& g, int64_t j) {
  int sid = 0;
  for (int s = 1; s < g.nstreams; s++)
    if (g.s[s].nchunks > 0 && g.s[s].chunk0 <= j) sid = s;
  return sid;
}

__device__ __forceinline__ int64_t chunk_count(const Geo& g, int sid, int64_t jl) {
  int64_t B[3], l[3], start;
  chunk_brick(g.s[sid], g.b, jl, B, l, &start);
  return l[0] * l[1] * l[2];
}

__global__ void __launch_bounds__(256) k_chunk_words(const __grid_constant__ Geo g,
                                                     const uint16_t* __restrict__ codes,
                                                     const uint16_t* __restrict__ enc,
                                                     uint32_t* __restrict__ words) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= g.total_chunks) return;
  const int sid = stream_of_chunk(g, j);
  const int64_t cnt = chunk_count(g, sid, j - g.s[sid].chunk0);
  const uint16_t* c = codes + j * g.bvol;
  const uint16_t* e = enc + (int64_t)sid * kAlphabet;
  uint32_t bits = 0;
  for (int64_t i = lane; i < cnt; i += 32) bits += e[c[i]] & 15u;
  for (int off = 16; off > 0; off >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, off);
  if (lane == 0) words[j] = (bits + 31) >> 5;
}

int launch_chunk_words(const Geo& g, const uint16_t* codes, const uint16_t* enc, uint32_t* words,
                       cudaStream_t s) {
  if (g.total_chunks == 0) return STZ_OK;
  int64_t blocks = cdiv(g.total_chunks * 32, 256);
  ProfScope ps_("k_chunk_words", s);
  k_chunk_words<<<(unsigned)blocks, 256, 0, s>>>(g, codes, enc, words);
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------- scan
// Exclusive prefix sums of two u32 arrays (chunk payload words, chunk outlier
// counts) into u64 offsets, in two launches over tiles of 4096: per-tile sums,
// then per-tile scans offset by the sum of the earlier tiles.
constexpr int kScanThreads = 1024, kScanTile = 4096;

__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              unsigned long long* wsum,
                                                              unsigned long long* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  *total = wsum[31];
  return x - v + (w > 0 ? wsum[w - 1] : 0ull);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* __restrict__ a,
                                                             const uint32_t* __restrict__ b,
                                                             int64_t n,
                                                             unsigned long long* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  unsigned long long sa = 0, sb = 0;
  for (int k = 0; k < kScanTile / kScanThreads; k++) {
    const int64_t i = base + k * kScanThreads + threadIdx.x;
    if (i < n) {
      sa += a[i];
      sb += b[i];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  __shared__ unsigned long long ra[32], rb[32];
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x >> 5] = sa;
    rb[threadIdx.x >> 5] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long ta = 0, tb = 0;
    for (int w = 0; w < kScanThreads / 32; w++) {
      ta += ra[w];
      tb += rb[w];
    }
    sums[2 * blockIdx.x] = ta;
    sums[2 * blockIdx.x + 1] = tb;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(
    const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, int64_t n,
    const unsigned long long* __restrict__ sums, unsigned long long* __restrict__ oa,
    unsigned long long* __restrict__ ob) {
  __shared__ uint32_t ta[kScanTile], tbuf[kScanTile];
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long pre[2];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  if (threadIdx.x < 32) {
    unsigned long long pa = 0, pb = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += 32) {
      pa += sums[2 * t];
      pb += sums[2 * t + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
      pa += __shfl_xor_sync(0xffffffffu, pa, o);
      pb += __shfl_xor_sync(0xffffffffu, pb, o);
    }
    if (threadIdx.x == 0) {
      pre[0] = pa;
      pre[1] = pb;
    }
  }
  for (int k = 0; k < kScanTile / kScanThreads; k++) {
    const int j = k * kScanThreads + threadIdx.x;
    const int64_t i = base + j;
    ta[j] = i < n ? a[i] : 0u;
    tbuf[j] = i < n ? b[i] : 0u;
  }
  __syncthreads();
  constexpr int per = kScanTile / kScanThreads;
  for (int arr = 0; arr < 2; arr++) {
    const uint32_t* t = arr == 0 ? ta : tbuf;
    unsigned long long* o = arr == 0 ? oa : ob;
    unsigned long long loc[per];
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < per; k++) {
      loc[k] = sum;
      sum += t[threadIdx.x * per + k];
    }
    unsigned long long total;
    const unsigned long long off = block_excl_scan(sum, wsum, &total) + pre[arr];
#pragma unroll
    for (int k = 0; k < per; k++) {
      const int64_t i = base + threadIdx.x * per + k;
      if (i < n) o[i] = off + loc[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) o[n] = pre[arr] + total;
    __syncthreads();
  }
}

int launch_scan2(const uint32_t* a, const uint32_t* b, int64_t n, unsigned long long* sums,
                 unsigned long long* oa, unsigned long long* ob, cudaStream_t s) {
  const int64_t nb = imax(1, cdiv(n, kScanTile));
  {
    ProfScope ps_("k_scan_tiles", s);
    k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, s>>>(a, b, n, sums);
  }
  ProfScope ps_("k_scan_apply", s);
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(a, b, n, sums, oa, ob);
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------- bit packing
constexpr int kPackWarps = 8;

__global__ void __launch_bounds__(kPackWarps * 32) k_pack(
    const __grid_constant__ Geo g, const uint16_t* __restrict__ codes,
    const uint16_t* __restrict__ enc, const unsigned long long* __restrict__ word_off,
    const SectDev* __restrict__ sect, uint8_t* __restrict__ out, const DevParams* dp) {
  extern __shared__ uint32_t wbuf[];  // kPackWarps * maxw
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t maxw = (g.bvol * kMaxCodeLen + 31) / 32;
  uint32_t* buf = wbuf + w * maxw;
  const int64_t j = (int64_t)blockIdx.x * kPackWarps + w;
  if (j >= g.total_chunks) return;
  if (dp->status & kStatCapacity) return;
  const int sid = stream_of_chunk(g, j);
  const int64_t cnt = chunk_count(g, sid, j - g.s[sid].chunk0);
  const int64_t nw = (int64_t)(word_off[j + 1] - word_off[j]);
  for (int64_t i = lane; i < nw; i += 32) buf[i] = 0;
  __syncwarp();
  const uint16_t* c = codes + j * g.bvol;
  const uint16_t* e = enc + (int64_t)sid * kAlphabet;
  const SectDev& sd = sect[sid];
  const int64_t q = (cnt + kNSub - 1) / kNSub;
  uint16_t* so = (uint16_t*)(out + sd.sect_off + sd.off_subs) + (j - g.s[sid].chunk0) * (kNSub - 1);
  uint32_t base = 0;
  for (int64_t i0 = 0; i0 < cnt; i0 += 32) {
    const int64_t i = i0 + lane;
    uint32_t code = 0, len = 0;
    if (i < cnt) {
      uint32_t v = e[c[i]];
      code = v >> 4;
      len = v & 15u;
    }
    uint32_t incl = len;
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += t;
    }
    const uint32_t p = base + incl - len;
#pragma unroll
    for (int u = 1; u < kNSub; u++)
      if (i == u * q && i < cnt) so[u - 1] = (uint16_t)p;
    if (len) {
      const uint32_t wi = p >> 5, r = p & 31u;
      if (r + len <= 32u) {
        atomicOr(&buf[wi], code << (32u - r - len));
      } else {
        atomicOr(&buf[wi], code >> (r + len - 32u));
        atomicOr(&buf[wi + 1], code << (64u - r - len));
      }
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0)
    for (int u = 1; u < kNSub; u++)
      if (u * q >= cnt) so[u - 1] = (uint16_t)base;
  __syncwarp();
  uint32_t* dst = (uint32_t*)(out + sd.sect_off + sd.off_payload) + (word_off[j] - sd.word0);
  for (int64_t i = lane; i < nw; i += 32) dst[i] = buf[i];
}

int launch_pack(const Geo& g, const uint16_t* codes, const uint16_t* enc,
                const unsigned long long* word_off, const SectDev* sect, uint8_t* out,
                const DevParams* dp, cudaStream_t s) {
  if (g.total_chunks == 0) return STZ_OK;
  const int64_t maxw = (g.bvol * kMaxCodeLen + 31) / 32;
  size_t smem = sizeof(uint32_t) * kPackWarps * maxw;
  if (cudaFuncSetAttribute(k_pack, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return STZ_ERR_CUDA;
  int64_t blocks = cdiv(g.total_chunks, kPackWarps);
  ProfScope ps_("k_pack", s);
  k_pack<<<(unsigned)blocks, kPackWarps * 32, smem, s>>>(g, codes, enc, word_off, sect, out, dp);
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------- decode tables
__global__ void __launch_bounds__(256) k_lut(const __grid_constant__ DecTables tb,
                                             uint32_t* __restrict__ lut,
                                             uint32_t* __restrict__ status) {
  __shared__ int cnt[32];
  __shared__ uint32_t fcode[32];
  __shared__ int fidx[32];
  __shared__ int bad;
  const int sid = tb.lut_sid[blockIdx.x];
  const DecStream& d = tb.ds[sid];
  uint32_t* t = lut + (int64_t)sid * kLutSize;
  const int tid = threadIdx.x;
  if (tid < 32) cnt[tid] = 0;
  if (tid == 0) bad = 0;
  for (int i = tid; i < kLutSize; i += blockDim.x) t[i] = 0;
  __syncthreads();
  const uint16_t* syms = (const uint16_t*)(d.sect + d.off_syms);
  const uint8_t* lens = d.sect + d.off_lens;
  for (int64_t k = tid; k < (int64_t)d.nlive; k += blockDim.x) {
    int L = lens[k], sym = syms[k];
    if (L < 1 || L > kMaxCodeLen || sym >= kAlphabet) {
      bad = 1;
      continue;
    }
    if (k > 0) {
      int Lp = lens[k - 1], sp = syms[k - 1];
      if (!(L > Lp || (L == Lp && sym > sp))) bad = 1;
    }
    atomicAdd(&cnt[L], 1);
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t code = 0;
    int idx = 0;
    long long kraft = 0;
    for (int L = 1; L <= kMaxCodeLen; L++) {
      fcode[L] = code;
      fidx[L] = idx;
      code = (code + (uint32_t)cnt[L]) << 1;
      idx += cnt[L];
      kraft += (long long)cnt[L] << (kMaxCodeLen - L);
    }
    if (kraft > kLutSize) bad = 1;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) atomicOr(status, kStatCorrupt);
    return;
  }
  for (int64_t k = tid; k < (int64_t)d.nlive; k += blockDim.x) {
    const int L = lens[k], sym = syms[k];
    const uint32_t code = fcode[L] + (uint32_t)(k - fidx[L]);
    const uint32_t lo = code << (kMaxCodeLen - L), hi = (code + 1) << (kMaxCodeLen - L);
    const uint32_t v = ((uint32_t)sym << 8) | (uint32_t)L;
    for (uint32_t i = lo; i < hi; i++) t[i] = v;
  }
}

int launch_lut(const DecTables& tb, uint32_t* lut, uint32_t* status, cudaStream_t s) {
  if (tb.nlut == 0) return STZ_OK;
  ProfScope ps_("k_lut", s);
  k_lut<<<tb.nlut, 256, 0, s>>>(tb, lut, status);
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------- chunk decode
// One thread per sub-chunk: a chunk of n symbols is cut into nsub runs of
// q = ceil(n / nsub) symbols whose start bits are stored, so every run decodes
// independently.  A run that does not end exactly where the next one starts,
// reads past its chunk, or meets an invalid code marks the container corrupt.
__global__ void __launch_bounds__(kDecThreads) k_decode_chunks(
    const __grid_constant__ Geo g, const __grid_constant__ DecTables tb,
    const uint32_t* __restrict__ lut, uint16_t* __restrict__ codes,
    uint32_t* __restrict__ status) {
  __shared__ uint32_t t[kLutSize];
  int jb = 0;
  for (int k = 1; k < tb.njobs; k++)
    if (tb.jobs[k].block0 <= (int64_t)blockIdx.x) jb = k;
  const DecChunkJob& job = tb.jobs[jb];
  const int sid = job.sid;
  const uint32_t* src = lut + (int64_t)sid * kLutSize;
  for (int i = threadIdx.x; i < kLutSize; i += blockDim.x) t[i] = src[i];
  __syncthreads();
  const DecStream& d = tb.ds[sid];
  const int nsub = d.nsub;
  const int64_t qq = ((int64_t)blockIdx.x - job.block0) * kDecThreads + threadIdx.x;
  const int64_t q = qq / nsub;
  const int u = (int)(qq - q * nsub);
  if (q >= job.nchunks_job) return;
  const StreamGeo& sg = g.s[sid];
  const int64_t B0 = job.lo[0] + q / (job.cnt[1] * job.cnt[2]);
  const int64_t B1 = job.lo[1] + (q / job.cnt[2]) % job.cnt[1];
  const int64_t B2 = job.lo[2] + q % job.cnt[2];
  const int64_t jl = (B0 * sg.nb[1] + B1) * sg.nb[2] + B2;
  const int64_t cnt = imin(g.b[0], sg.e[0] - B0 * g.b[0]) * imin(g.b[1], sg.e[1] - B1 * g.b[1]) *
                      imin(g.b[2], sg.e[2] - B2 * g.b[2]);
  const int64_t per = (cnt + nsub - 1) / nsub;
  const int64_t i0 = imin(cnt, (int64_t)u * per), i1 = imin(cnt, (int64_t)(u + 1) * per);
  const uint32_t* coff = (const uint32_t*)(d.sect + d.off_chunks);
  const uint16_t* soff = (const uint16_t*)(d.sect + d.off_subs) + jl * (nsub - 1);
  const uint32_t* pay = (const uint32_t*)(d.sect + d.off_payload);
  const uint64_t w0 = coff[jl];
  const uint64_t w1 = jl + 1 < (int64_t)d.nchunks ? coff[jl + 1] : d.pw;
  uint16_t* out = codes + (job.slot_base + q) * g.bvol;
  const uint64_t cbits = w1 >= w0 ? (w1 - w0) * 32 : 0;
  const uint64_t b0 = u == 0 ? 0 : soff[u - 1];
  const uint64_t b1 = u + 1 < nsub ? soff[u] : cbits;
  if (w0 > w1 || w1 > d.pw || b0 > b1 || b1 > cbits) {
    atomicOr(status, kStatCorrupt);
    for (int64_t i = i0; i < i1; i++) out[i] = 0;
    return;
  }
  const uint32_t* wp = pay + w0 + (b0 >> 5);
  const uint32_t* we = pay + w1;
  unsigned long long buf = 0;
  int nb = 0;
  uint64_t consumed = 0;
  {
    const int sh = (int)(b0 & 31);
    uint32_t word = wp < we ? *wp : 0u;
    wp++;
    buf = (unsigned long long)word << (32 + sh);
    nb = 32 - sh;
  }
  bool badcode = false;
  // decode one symbol: refill below 32 buffered bits, look up the next 12
  auto next = [&]() -> uint32_t {
    if (nb < 32) {
      uint32_t word = wp < we ? *wp : 0u;
      wp++;
      buf |= (unsigned long long)word << (32 - nb);
      nb += 32;
    }
    const uint32_t ent = t[buf >> (64 - kMaxCodeLen)];
    int L = (int)(ent & 255u);
    if (L == 0) {
      badcode = true;
      L = 1;
    }
    buf <<= L;
    nb -= L;
    consumed += (uint64_t)L;
    return ent >> 8;
  };
  int64_t i = i0;
  // 8 symbols per 16-byte store where the run start is 16-byte aligned
  if ((((uintptr_t)(out + i)) & 15) == 0) {
    for (; i + 8 <= i1; i += 8) {
      uint32_t v[4];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const uint32_t lo = next();
        const uint32_t hi = next();
        v[k] = lo | (hi << 16);
      }
      *(uint4*)(out + i) = make_uint4(v[0], v[1], v[2], v[3]);
    }
  }
  for (; i < i1; i++) out[i] = (uint16_t)next();
  const bool exact = u + 1 < nsub ? (b0 + consumed == b1) : (b0 + consumed <= b1);
  if (badcode || !exact) atomicOr(status, kStatCorrupt);
}

int launch_decode_chunks(const Geo& g, const DecTables& tb, const uint32_t* lut,
                         uint16_t* codes, uint32_t* status, cudaStream_t s) {
  if (tb.nblocks == 0) return STZ_OK;
  ProfScope ps_("k_decode_chunks", s);
  k_decode_chunks<<<(unsigned)tb.nblocks, kDecThreads, 0, s>>>(g, tb, lut, codes, status);
  return cuda_ok(cudaGetLastError());
}

}  // namespace stz
