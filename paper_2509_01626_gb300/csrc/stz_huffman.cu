// stz_huffman.cu -- Huffman coding of each sub-block's quantization codes as
// one unit (Sec. 2.1 step 3, Sec. 3.3), cut into brick chunks that decode
// independently (the random-access decoding the paper leaves to future work,
// Sec. 5).
//
// Code construction (one thread block per stream, all streams at once):
// live symbols sorted by (frequency, symbol); two-queue Huffman merge with a
// leaf winning ties; code counts per length; if the longest exceeds 12 the
// longer codes are clamped to 12 and the Kraft excess is removed by moving
// codes one length deeper, deepest lengths first; lengths handed out by
// frequency rank; canonical codes by (length, symbol), MSB-first.
// Decoding: each block stages its chunks' payload words in shared memory and
// one thread decodes one sub-chunk through a 4096-entry table indexed by the
// next 12 bits.
#include "stz_kernels.cuh"
#include "stz_prof.cuh"

namespace stz {

// ---------------------------------------------------------------- histograms
// Histogram of one stream from its chunk slots: a block takes kHistChunks
// chunks at once, one 16-byte word (8 codes) of each per thread, so that all
// its loads are in flight before the shared-memory counts; the most frequent
// symbol (the zero-error code) is counted by ballot.
constexpr int kHistChunks = 4;

__global__ void __launch_bounds__(256) k_stream_hist(const __grid_constant__ Geo g, int sid,
                                                     const uint16_t* __restrict__ codes,
                                                     uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kAlphabet];
  for (int i = threadIdx.x; i < kAlphabet; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const StreamGeo& sg = g.s[sid];
  const int lane = threadIdx.x & 31;
  const int words = (int)(g.bvol / 8);  // 16-byte words per chunk slot
  for (int64_t j0 = (int64_t)blockIdx.x * kHistChunks; j0 < sg.nchunks;
       j0 += (int64_t)gridDim.x * kHistChunks) {
    uint4 v[kHistChunks];
    int cnt[kHistChunks];
#pragma unroll
    for (int u = 0; u < kHistChunks; u++) {
      const int64_t j = j0 + u;
      cnt[u] = 0;
      v[u] = make_uint4(0u, 0u, 0u, 0u);
      if (j < sg.nchunks) {
        int64_t B[3], l[3], start;
        chunk_brick(sg, g.b, j, B, l, &start);
        cnt[u] = (int)(l[0] * l[1] * l[2]);
        if ((int)threadIdx.x < words && 8 * (int)threadIdx.x < cnt[u])
          v[u] = __ldg((const uint4*)(codes + (sg.chunk0 + j) * g.bvol) + threadIdx.x);
      }
    }
#pragma unroll
    for (int u = 0; u < kHistChunks; u++) {
      const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
      for (int e = 0; e < 8; e++) {
        const int sym = (int)((w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
        const bool in = 8 * (int)threadIdx.x + e < cnt[u];
        const unsigned bm = __ballot_sync(0xffffffffu, in && sym == kRadius);
        if (lane == 0 && bm) atomicAdd(&h[kRadius], (uint32_t)__popc(bm));
        if (in && sym != kRadius) atomicAdd(&h[sym], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kAlphabet; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[(int64_t)sid * kAlphabet + i], h[i]);
}

int launch_stream_hist(const Geo& g, int sid, const uint16_t* codes, uint32_t* hist,
                       cudaStream_t s) {
  if (g.s[sid].nchunks == 0) return STZ_OK;
  // one thread per 16-byte word of a chunk slot
  if (g.bvol % 8 != 0 || g.bvol > 8 * 256) return STZ_ERR_ARG;
  const int blocks = (int)imin(cdiv(g.s[sid].nchunks, kHistChunks), 304);
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

// First index in [lo, hi) whose value v(index) exceeds m, values
// non-decreasing; hi if none.  The whole warp searches: 32 probes a step.
template <typename V>
__device__ __forceinline__ int warp_upper(V v, int lo, int hi, uint32_t m, int lane) {
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) >> 5;
    const int p = min(lo + (lane + 1) * step - 1, hi - 1);  // lane 31 probes hi - 1
    const unsigned b = __ballot_sync(0xffffffffu, v(p) > m);
    if (!b) return hi;
    const int f = __ffs(b) - 1;
    const int pf = min(lo + (f + 1) * step - 1, hi - 1);
    lo = f == 0 ? lo : min(lo + f * step - 1, hi - 1) + 1;
    hi = pf + 1;  // v(pf) > m: the answer is at most pf
  }
  const int p = lo + lane;
  const unsigned b = __ballot_sync(0xffffffffu, p < hi && v(p) > m);
  return b ? lo + __ffs(b) - 1 : hi;
}

__global__ void __launch_bounds__(kBookThreads) k_codebook(const uint32_t* __restrict__ hist,
                                                           uint16_t* __restrict__ enc,
                                                           BookDev* __restrict__ books, int s0) {
  __shared__ unsigned long long key[kAlphabet];
  __shared__ uint32_t iw[kAlphabet];
  __shared__ uint16_t par_leaf[kAlphabet];
  __shared__ uint16_t par_int[kAlphabet];
  __shared__ uint8_t dep[kAlphabet];
  __shared__ uint8_t len_of[kAlphabet];
  __shared__ int bl[64];
  __shared__ uint32_t first_code[32];
  __shared__ int first_index[32];
  __shared__ int wcnt[2 * kBookThreads / 32][kMaxCodeLen + 1];  // per warp-group, per length
  __shared__ uint16_t merged[kAlphabet];  // a merge round's picks: leaf, or 0x8000 | node
  __shared__ int s_n;
  const int s = s0 + blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t* h = hist + (int64_t)s * kAlphabet;
  if (tid == 0) s_n = 0;
  if (tid < 64) bl[tid] = 0;
  __syncthreads();
  // compact the live symbols (in symbol order) into key[0..n)
  for (int r = 0; r < kAlphabet / kBookThreads; r++) {
    const int sym = r * kBookThreads + tid;
    const uint32_t f = h[sym];
    len_of[sym] = 0;
    const unsigned bm = __ballot_sync(0xffffffffu, f != 0);
    int base = 0;
    if (lane == 0) base = atomicAdd(&s_n, __popc(bm));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (f) key[base + __popc(bm & ((1u << lane) - 1u))] = ((unsigned long long)f << 11) | (unsigned long long)sym;
  }
  __syncthreads();
  const int nl = s_n;
  int P = 1;
  while (P < nl) P <<= 1;
  for (int i = nl + tid; i < P; i += blockDim.x) key[i] = ~0ull;
  __syncthreads();
  if (P > 1) bitonic_sort_u64(key, P);  // (frequency, symbol) ascending
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
  // The two-queue merge: leaves in (frequency, symbol) order, internal nodes
  // in creation order, always the two lightest heads, a leaf before an
  // internal node of equal weight.  Its picks are the merge of the two
  // sorted queues, so one warp takes them in rounds: with m the weight of the
  // next node (the two lightest heads), every queued node of weight <= m is
  // picked before any node created from here on (those weigh >= m and are
  // newer), so the t nodes of weight <= m pair up in merge order into
  // floor(t / 2) new nodes at once; an odd one waits for the next round.
  // A stream's rounds are about the log of its weight (20-24 measured),
  // instead of one dependent step per node.
  if (w == 0) {
    auto lwt = [&](int x) -> uint32_t { return (uint32_t)(key[x] >> 11); };
    auto iwt = [&](int x) -> uint32_t { return iw[x]; };
    int i = 0, j = 0, k = 0;
    while (k < nl - 1) {
      uint32_t m = 0;
      {
        int ii = i, jj = j;
#pragma unroll
        for (int p = 0; p < 2; p++) {
          const uint32_t lv = ii < nl ? lwt(ii) : 0u, iv = jj < k ? iw[jj] : 0u;
          const bool leaf = ii < nl && (jj >= k || lv <= iv);
          m += leaf ? lv : iv;
          ii += leaf ? 1 : 0;
          jj += leaf ? 0 : 1;
        }
      }
      const int tL = warp_upper(lwt, i, nl, m, lane) - i;
      const int tI = warp_upper(iwt, j, k, m, lane) - j;
      const int t = tL + tI, P = t >> 1;
      // each of the t nodes' place in merge order: its index in its queue
      // plus the nodes of the other queue that go before it
      for (int r = lane; r < t; r += 32) {
        if (r < tL) {
          const uint32_t wv = lwt(i + r);
          int lo = j, hi = j + tI;  // internal nodes lighter than the leaf
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (iw[mid] < wv) lo = mid + 1;
            else hi = mid;
          }
          merged[r + lo - j] = (uint16_t)(i + r);
        } else {
          const int q = r - tL;
          const uint32_t wv = iw[j + q];
          int lo = i, hi = i + tL;  // leaves not heavier than the node
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (lwt(mid) <= wv) lo = mid + 1;
            else hi = mid;
          }
          merged[q + lo - i] = (uint16_t)(0x8000 | (j + q));
        }
      }
      __syncwarp();
      int cl = 0;  // leaves among the picked
      for (int q = lane; q < P; q += 32) {
        uint32_t sum = 0;
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int e = merged[2 * q + h];
          if (e & 0x8000) {
            sum += iw[e & 0x7FFF];
            par_int[e & 0x7FFF] = (uint16_t)(k + q);
          } else {
            sum += lwt(e);
            par_leaf[e] = (uint16_t)(k + q);
            cl++;
          }
        }
        iw[k + q] = sum;
      }
      cl = (int)__reduce_add_sync(0xffffffffu, (unsigned)cl);
      __syncwarp();
      i += cl;
      j += 2 * P - cl;
      k += P;
    }
  }
  __syncthreads();
  // depth of every internal node by pointer jumping (the root, node nl-2, has
  // depth 0); a leaf's depth is its parent's plus one
  {
    // the internal weights are no longer needed: iw holds the ancestors
    uint32_t* anc = iw;
    for (int k = tid; k < nl - 1; k += blockDim.x) {
      const bool root = k == nl - 2;
      dep[k] = root ? 0 : 1;
      anc[k] = root ? (uint32_t)k : (uint32_t)par_int[k];
    }
    __syncthreads();
    for (int round = 0; round < 12; round++) {  // 2^12 > 2047 nodes
      uint8_t nd[2];
      uint32_t na[2];
      int cnt = 0;
      for (int k = tid; k < nl - 1 && cnt < 2; k += blockDim.x, cnt++) {
        const uint32_t a1 = anc[k];
        nd[cnt] = (uint8_t)(dep[k] + dep[a1]);
        na[cnt] = anc[a1];
      }
      __syncthreads();
      cnt = 0;
      for (int k = tid; k < nl - 1 && cnt < 2; k += blockDim.x, cnt++) {
        dep[k] = nd[cnt];
        anc[k] = na[cnt];
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < nl; i += blockDim.x) atomicAdd(&bl[min(dep[par_leaf[i]] + 1, 63)], 1);
  __syncthreads();
  if (tid == 0) {
    int maxd = 0;
    for (int d = 1; d < 64; d++)
      if (bl[d]) maxd = d;
    // lengths above the limit: clamp, then remove the Kraft excess by moving
    // codes one length deeper, deepest lengths first
    if (maxd > kMaxCodeLen) {
      for (int L = maxd; L > kMaxCodeLen; L--) {
        bl[kMaxCodeLen] += bl[L];
        bl[L] = 0;
      }
      long long excess = -(1ll << kMaxCodeLen);
      for (int L = 1; L <= kMaxCodeLen; L++) excess += (long long)bl[L] << (kMaxCodeLen - L);
      for (int guard = 0; excess > 0 && guard < 4 * kMaxCodeLen; guard++) {
        int moved = 0;
        for (int L = kMaxCodeLen - 1; L >= 1 && excess > 0; L--) {
          const long long unit = 1ll << (kMaxCodeLen - L - 1);
          long long t = excess / unit;
          if (t > bl[L]) t = bl[L];
          bl[L] -= (int)t;
          bl[L + 1] += (int)t;
          excess -= t * unit;
          moved += t > 0;
        }
        if (excess > 0 && !moved) {
          int L = kMaxCodeLen - 1;
          while (L >= 1 && bl[L] == 0) L--;
          if (L < 1) break;
          bl[L] -= 1;
          bl[L + 1] += 1;
          excess -= 1ll << (kMaxCodeLen - L - 1);
        }
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
  // canonical order (length, symbol): rank of a symbol inside its length class
  // from ballots over the symbols in order; warp-group g covers symbols 32g..32g+31
  int myL[2], myr[2];
  for (int r = 0; r < 2; r++) {
    const int sym = r * kBookThreads + tid;
    const int L = len_of[sym];
    myL[r] = L;
    myr[r] = 0;
    for (int LL = 1; LL <= kMaxCodeLen; LL++) {
      const unsigned bm = __ballot_sync(0xffffffffu, L == LL);
      if (L == LL) myr[r] = __popc(bm & ((1u << lane) - 1u));
      if (lane == 0) wcnt[r * (kBookThreads / 32) + w][LL] = __popc(bm);
    }
  }
  __syncthreads();
  if (tid <= kMaxCodeLen && tid >= 1) {  // exclusive prefix over warp-groups, per length
    int run = 0;
    for (int gi = 0; gi < 2 * kBookThreads / 32; gi++) {
      const int c = wcnt[gi][tid];
      wcnt[gi][tid] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int r = 0; r < 2; r++) {
    const int sym = r * kBookThreads + tid;
    const int L = myL[r];
    if (L == 0) {
      e[sym] = 0;
      continue;
    }
    const int k = first_index[L] + wcnt[r * (kBookThreads / 32) + w][L] + myr[r];
    const uint32_t code = first_code[L] + (uint32_t)(k - first_index[L]);
    e[sym] = (uint16_t)((code << 4) | (uint32_t)L);
    bk->sym[k] = (uint16_t)sym;
    bk->len[k] = (uint8_t)L;
  }
  if (tid == 0) bk->nlive = (uint32_t)nl;
}

int launch_codebook(const Geo& g, const uint32_t* hist, uint16_t* enc, BookDev* books,
                    cudaStream_t s, int s0, int ns) {
  if (ns < 0) ns = g.nstreams - s0;
  if (s0 < 0 || s0 + ns > g.nstreams) return STZ_ERR_ARG;
  if (ns == 0) return STZ_OK;
  ProfScope ps_("k_codebook", s);
  k_codebook<<<ns, kBookThreads, 0, s>>>(hist, enc, books, s0);
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

// stream and symbol count of chunk j in 32-bit arithmetic (brick counts and
// extents of one stream fit in 32 bits)
__device__ __forceinline__ void chunk_sid_cnt(const Geo& g, int64_t j, int& sid, int& cnt) {
  sid = stream_of_chunk(g, j);
  const StreamGeo& sg = g.s[sid];
  const int jl = (int)(j - sg.chunk0);
  const int nb1 = (int)sg.nb[1], nb2 = (int)sg.nb[2];
  const int B0 = jl / (nb1 * nb2), r = jl - B0 * nb1 * nb2;
  const int B1 = r / nb2, B2 = r - B1 * nb2;
  cnt = min(g.b[0], (int)sg.e[0] - B0 * g.b[0]) * min(g.b[1], (int)sg.e[1] - B1 * g.b[1]) *
        min(g.b[2], (int)sg.e[2] - B2 * g.b[2]);
}

// Block-wide exclusive scan of one u32 per thread (256 threads).
__device__ __forceinline__ uint32_t block_scan_256(uint32_t v, uint32_t* wsum, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < 8 ? wsum[lane] : 0u;
    for (int o = 1; o < 8; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < 8) wsum[lane] = t;
  }
  __syncthreads();
  *total = wsum[7];
  return x - v + (w > 0 ? wsum[w - 1] : 0u);
}


// Up to 8 symbols [i, min(i + 8, end)) of a chunk: their encode entries
// (code << 4 | length; 0 past the end).  The tables (4 KiB per stream) are
// read through the read-only cache.
__device__ __forceinline__ void enc8(const uint16_t* __restrict__ c, int i, int end,
                                     const uint16_t* __restrict__ e, uint32_t (&ent)[8]) {
  if (i + 8 <= end) {
    const uint4 v = __ldg((const uint4*)(c + i));
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
      ent[2 * k] = __ldg(e + (u[k] & 0xFFFFu));
      ent[2 * k + 1] = __ldg(e + (u[k] >> 16));
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; k++) ent[k] = i + k < end ? (uint32_t)__ldg(e + __ldg(c + i + k)) : 0u;
  }
}

// One warp per chunk; lane l owns the chunk's symbols [64 l, 64 l + 64).
constexpr int kLaneSyms = 64;
static_assert(32 * kLaneSyms >= kBrick3D[0] * kBrick3D[1] * kBrick3D[2] &&
                  32 * kLaneSyms >= kBrick2D[0] * kBrick2D[1] * kBrick2D[2],
              "a warp covers a brick");

// Bits of the symbols [s0, s1) of a chunk.
__device__ __forceinline__ uint32_t run_bits(const uint16_t* __restrict__ c, int s0, int s1,
                                             const uint16_t* __restrict__ e) {
  uint32_t bits = 0;
  for (int i = s0; i < s1; i += 8) {
    uint32_t ent[8];
    enc8(c, i, s1, e, ent);
#pragma unroll
    for (int k = 0; k < 8; k++) bits += ent[k] & 15u;
  }
  return bits;
}

// Encode entries of the 8 symbols held in one 16-byte word of codes.
__device__ __forceinline__ void ent8(const uint4& v, const uint16_t* __restrict__ e,
                                     uint32_t (&ent)[8]) {
  const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int k = 0; k < 4; k++) {
    ent[2 * k] = __ldg(e + (u[k] & 0xFFFFu));
    ent[2 * k + 1] = __ldg(e + (u[k] >> 16));
  }
}

// Payload words per chunk, and the bits of each lane's run of 64 symbols
// (the packing pass's lane split).  A whole chunk is read with coalesced
// 16-byte loads, eight in flight per lane: load k gives lane t the symbols
// [8 (32 k + t), +8), which belong to lane run 4 k + t / 8; the eight lanes
// of a run add their bits by shuffle, and lane r collects run r's sum.
__global__ void __launch_bounds__(256) k_chunk_words(const __grid_constant__ Geo g,
                                                     const uint16_t* __restrict__ codes,
                                                     const uint16_t* __restrict__ enc,
                                                     uint32_t* __restrict__ words,
                                                     uint16_t* __restrict__ lane_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= g.total_chunks) return;
  int sid, cnt;
  chunk_sid_cnt(g, j, sid, cnt);
  const uint16_t* c = codes + j * g.bvol;
  const uint16_t* e = enc + (int64_t)sid * kAlphabet;
  uint32_t mine = 0;
  if (cnt == 32 * kLaneSyms) {
    const uint4* c4 = (const uint4*)c;
    uint4 v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = __ldg(c4 + 32 * k + lane);
#pragma unroll
    for (int k = 0; k < 8; k++) {
      uint32_t ent[8];
      ent8(v[k], e, ent);
      uint32_t b = 0;
#pragma unroll
      for (int m = 0; m < 8; m++) b += ent[m] & 15u;
      b += __shfl_xor_sync(0xffffffffu, b, 1);
      b += __shfl_xor_sync(0xffffffffu, b, 2);
      b += __shfl_xor_sync(0xffffffffu, b, 4);
      const uint32_t t = __shfl_sync(0xffffffffu, b, 8 * (lane & 3));
      if ((lane >> 2) == k) mine = t;
    }
  } else {
    const int s0 = lane * kLaneSyms, s1 = min(cnt, s0 + kLaneSyms);
    mine = run_bits(c, s0, s1, e);
  }
  lane_bits[j * 32 + lane] = (uint16_t)mine;
  uint32_t bits = mine;
  for (int o = 16; o > 0; o >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, o);
  if (lane == 0) words[j] = (bits + 31) >> 5;
}

int launch_chunk_words(const Geo& g, const uint16_t* codes, const uint16_t* enc, uint32_t* words,
                       uint16_t* lane_bits, cudaStream_t s) {
  if (g.total_chunks == 0) return STZ_OK;
  // a warp covers a chunk; 16-byte code loads need chunks on 16-byte bounds
  if (g.bvol > 32 * kLaneSyms || g.bvol % 8 != 0) return STZ_ERR_ARG;
  ProfScope ps_("k_chunk_words", s, 2.0 * (double)total_symbols(g));  // one read of the codes
  k_chunk_words<<<(unsigned)cdiv(g.total_chunks, 8), 256, 0, s>>>(g, codes, enc, words,
                                                                   lane_bits);
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
// Payload of every chunk.  One warp per chunk: each lane takes the bit count
// of its run of 64 symbols from the counting pass, a warp scan gives each
// lane its first bit, then each lane appends its codes, two at a time, to a
// 64-bit accumulator and stores the 32-bit words that fill.  A word that
// straddles two lanes' runs (only the first word of a lane whose run does not
// start on a word) is stored by the lane before, which ORs in the part the
// later lane hands it by shuffle.  Every lane but the chunk's last holds 64
// symbols, so at least 64 bits: only neighbouring lanes ever share a word.
// The lanes holding a sub-chunk start sum the lengths before it for the
// sub-chunk's bit offset.  A whole chunk is read with coalesced 16-byte loads
// and handed to the lanes through shared memory (16-byte units XOR-swizzled
// so that neither the writes nor the per-lane reads conflict); a lane with a
// whole run then works from registers, the outlier listing included.
template <typename T>
__global__ void __launch_bounds__(256) k_pack(const __grid_constant__ Geo g,
                                              const uint16_t* __restrict__ codes,
                                              const uint16_t* __restrict__ enc,
                                              const uint16_t* __restrict__ lane_bits,
                                              const unsigned long long* __restrict__ word_off,
                                              const SectDev* __restrict__ sect,
                                              uint8_t* __restrict__ out,
                                              const DevParams* __restrict__ dp,
                                              const T* __restrict__ field,
                                              const uint32_t* __restrict__ chunk_outliers,
                                              const unsigned long long* __restrict__ out_off) {
  if (dp->status & kStatCapacity) return;
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= g.total_chunks) return;
  int sid, cnt;
  chunk_sid_cnt(g, j, sid, cnt);
  const uint16_t* e = enc + (int64_t)sid * kAlphabet;
  const uint16_t* c = codes + j * g.bvol;
  const int s0 = lane * kLaneSyms, s1 = min(cnt, s0 + kLaneSyms);
  const bool whole = s1 - s0 == kLaneSyms;
  uint4 v[8];
  if (cnt == 32 * kLaneSyms) {  // every lane's run whole: coalesced, then transposed
    __shared__ uint4 stage[8][256];  // 4 KiB per warp
    uint4* st = stage[threadIdx.x >> 5];
    const uint4* c4 = (const uint4*)c;
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = __ldg(c4 + 32 * k + lane);
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int u = 32 * k + lane;
      st[u ^ ((u >> 3) & 7)] = v[k];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int u = 8 * lane + k;
      v[k] = st[u ^ ((u >> 3) & 7)];
    }
  } else if (whole) {
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = __ldg((const uint4*)(c + s0) + k);
  }
  const bool has_out = chunk_outliers[j] != 0;
  const uint32_t bits = lane_bits[j * 32 + lane];
  uint32_t incl = bits;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t p = incl - bits;  // first bit of this lane, from the chunk start
  const SectDev& sd = sect[sid];
  uint16_t* so =
      (uint16_t*)(out + sd.sect_off + sd.off_subs) + (j - g.s[sid].chunk0) * (kNSub - 1);
  uint32_t* dst = (uint32_t*)(out + sd.sect_off + sd.off_payload) + (word_off[j] - sd.word0);
  const int q = (cnt + kNSub - 1) / kNSub;
#pragma unroll
  for (int u = 1; u < kNSub; u++) {
    const int bnd = u * q;
    if (bnd >= cnt) {
      if (lane == 31) so[u - 1] = (uint16_t)incl;  // the chunk's total
    } else if (bnd >= s0 && bnd < s1) {
      so[u - 1] = (uint16_t)(p + run_bits(c, s0, bnd, e));
    }
  }
  uint32_t widx = p >> 5, nacc = p & 31u, first_part = 0;
  bool first_pending = nacc != 0;
  unsigned long long acc = 0;
  auto push8 = [&](const uint32_t (&ent)[8]) {
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      // two codes joined (at most 24 bits); past the end both are empty
      const uint32_t L1 = ent[k + 1] & 15u;
      const uint32_t L = (ent[k] & 15u) + L1;
      const uint32_t code = ((ent[k] >> 4) << L1) | (ent[k + 1] >> 4);
      acc = (acc << L) | code;
      nacc += L;  // below 32 + 24: at most one word fills
      if (nacc >= 32) {
        nacc -= 32;
        const uint32_t w = (uint32_t)(acc >> nacc);
        if (first_pending) {
          first_part = w;
          first_pending = false;
        } else {
          dst[widx] = w;
        }
        widx++;
      }
    }
  };
  unsigned long long zmask = 0;  // symbols 0 (outliers) of a whole run
  if (whole) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      uint32_t ent[8];
      ent8(v[k], e, ent);
      push8(ent);
      if (has_out) {
        const uint32_t u[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
        for (int h = 0; h < 4; h++) {
          if ((u[h] & 0xFFFFu) == 0u) zmask |= 1ull << (8 * k + 2 * h);
          if ((u[h] >> 16) == 0u) zmask |= 1ull << (8 * k + 2 * h + 1);
        }
      }
    }
  } else {
    for (int i = s0; i < s1; i += 8) {
      uint32_t ent[8];
      enc8(c, i, s1, e, ent);
      push8(ent);
    }
  }
  bool has_last = nacc > 0 && s1 > s0;
  const uint32_t last = has_last ? (uint32_t)(acc << (32u - nacc)) : 0u;
  if (has_last && first_pending) {  // the lane's whole run lies in its first word
    first_part = last;
    has_last = false;
  }
  uint32_t from_next = __shfl_down_sync(0xffffffffu, first_part, 1);
  if (lane == 31) from_next = 0;
  if (has_last) dst[widx] = last | from_next;
  // the chunk's outliers (symbol 0): stream position and raw value, in stream
  // order from the chunk's offset in the stream's outlier list
  if (!has_out) return;
  uint32_t nz = 0;
  if (whole) {
    nz = (uint32_t)__popcll(zmask);
  } else {
    for (int i = s0; i < s1; i++) nz += __ldg(c + i) == 0;
  }
  uint32_t zincl = nz;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, zincl, o);
    if (lane >= o) zincl += y;
  }
  if (nz == 0) return;
  const StreamGeo& sg = g.s[sid];
  int64_t B[3], l[3], start;
  chunk_brick(sg, g.b, j - sg.chunk0, B, l, &start);
  const int64_t st = level_stride(g.L, sg.level);
  uint32_t* opos = (uint32_t*)(out + sd.sect_off + sd.off_opos);
  T* oval = (T*)(out + sd.sect_off + sd.off_oval);
  unsigned long long k = out_off[j] - sd.out0 + (zincl - nz);
  auto list = [&](int i) {
    const int64_t lz = i / (l[1] * l[2]), ly = (i / l[2]) % l[1], lx = i % l[2];
    int64_t pt[3] = {B[0] * g.b[0] + lz, B[1] * g.b[1] + ly, B[2] * g.b[2] + lx};
    if (sg.level > 1)
      for (int a = 0; a < 3; a++) pt[a] = 2 * pt[a] + sg.o[a];
    opos[k] = (uint32_t)(start + i);
    oval[k] = field[((pt[0] * st) * g.n[1] + pt[1] * st) * g.n[2] + pt[2] * st];
    k++;
  };
  if (whole) {
    while (zmask) {
      list(s0 + __ffsll((long long)zmask) - 1);
      zmask &= zmask - 1;
    }
  } else {
    for (int i = s0; i < s1; i++)
      if (__ldg(c + i) == 0) list(i);
  }
}

int launch_pack(const Geo& g, const uint16_t* codes, const uint16_t* enc,
                const uint16_t* lane_bits, const unsigned long long* word_off,
                const SectDev* sect, uint8_t* out, const DevParams* dp, const void* field,
                const uint32_t* chunk_outliers, const unsigned long long* out_off,
                cudaStream_t s) {
  if (g.total_chunks == 0) return STZ_OK;
  if (g.bvol > 32 * kLaneSyms || g.bvol % 8 != 0) return STZ_ERR_ARG;
  const unsigned grid = (unsigned)cdiv(g.total_chunks, 8);
  // reads the codes; the payload it writes is added once its size is known
  ProfScope ps_("k_pack", s, 2.0 * (double)total_symbols(g));
  if (g.dtype == STZ_F32)
    k_pack<float><<<grid, 256, 0, s>>>(g, codes, enc, lane_bits, word_off, sect, out, dp,
                                       (const float*)field, chunk_outliers, out_off);
  else
    k_pack<double><<<grid, 256, 0, s>>>(g, codes, enc, lane_bits, word_off, sect, out, dp,
                                        (const double*)field, chunk_outliers, out_off);
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------- decode tables
// Block 0 also clears the decode's parameter words (its status among them).
// A table that cannot be built is left empty: every lookup then fails, so the
// decode of any chunk of that stream reports the container corrupt.
// Decode table of a stream: one 32-bit entry per 12-bit window, holding the
// first code that starts the window and, when the second code also ends
// inside it, that one too:
//   bits  0-10 first symbol,  bits 11-14 its length (0: no code starts so)
//   bits 16-26 second symbol, bits 27-30 its length (0: not inside the window)
// so that (entry & 0x07FF07FF) is the two symbols as a pair of u16.
// kLutParts blocks per stream, each filling an equal share of the windows
constexpr int kLutParts = 8;
static_assert(kLutSize % (kLutParts * 256) == 0, "a block fills whole rounds of windows");
__global__ void __launch_bounds__(256) k_lut(const __grid_constant__ DecTables tb,
                                             uint32_t* __restrict__ lut,
                                             uint32_t* __restrict__ clear, int nclear) {
  __shared__ int cnt[32];
  __shared__ uint32_t fcode[32];
  __shared__ int fidx[32];
  __shared__ int start[32];  // first codebook entry of each length, -1: none
  __shared__ int bad;
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < nclear; i += blockDim.x) clear[i] = 0u;
  const int sid = tb.lut_sid[blockIdx.x / kLutParts];
  const int part = blockIdx.x % kLutParts;  // this block's share of the windows
  const DecStream& d = tb.ds[sid];
  uint32_t* t = lut + (int64_t)sid * kLutSize;
  const int tid = threadIdx.x;
  if (tid < 32) start[tid] = -1;
  if (tid == 0) bad = 0;
  __syncthreads();
  const uint16_t* syms = (const uint16_t*)(d.sect + d.off_syms);
  const uint8_t* lens = d.sect + d.off_lens;
  const int nlive = d.nlive > (uint64_t)kAlphabet ? kAlphabet : (int)d.nlive;
  if (d.nlive > (uint64_t)kAlphabet && tid == 0) bad = 1;
  // the codebook lists (symbol, length) by (length, symbol): each length's
  // entries are one run, found from where the length changes
  for (int k = tid; k < nlive; k += blockDim.x) {
    const int L = lens[k], sym = syms[k];
    if (L < 1 || L > kMaxCodeLen || sym >= kAlphabet) {
      bad = 1;
      continue;
    }
    const int Lp = k > 0 ? lens[k - 1] : 0, sp = k > 0 ? syms[k - 1] : -1;
    if (!(L > Lp || (L == Lp && sym > sp))) bad = 1;
    else if (L != Lp) start[L] = k;
  }
  __syncthreads();
  if (tid == 0 && !bad) {
    int next = nlive;  // start of the next longer length present
    for (int L = kMaxCodeLen; L >= 1; L--) {
      cnt[L] = start[L] < 0 ? 0 : next - start[L];
      if (start[L] >= 0) next = start[L];
    }
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
  constexpr int kPart = kLutSize / kLutParts;
  if (bad) {  // an empty table: every lookup then flags the chunk as corrupt
    for (int i = part * kPart + tid; i < (part + 1) * kPart; i += blockDim.x) t[i] = 0;
    return;
  }
  // the code that starts window w (its top bits; only lengths <= maxlen
  // count): symbol | length << 11, or 0 when none does.  A code of length L
  // starts w when the L-bit prefix of w falls in length L's range of
  // canonical codes.
  auto first = [&](uint32_t w, int maxlen) -> uint32_t {
    for (int L = 1; L <= maxlen; L++) {
      const uint32_t r = (w >> (kMaxCodeLen - L)) - fcode[L];
      if (r < (uint32_t)cnt[L]) return (uint32_t)syms[fidx[L] + (int)r] | ((uint32_t)L << 11);
    }
    return 0u;
  };
  for (int i = part * kPart + tid; i < (part + 1) * kPart; i += blockDim.x) {
    const uint32_t e0 = first((uint32_t)i, kMaxCodeLen);
    const int L0 = (int)(e0 >> 11);
    uint32_t e1 = 0;
    if (L0 > 0 && L0 < kMaxCodeLen)  // the window's remaining 12 - L0 bits
      e1 = first(((uint32_t)i << L0) & (kLutSize - 1), kMaxCodeLen - L0);
    t[i] = e0 | (e1 << 16);
  }
}

int launch_lut(const DecTables& tb, uint32_t* lut, uint32_t* clear, int nclear,
               cudaStream_t s) {
  if (tb.nlut == 0) return STZ_ERR_ARG;
  ProfScope ps_("k_lut", s);
  k_lut<<<tb.nlut * kLutParts, 256, 0, s>>>(tb, lut, clear, nclear);
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------- chunk decode
// A chunk of n symbols is cut into nsub runs of q = ceil(n / nsub) symbols
// whose start bits are stored, so every run decodes independently: one
// thread per run, kDecThreads / nsub consecutive chunks of a job per block.
// The block first copies its chunks' payload words into shared memory
// (coalesced, two zero words after each chunk), in rounds of at most
// kStageWords words when they do not fit at once, so the decode loop reads
// only shared memory: a 32-bit window at bit `pos` of the word pair
// (cur, nxt), looked up in the 16-bit table.  A run that does not end exactly
// where the next one starts, reads past its chunk, or meets an invalid code
// marks the container corrupt (its chunk's codes are then unspecified).
// 4-byte asynchronous copy global -> shared (Ampere+ cp.async), and the wait
// for all of this thread's copies
__device__ __forceinline__ void cp_async4(uint32_t* dst_smem, const uint32_t* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Blocks of the chunk decoder per SM, and the payload words a block stages
// at once: beside the 16 KiB decode table, 5 blocks per SM leave room for a
// 24 KiB stage (8 runs per chunk, 32 chunks per block: 3 bits per symbol at
// once); 6 blocks would leave 16.9 KiB (measured slower: more staging rounds)
#ifndef STZ_DEC_BLOCKS
#define STZ_DEC_BLOCKS 5
#endif
constexpr int kDecBlocks = STZ_DEC_BLOCKS;
constexpr int kStageWords = kDecBlocks >= 6 ? 4320 : 6144;
constexpr int kMaxChunkWords = (4096 * kMaxCodeLen + 31) / 32;  // bricks hold <= 4096 cells
static_assert(kMaxChunkWords + 2 <= kStageWords, "a chunk must fit the stage");
// A launch of at most one block per SM (a level-1 stream, a small region)
// has the SM's shared memory to itself: its blocks stage 64 KiB of payload,
// so that a level-1 block's 32 chunks (about 3.6 bits per symbol) arrive in
// one round instead of two, halving the serial decode chains that round
// after round would otherwise run one after the other.
constexpr int kBigStageWords = 16384;
__host__ __device__ constexpr size_t dec_smem(int stage_words) {
  return sizeof(uint32_t) * stage_words + sizeof(uint32_t) * kLutSize +
         sizeof(uint32_t) * kDecThreads + sizeof(uint32_t) * (kDecThreads + 1) +
         sizeof(uint32_t) * kDecThreads + sizeof(int) * kDecThreads;
}
constexpr size_t kDecSmem = dec_smem(kStageWords);
static_assert((sizeof(uint32_t) * kStageWords) % 16 == 0 &&
                  (sizeof(uint32_t) * kStageWords + sizeof(uint32_t) * kLutSize) % 16 == 0,
              "shared arrays of the chunk decoder must stay aligned");

// first index i in the ascending list p[0, n) with p[i] >= v
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ p, int64_t n,
                                                    int64_t v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)__ldg(p + mid) < v) lo = mid + 1;
    else hi = mid;
  }
  return (uint32_t)lo;
}

// One block's share of a chunk job: chunks [bidx * cpb, ...) of the job's
// brick range of one stream.  lutg: the stream's decode table.
__device__ __forceinline__ void decode_block(const DecChunkJob& job, const DecStream& d,
                                             const StreamGeo& sg, const int32_t gb[3],
                                             int64_t bvol, const uint32_t* __restrict__ lutg,
                                             uint16_t* __restrict__ codes,
                                             uint32_t* __restrict__ sub_olo,
                                             uint32_t* __restrict__ status, int64_t bidx,
                                             int stage_words) {
  extern __shared__ __align__(16) unsigned char dsm[];
  // arrays in order of alignment: the 16-byte-loaded table first, then 4-byte
  uint32_t* stage = (uint32_t*)dsm;
  uint32_t* t = stage + stage_words;
  uint32_t* cw0 = (uint32_t*)(t + kLutSize);     // chunk's first word in the stream payload
  uint32_t* S = cw0 + kDecThreads;               // padded-size prefix sums
  uint32_t* cjl = S + kDecThreads + 1;                            // chunk index in stream
  int* ccnt = (int*)(cjl + kDecThreads);                          // symbols; -1: bad chunk
  __shared__ uint32_t wsum[8];
  const int tid = threadIdx.x;
  {
    const uint4* src = (const uint4*)lutg;
    for (int i = tid; i < kLutSize / 4; i += blockDim.x) ((uint4*)t)[i] = __ldg(src + i);
  }
  const int nsub = d.nsub;
  const int cpb = kDecThreads / nsub;  // chunks per block
  const int64_t qb = bidx * cpb;
  const int nch = (int)min((int64_t)cpb, job.nchunks_job - qb);
  const uint32_t* coff = (const uint32_t*)(d.sect + d.off_chunks);
  const uint32_t* pay = (const uint32_t*)(d.sect + d.off_payload);
  // the block's chunks: index in the stream, symbols, payload words
  uint32_t psz = 0;
  if (tid < nch) {
    const int q32 = (int)(qb + tid), c1 = (int)job.cnt[1], c2 = (int)job.cnt[2];
    const int r0 = q32 / (c1 * c2), rr = q32 - r0 * c1 * c2, r1 = rr / c2, r2 = rr - r1 * c2;
    const int B0 = (int)job.lo[0] + r0, B1 = (int)job.lo[1] + r1, B2 = (int)job.lo[2] + r2;
    const int64_t jl = ((int64_t)B0 * sg.nb[1] + B1) * sg.nb[2] + B2;
    const int cnt = min(gb[0], (int)sg.e[0] - B0 * gb[0]) *
                    min(gb[1], (int)sg.e[1] - B1 * gb[1]) *
                    min(gb[2], (int)sg.e[2] - B2 * gb[2]);
    const uint64_t w0 = coff[jl];
    const uint64_t w1 = jl + 1 < (int64_t)d.nchunks ? coff[jl + 1] : d.pw;
    const bool ok = w0 <= w1 && w1 <= d.pw && w1 - w0 <= (uint64_t)kMaxChunkWords;
    cw0[tid] = w0;
    cjl[tid] = (uint32_t)jl;
    ccnt[tid] = ok ? cnt : -1;
    psz = ok ? (uint32_t)(w1 - w0) + 2u : 0u;
  }
  uint32_t total;
  const uint32_t excl = block_scan_256(psz, wsum, &total);
  if (tid < nch) S[tid] = excl;
  if (tid == 0) S[nch] = total;
  // this thread's run
  const int c = tid / nsub, u = tid - c * nsub;
  bool bad = false;
  int a = 0;
  while (a < nch) {
    __syncthreads();
    const uint32_t base = S[a];
    const int b = a + __syncthreads_count(tid >= a && tid < nch && S[tid + 1] - base <= (uint32_t)stage_words);
    {
      // copy chunks [a, b): one warp per chunk, lanes over its words, every
      // copy asynchronous (none waits for the one before), then one wait
      const int lane = tid & 31;
      for (int cc = a + (tid >> 5); cc < b; cc += kDecThreads / 32) {
        const uint32_t len = S[cc + 1] - S[cc];
        uint32_t* dst = stage + (S[cc] - base);
        const uint32_t* src = pay + cw0[cc];
        for (uint32_t k = lane; k < len; k += 32) {
          if (k + 2 < len) cp_async4(dst + k, src + k);
          else dst[k] = 0u;
        }
      }
      cp_async_wait_all();
    }
    __syncthreads();
    if (c >= a && c < b) {
      const int cnt = ccnt[c];
      const int per = (max(cnt, 0) + nsub - 1) / nsub;
      const int i0 = min(max(cnt, 0), u * per), i1 = min(max(cnt, 0), (u + 1) * per);
      uint16_t* out = codes + (job.slot_base + qb + c) * bvol;
      const uint32_t words = S[c + 1] - S[c] - 2;  // garbage when the chunk is bad (unused)
      const uint64_t cbits = (uint64_t)words * 32;
      const uint16_t* soff = (const uint16_t*)(d.sect + d.off_subs) + (int64_t)cjl[c] * (nsub - 1);
      const uint32_t b0 = u == 0 ? 0u : soff[u - 1];
      const uint64_t b1 = u + 1 < nsub ? (uint64_t)soff[u] : cbits;
      if (cnt < 0 || b0 > b1 || b1 > cbits) {
        bad = true;
        for (int i = i0; i < i1; i++) out[i] = 0;
      } else {
        const uint32_t* sp = stage + (S[c] - base);
        const int lim = (int)words + 1;  // last staged (pad) word of the chunk
        int k = (int)(b0 >> 5);
        int pos = (int)(b0 & 31);
        uint32_t cur = sp[k], nxt = sp[k + 1];
        // the smallest entry met: below 1 << 11 once a window starts no code
        // (every valid entry has its first length, >= 1, at bit 11; an
        // invalid window stops the position)
        uint32_t mn = 0xFFFFFFFFu;
        // nbits <= 24 and pos < 32, so at most one word is crossed; the step
        // is written without a branch (the next word's load is predicated)
        auto advance = [&](uint32_t nbits) {
          pos += (int)nbits;
          const int carry = pos >> 5;
          pos &= 31;
          cur = carry ? nxt : cur;
          k += carry;
          bad |= k >= lim;  // past the chunk's payload and first pad word
          k = min(k, lim - 1);
          if (carry) nxt = sp[k + 1];
        };
        // the next two symbols as a u16 pair: one lookup, and a second one
        // only when the second code does not end inside the first window
        auto next2 = [&]() -> uint32_t {
          const uint32_t win = __funnelshift_l(nxt, cur, pos);
          const uint32_t e = t[win >> (32 - kMaxCodeLen)];
          const uint32_t L0 = (e >> 11) & 15u;
          uint32_t L1 = e >> 27;
          uint32_t pair = e & 0x07FF07FFu;
          mn = min(mn, e);
          if (L1 == 0u) {
            const uint32_t e1 = t[(win << L0) >> (32 - kMaxCodeLen)];
            L1 = (e1 >> 11) & 15u;
            mn = min(mn, e1 & 0xFFFFu);
            pair = (pair & 0x7FFu) | ((e1 & 0x7FFu) << 16);
          }
          advance(L0 + L1);
          return pair;
        };
        auto next1 = [&]() -> uint32_t {
          const uint32_t win = __funnelshift_l(nxt, cur, pos);
          const uint32_t e = t[win >> (32 - kMaxCodeLen)];
          mn = min(mn, e & 0xFFFFu);
          advance((e >> 11) & 15u);
          return e & 0x7FFu;
        };
        int i = i0;
        // 8 symbols per 16-byte store where the run start is 16-byte aligned
        if ((((uintptr_t)(out + i)) & 15) == 0) {
          for (; i + 8 <= i1; i += 8) {
            uint32_t v[4];
#pragma unroll
            for (int m = 0; m < 4; m++) v[m] = next2();
            *(uint4*)(out + i) = make_uint4(v[0], v[1], v[2], v[3]);
          }
        }
        for (; i < i1; i++) out[i] = (uint16_t)next1();
        bad |= mn < (1u << 11);
        const uint64_t end = (uint64_t)k * 32 + (uint64_t)pos;
        bad |= u + 1 < nsub ? end != b1 : end > b1;
      }
    }
    a = b;
  }
  // where this sub-chunk's outliers start in the stream's outlier list (the
  // list is ascending by stream position and a chunk's positions are
  // contiguous): one search per sub-chunk here instead of one per outlier in
  // the predictors
  if (d.dense && c < nch) {
    const uint32_t* opos = (const uint32_t*)(d.sect + d.off_opos);
    const int64_t jl = cjl[c];
    const int64_t B0 = jl / (sg.nb[1] * sg.nb[2]), B1 = (jl / sg.nb[2]) % sg.nb[1],
                  B2 = jl % sg.nb[2];
    const int64_t l0 = imin(gb[0], sg.e[0] - B0 * gb[0]);
    const int64_t l1 = imin(gb[1], sg.e[1] - B1 * gb[1]);
    const int64_t l2 = imin(gb[2], sg.e[2] - B2 * gb[2]);
    const int64_t start = B0 * gb[0] * sg.e[1] * sg.e[2] + B1 * gb[1] * l0 * sg.e[2] +
                          B2 * gb[2] * l0 * l1;
    const int cntc = (int)(l0 * l1 * l2);
    const int per = (cntc + nsub - 1) / nsub;
    uint32_t* dst = sub_olo + (job.slot_base + qb + c) * (kNSub + 1);
    const int64_t n = (int64_t)d.nout;
    dst[u] = lower_bound_u32(opos, n, start + min(u * per, cntc));
    if (u == nsub - 1) dst[nsub] = lower_bound_u32(opos, n, start + cntc);
  }
  if (bad) atomicOr(status, kStatCorrupt);
}

__global__ void __launch_bounds__(kDecThreads, kDecBlocks) k_decode_chunks(
    const __grid_constant__ Geo g, const __grid_constant__ DecTables tb,
    const uint32_t* __restrict__ lut, uint16_t* __restrict__ codes,
    uint32_t* __restrict__ sub_olo, uint32_t* __restrict__ status, int stage_words) {
  // virtual blocks of 32 chunks, the grid striding over them (a grid smaller
  // than the work leaves SMs to kernels running beside it)
  for (int64_t vb = blockIdx.x; vb < tb.nblocks; vb += gridDim.x) {
    if (vb != (int64_t)blockIdx.x) __syncthreads();  // the shared stage and table are reused
    int jb = 0;
    for (int k = 1; k < tb.njobs; k++)
      if (tb.jobs[k].block0 <= vb) jb = k;
    const DecChunkJob& job = tb.jobs[jb];
    const int sid = job.sid;
    decode_block(job, tb.ds[sid], g.s[sid], g.b, g.bvol, lut + (int64_t)sid * kLutSize, codes,
                 sub_olo, status, vb - job.block0, stage_words);
  }
}

// The chunk jobs of many region decodes in one launch (the batched served
// form): each job carries its own stream, decode table and outputs.
__global__ void __launch_bounds__(kDecThreads, kDecBlocks) k_decode_chunks_multi(
    const DecJobMulti* __restrict__ jobs, int njobs) {
  int lo = 0, hi = njobs - 1;  // the last job whose first block is <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].job.block0 <= (int64_t)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const DecJobMulti& m = jobs[lo];
  decode_block(m.job, m.ds, m.sg, m.b, m.bvol, m.lut, m.codes, m.sub_olo, m.status,
               (int64_t)blockIdx.x - m.job.block0, kStageWords);
}

int launch_decode_chunks_multi(const DecJobMulti* jobs_dev, int njobs, int64_t nblocks,
                               double bytes, cudaStream_t s) {
  if (nblocks == 0 || njobs == 0) return STZ_OK;
  if (allow_smem((const void*)k_decode_chunks_multi, kDecSmem) != STZ_OK)
    return STZ_ERR_CUDA;
  ProfScope ps_("k_decode_chunks", s, bytes);
  k_decode_chunks_multi<<<(unsigned)nblocks, kDecThreads, kDecSmem, s>>>(jobs_dev, njobs);
  return cuda_ok(cudaGetLastError());
}

int launch_decode_chunks(const Geo& g, const DecTables& tb, const uint32_t* lut,
                         uint16_t* codes, uint32_t* sub_olo, uint32_t* status, double bytes,
                         cudaStream_t s, int64_t max_grid) {
  if (tb.nblocks == 0) return STZ_OK;
  static_assert(kDecThreads == 256, "block_scan_256 assumes 256 threads");
  const int64_t grid = max_grid > 0 ? imin(tb.nblocks, max_grid) : tb.nblocks;
  // a launch of at most one block per SM takes the big stage
  const int stage = grid <= (int64_t)launch_sms() ? kBigStageWords : kStageWords;
  const size_t smem = dec_smem(stage);
  if (allow_smem((const void*)k_decode_chunks, smem) != STZ_OK) return STZ_ERR_CUDA;
  ProfScope ps_("k_decode_chunks", s, bytes);
  k_decode_chunks<<<(unsigned)grid, kDecThreads, smem, s>>>(g, tb, lut, codes, sub_olo, status,
                                                            stage);
  return cuda_ok(cudaGetLastError());
}

int decode_blocks_per_sm() { return kDecBlocks; }

}  // namespace stz
