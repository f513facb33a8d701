// stz_container.cu -- the self-describing byte container, written in place
// on the device once the sizes are known (no assembly copy).
//
// Layout (little-endian): a 256-byte header, a 48-byte directory entry per
// stream, then per stream an 8-byte aligned section: canonical codebook
// (u16 symbols, u8 lengths), u32 word offset of each chunk, the u32 payload
// words, u32 outlier positions (ascending stream positions) and the raw
// outlier values in the field's type.
#include "stz_kernels.cuh"
#include "stz_prof.cuh"

namespace stz {

__device__ __forceinline__ unsigned long long al4(unsigned long long v) { return (v + 3) & ~3ull; }
__device__ __forceinline__ unsigned long long al8(unsigned long long v) { return (v + 7) & ~7ull; }

__device__ __forceinline__ void put_u16(uint8_t* p, uint32_t v) {
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
}
__device__ __forceinline__ void put_u32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
__device__ __forceinline__ void put_u64(uint8_t* p, unsigned long long v) {
  for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
__device__ __forceinline__ void put_f64(uint8_t* p, double v) {
  put_u64(p, (unsigned long long)__double_as_longlong(v));
}

// One thread per stream lays out its section; the section offsets are the
// prefix sums of the sizes.  64 threads cover kMaxStreams.
constexpr int kLayoutThreads = 64;
static_assert(kMaxStreams <= kLayoutThreads, "one thread per stream");

__global__ void __launch_bounds__(kLayoutThreads) k_layout(
    const __grid_constant__ Geo g, const DevParams* __restrict__ dp, int eb_mode,
    const unsigned long long* __restrict__ word_off,
    const unsigned long long* __restrict__ out_off, const BookDev* __restrict__ books,
    LayoutDev* __restrict__ lay, uint8_t* __restrict__ out, unsigned long long cap) {
  __shared__ unsigned long long size[kLayoutThreads];
  const int t = threadIdx.x;
  const unsigned long long ps = g.dtype == STZ_F32 ? 4 : 8;
  SectDev d;
  if (t < g.nstreams) {
    const StreamGeo& sg = g.s[t];
    const unsigned long long nch = (unsigned long long)sg.nchunks;
    d.word0 = word_off[sg.chunk0];
    d.out0 = out_off[sg.chunk0];
    d.pw = word_off[sg.chunk0 + sg.nchunks] - d.word0;
    d.nout = out_off[sg.chunk0 + sg.nchunks] - d.out0;
    d.nlive = books[t].nlive;
    d.off_syms = 0;
    d.off_lens = 2 * d.nlive;
    d.off_chunks = al4(3 * d.nlive);
    d.off_subs = d.off_chunks + 4 * nch;
    d.off_payload = al4(d.off_subs + 2 * nch * (kNSub - 1));
    d.off_opos = d.off_payload + 4 * d.pw;
    d.off_oval = al8(d.off_opos + 4 * d.nout);
    d.size = al8(d.off_oval + ps * d.nout);
    size[t] = d.size;
  }
  __syncthreads();
  const unsigned long long dir_end =
      kHeaderBytes + (unsigned long long)g.nstreams * kDirEntryBytes;
  unsigned long long off = dir_end, total = dir_end;
  for (int k = 0; k < g.nstreams; k++) {
    off += k < t ? size[k] : 0ull;
    total += size[k];
  }
  if (t < g.nstreams) {
    d.sect_off = off;
    lay->s[t] = d;
  }
  if (t == 0) lay->total = total;
  if (total > cap) {
    if (t == 0) atomicOr((uint32_t*)&dp->status, kStatCapacity);
    return;
  }
  if (t < g.nstreams) {
    uint8_t* e = out + kHeaderBytes + (size_t)t * kDirEntryBytes;
    put_u64(e + 0, d.sect_off);
    put_u64(e + 8, (unsigned long long)g.s[t].nsym);
    put_u32(e + 16, (uint32_t)g.s[t].nchunks);
    put_u32(e + 20, (uint32_t)d.nlive);
    put_u64(e + 24, d.pw);
    put_u64(e + 32, d.nout);
    put_u64(e + 40, 0);
  }
  for (int i = t; i < kHeaderBytes; i += kLayoutThreads) out[i] = 0;
  __syncthreads();
  if (t != 0) return;
  out[0] = 'S';
  out[1] = 'T';
  out[2] = 'Z';
  out[3] = '1';
  put_u16(out + 4, 1);
  out[6] = (uint8_t)g.dtype;
  out[7] = (uint8_t)g.ndim;
  out[8] = (uint8_t)g.L;
  out[9] = (uint8_t)eb_mode;
  out[10] = (uint8_t)kMaxCodeLen;
  out[11] = (uint8_t)kNSub;
  put_u32(out + 12, kRadius);
  for (int a = 0; a < 3; a++) put_u32(out + 16 + 4 * a, (uint32_t)g.b[a]);
  put_u32(out + 28, (uint32_t)g.nstreams);
  for (int a = 0; a < 3; a++) put_u64(out + 32 + 8 * a, (unsigned long long)g.n[a]);
  put_f64(out + 56, dp->eb);
  put_f64(out + 64, dp->eb_abs);
  put_f64(out + 72, dp->vmin);
  put_f64(out + 80, dp->vmax);
  put_u64(out + 88, total);
  for (int l = 1; l <= g.L; l++) {
    put_f64(out + 96 + 8 * (l - 1), dp->eb_level[l]);
    put_f64(out + 144 + 8 * (l - 1), dp->two_eb_d[l]);
  }
  put_f64(out + 192, dp->eb_ratio);
  out[200] = (uint8_t)dp->pred;
}

int launch_layout(const Geo& g, const DevParams* dp, int eb_mode,
                  const unsigned long long* word_off, const unsigned long long* out_off,
                  const BookDev* books, LayoutDev* lay, uint8_t* out, size_t cap,
                  cudaStream_t s) {
  ProfScope ps_("k_layout", s);
  k_layout<<<1, kLayoutThreads, 0, s>>>(g, dp, eb_mode, word_off, out_off, books, lay, out,
                                        (unsigned long long)cap);
  return cuda_ok(cudaGetLastError());
}

// Codebooks, padding and chunk word offsets of every stream.
__global__ void __launch_bounds__(256) k_sections(const __grid_constant__ Geo g,
                                                  const LayoutDev* __restrict__ lay,
                                                  const BookDev* __restrict__ books,
                                                  const unsigned long long* __restrict__ word_off,
                                                  const DevParams* __restrict__ dp,
                                                  uint8_t* __restrict__ out) {
  if (dp->status & kStatCapacity) return;
  const unsigned long long ps = g.dtype == STZ_F32 ? 4 : 8;
  if ((int)blockIdx.x < g.nstreams) {
    const int s = blockIdx.x;
    const SectDev& d = lay->s[s];
    uint8_t* sec = out + d.sect_off;
    const BookDev& bk = books[s];
    for (unsigned long long k = threadIdx.x; k < d.nlive; k += blockDim.x) {
      put_u16(sec + d.off_syms + 2 * k, bk.sym[k]);
      sec[d.off_lens + k] = bk.len[k];
    }
    if (threadIdx.x == 0) {
      for (unsigned long long p = d.off_lens + d.nlive; p < d.off_chunks; p++) sec[p] = 0;
      const unsigned long long sub_end =
          d.off_subs + 2ull * (unsigned long long)g.s[s].nchunks * (kNSub - 1);
      for (unsigned long long p = sub_end; p < d.off_payload; p++) sec[p] = 0;
      for (unsigned long long p = d.off_opos + 4 * d.nout; p < d.off_oval; p++) sec[p] = 0;
      for (unsigned long long p = d.off_oval + ps * d.nout; p < d.size; p++) sec[p] = 0;
    }
  }
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < g.total_chunks; j += nth) {
    int sid = 0;
    for (int s = 1; s < g.nstreams; s++)
      if (g.s[s].nchunks > 0 && g.s[s].chunk0 <= j) sid = s;
    const SectDev& d = lay->s[sid];
    uint32_t* co = (uint32_t*)(out + d.sect_off + d.off_chunks);
    co[j - g.s[sid].chunk0] = (uint32_t)(word_off[j] - d.word0);
  }
}

int launch_sections(const Geo& g, const LayoutDev* lay, const BookDev* books,
                    const unsigned long long* word_off, const DevParams* dp, uint8_t* out,
                    cudaStream_t s) {
  int64_t blocks = imax(g.nstreams, imin(cdiv(g.total_chunks, 256), 1024));
  ProfScope ps_("k_sections", s);
  k_sections<<<(unsigned)blocks, 256, 0, s>>>(g, lay, books, word_off, dp, out);
  return cuda_ok(cudaGetLastError());
}

}  // namespace stz
