// stz_api.cu -- the C ABI (include/stz.h): argument checks, workspace
// planning, container header parsing and launch sequencing.  Every step of
// the method runs in the kernels of the other translation units.
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "stz_kernels.cuh"
#include "stz_prof.cuh"

namespace stz {

void make_geo(const int64_t n[3], int ndim, int dtype, int L, const int b[3], Geo* g) {
  memset(g, 0, sizeof(*g));
  for (int a = 0; a < 3; a++) {
    g->n[a] = n[a];
    g->b[a] = b[a];
  }
  g->L = L;
  g->ndim = ndim;
  g->dtype = dtype;
  g->nstreams = 1 + 7 * (L - 1);
  g->bvol = (int64_t)b[0] * b[1] * b[2];
  int64_t chunk0 = 0;
  for (int s = 0; s < g->nstreams; s++) {
    StreamGeo& sg = g->s[s];
    if (s == 0) {
      sg.level = 1;
      grid_extent(n, L, 1, sg.e);
      sg.o[0] = sg.o[1] = sg.o[2] = 0;
    } else {
      const int l = 2 + (s - 1) / 7, k = 1 + (s - 1) % 7;
      sg.level = l;
      sg.o[0] = (k >> 2) & 1;
      sg.o[1] = (k >> 1) & 1;
      sg.o[2] = k & 1;
      int64_t m[3];
      grid_extent(n, L, l, m);
      for (int a = 0; a < 3; a++) sg.e[a] = m[a] >= sg.o[a] ? (m[a] - sg.o[a] + 1) / 2 : 0;
    }
    sg.nsym = sg.e[0] * sg.e[1] * sg.e[2];
    for (int a = 0; a < 3; a++) sg.nb[a] = sg.e[a] > 0 ? cdiv(sg.e[a], b[a]) : 0;
    sg.nchunks = sg.nb[0] * sg.nb[1] * sg.nb[2];
    sg.chunk0 = chunk0;
    chunk0 += sg.nchunks;
  }
  g->total_chunks = chunk0;
}

// ------------------------------------------------------------- read-backs
// The few bytes a call returns to the host (status word, container size,
// header) are written by a one-block kernel into mapped pinned host memory:
// no copy engine is involved, so these reads never queue behind large
// host<->device copies the caller has in flight on other streams.
// Bytes [0, n) from src to dst by the block: in 16-byte pieces where both are
// 16-byte aligned (each piece one write to the mapped host buffer, not 16),
// the tail byte by byte.
__device__ __forceinline__ void block_copy(const uint8_t* __restrict__ src,
                                           uint8_t* __restrict__ dst, int n) {
  int done = 0;
  if ((((uintptr_t)src | (uintptr_t)dst) & 15) == 0) {
    const int n16 = n >> 4;
    for (int i = threadIdx.x; i < n16; i += blockDim.x)
      ((uint4*)dst)[i] = ((const uint4*)src)[i];
    done = n16 << 4;
  }
  for (int i = done + threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
__global__ void k_readback(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, int n) {
  block_copy(src, dst, n);
}
// the same for two pieces at once
__global__ void k_readback2(const uint8_t* __restrict__ s0, uint8_t* __restrict__ d0, int n0,
                            const uint8_t* __restrict__ s1, uint8_t* __restrict__ d1, int n1) {
  block_copy(s0, d0, n0);
  block_copy(s1, d1, n1);
}

// Zero fill of device words by a kernel (not cudaMemsetAsync, which may be
// carried out by a copy engine and then wait behind the caller's copies).
__global__ void k_zero(uint32_t* __restrict__ p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0u;
}

static int zero_words(void* p, int64_t nwords, cudaStream_t st) {
  if (nwords <= 0) return STZ_OK;
  const int64_t blocks = imin(cdiv(nwords, 256), 1024);
  ProfScope ps_("k_zero", st);
  k_zero<<<(unsigned)blocks, 256, 0, st>>>((uint32_t*)p, nwords);
  return cuda_ok(cudaGetLastError());
}

int launch_zero_words(uint32_t* p, int64_t nwords, cudaStream_t s) {
  return zero_words(p, nwords, s);
}

namespace {
constexpr int kReadbackBytes = 4096;
thread_local uint8_t* tl_rb_host = nullptr;  // mapped, pinned, portable
thread_local uint8_t* tl_rb_dev = nullptr;   // its device address
}  // namespace

// This thread's read-back buffer, allocated on first use.
static int rb_ready() {
  if (tl_rb_host) return STZ_OK;
  if (cudaHostAlloc((void**)&tl_rb_host, kReadbackBytes,
                    cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    tl_rb_host = nullptr;
    return STZ_ERR_NOMEM;
  }
  if (cudaHostGetDevicePointer((void**)&tl_rb_dev, tl_rb_host, 0) != cudaSuccess) {
    cudaFreeHost(tl_rb_host);
    tl_rb_host = nullptr;
    return STZ_ERR_CUDA;
  }
  return STZ_OK;
}

// Queues a copy of n (<= 4096 - off) device bytes to offset off of this
// thread's read-back buffer; *host receives where they will be on the host.
static int readback(const void* src, int n, int off, cudaStream_t st, const uint8_t** host) {
  const int rr = rb_ready();
  if (rr != STZ_OK) return rr;
  if (n <= 0 || off < 0 || off + n > kReadbackBytes) return STZ_ERR_ARG;
  {
    ProfScope ps_("k_readback", st);
    k_readback<<<1, 256, 0, st>>>((const uint8_t*)src, tl_rb_dev + off, n);
  }
  if (cudaGetLastError() != cudaSuccess) return STZ_ERR_CUDA;
  *host = tl_rb_host + off;
  return STZ_OK;
}

// Two read-backs in one launch: n0 bytes to offset off0, n1 bytes to off1
// (the ranges must not overlap).
static int readback2(const void* s0, int n0, int off0, const void* s1, int n1, int off1,
                     cudaStream_t st, const uint8_t** h0, const uint8_t** h1) {
  const int rr = rb_ready();
  if (rr != STZ_OK) return rr;
  if (n0 <= 0 || off0 < 0 || off0 + n0 > kReadbackBytes || n1 <= 0 || off1 < 0 ||
      off1 + n1 > kReadbackBytes || (off0 < off1 + n1 && off1 < off0 + n0))
    return STZ_ERR_ARG;
  {
    ProfScope ps_("k_readback", st);
    k_readback2<<<1, 256, 0, st>>>((const uint8_t*)s0, tl_rb_dev + off0, n0,
                                   (const uint8_t*)s1, tl_rb_dev + off1, n1);
  }
  if (cudaGetLastError() != cudaSuccess) return STZ_ERR_CUDA;
  *h0 = tl_rb_host + off0;
  *h1 = tl_rb_host + off1;
  return STZ_OK;
}

static size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
static int64_t vol(const int64_t e[3]) { return e[0] * e[1] * e[2]; }

// Workspace plan; offsets in bytes from the workspace base.
struct WsPlan {
  size_t dp, range_part, grid[kMaxLevels + 1], codes, hist, chunk_out, chunk_words, lane_bits,
      word_off, out_off, enc, books, lay, lut, scan_sums, result, total;
};

static WsPlan plan_compress(const Geo& g) {
  WsPlan w;
  memset(&w, 0, sizeof(w));
  const size_t ps = g.dtype == STZ_F32 ? 4 : 8;
  size_t o = 0;
  w.dp = o;
  o += al256(sizeof(DevParams));
  w.range_part = o;
  o += al256(16 * (size_t)kRangeMaxBlocks);
  // reconstructed grids of levels 1..L-1 (level 1's also when L = 1: its
  // passes predict from it)
  for (int l = 1; l < (g.L > 1 ? g.L : 2); l++) {
    int64_t m[3];
    grid_extent(g.n, g.L, l, m);
    w.grid[l] = o;
    o += al256(ps * (size_t)vol(m));
  }
  w.codes = o;
  o += al256(2 * (size_t)(g.total_chunks * g.bvol));
  w.hist = o;
  o += al256(4 * (size_t)g.nstreams * kAlphabet);
  w.chunk_out = o;
  o += al256(4 * (size_t)g.total_chunks);
  w.chunk_words = o;
  o += al256(4 * (size_t)g.total_chunks);
  w.lane_bits = o;
  o += al256(2 * 32 * (size_t)g.total_chunks);
  w.word_off = o;
  o += al256(8 * (size_t)(g.total_chunks + 1));
  w.out_off = o;
  o += al256(8 * (size_t)(g.total_chunks + 1));
  w.enc = o;
  o += al256(2 * (size_t)g.nstreams * kAlphabet);
  w.books = o;
  o += al256(sizeof(BookDev) * (size_t)g.nstreams);
  w.lay = o;
  o += al256(sizeof(LayoutDev));
  w.lut = o;
  o += al256(4 * (size_t)g.nstreams * kLutSize);
  w.scan_sums = o;
  o += al256(16 * (size_t)(cdiv(g.total_chunks, 4096) + 1));
  w.result = o;
  o += al256(sizeof(unsigned long long) * 3);
  w.total = o;
  return w;
}

static int dims3(const int64_t* dims, int ndim, int64_t n[3]) {
  if (!dims || (ndim != 2 && ndim != 3)) return STZ_ERR_ARG;
  if (ndim == 3) {
    n[0] = dims[0];
    n[1] = dims[1];
    n[2] = dims[2];
  } else {
    n[0] = 1;
    n[1] = dims[0];
    n[2] = dims[1];
  }
  for (int a = 0; a < 3; a++)
    if (n[a] < 1 || n[a] > ((int64_t)1 << 31)) return STZ_ERR_ARG;
  if (n[0] * n[1] > ((int64_t)1 << 40) / n[2]) return STZ_ERR_ARG;
  return STZ_OK;
}

static const int* default_brick(int ndim) { return ndim == 3 ? kBrick3D : kBrick2D; }

static size_t bound_of(const Geo& g) {
  const size_t ps = g.dtype == STZ_F32 ? 4 : 8;
  size_t total = kHeaderBytes + (size_t)g.nstreams * kDirEntryBytes;
  for (int s = 0; s < g.nstreams; s++) {
    const StreamGeo& sg = g.s[s];
    size_t nsym = (size_t)sg.nsym, nch = (size_t)sg.nchunks;
    size_t nlive = nsym < (size_t)kAlphabet ? nsym : (size_t)kAlphabet;
    size_t pw = (nsym * kMaxCodeLen + 31) / 32 + nch;
    size_t sect = ((((3 * nlive + 3) & ~(size_t)3) + 4 * nch + 2 * nch * (kNSub - 1) + 3) &
                   ~(size_t)3) + 4 * pw + 4 * nsym;
    sect = ((sect + 7) & ~(size_t)7) + ps * nsym;
    total += (sect + 7) & ~(size_t)7;
  }
  return total;
}

// ------------------------------------------------------------ header parsing
struct Hdr {
  int dtype, ndim, L, eb_mode, maxlen, R, ns, nsub, pred;
  int b[3];
  int64_t n[3];
  double eb, eb_abs, two_eb[kMaxLevels + 1];
  uint64_t total;
  struct {
    uint64_t sect_off, nsym, pw, nout;
    uint32_t nch, nlive;
  } d[kMaxStreams];
};

static uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint64_t rd64(const uint8_t* p) { return (uint64_t)rd32(p) | ((uint64_t)rd32(p + 4) << 32); }
static double rdf64(const uint8_t* p) {
  uint64_t u = rd64(p);
  double v;
  memcpy(&v, &u, 8);
  return v;
}

struct SectHost {
  uint64_t off_syms, off_lens, off_chunks, off_subs, off_payload, off_opos, off_oval, size;
};
static SectHost sect_host(uint64_t nlive, uint64_t nch, uint64_t pw, uint64_t nout, uint64_t ps,
                          int nsub) {
  SectHost s;
  s.off_syms = 0;
  s.off_lens = 2 * nlive;
  s.off_chunks = (3 * nlive + 3) & ~3ull;
  s.off_subs = s.off_chunks + 4 * nch;
  s.off_payload = (s.off_subs + 2 * nch * (uint64_t)(nsub - 1) + 3) & ~3ull;
  s.off_opos = s.off_payload + 4 * pw;
  s.off_oval = (s.off_opos + 4 * nout + 7) & ~7ull;
  s.size = (s.off_oval + ps * nout + 7) & ~7ull;
  return s;
}

// Parse and check the header and directory (h holds `avail` bytes).
// Returns STZ_OK, STZ_ERR_CORRUPT, or STZ_ERR_ARG for valid containers with
// options this library does not decode (radius other than 1024, codes longer
// than 12 bits, bricks whose tiles exceed shared memory).
static int parse_hdr(const uint8_t* h, size_t avail, size_t comp_bytes, Hdr* H) {
  memset(H, 0, sizeof(*H));
  if (avail < (size_t)kHeaderBytes || memcmp(h, "STZ1", 4) != 0) return STZ_ERR_CORRUPT;
  if ((h[4] | (h[5] << 8)) != 1) return STZ_ERR_CORRUPT;
  H->dtype = h[6];
  H->ndim = h[7];
  H->L = h[8];
  H->eb_mode = h[9];
  H->maxlen = h[10];
  H->nsub = h[11];
  H->R = (int)rd32(h + 12);
  for (int a = 0; a < 3; a++) H->b[a] = (int)rd32(h + 16 + 4 * a);
  H->ns = (int)rd32(h + 28);
  for (int a = 0; a < 3; a++) H->n[a] = (int64_t)rd64(h + 32 + 8 * a);
  H->eb = rdf64(h + 56);
  H->eb_abs = rdf64(h + 64);
  H->total = rd64(h + 88);
  H->pred = h[200];
  if (H->dtype != STZ_F32 && H->dtype != STZ_F64) return STZ_ERR_CORRUPT;
  if (H->pred != kPredCubic && H->pred != kPredLinear && H->pred != kPredDirect)
    return STZ_ERR_CORRUPT;
  if (H->ndim != 2 && H->ndim != 3) return STZ_ERR_CORRUPT;
  if (H->L < 1 || H->L > kMaxLevels) return STZ_ERR_CORRUPT;
  if (H->eb_mode != STZ_EB_ABS && H->eb_mode != STZ_EB_REL) return STZ_ERR_CORRUPT;
  if (H->maxlen < 1 || H->maxlen > 24) return STZ_ERR_CORRUPT;
  if (H->R < 2 || H->R > 32768 || 2 * (int64_t)H->R > ((int64_t)1 << H->maxlen))
    return STZ_ERR_CORRUPT;
  for (int a = 0; a < 3; a++) {
    if (H->b[a] < 1 || H->b[a] > 4096) return STZ_ERR_CORRUPT;
    if (H->n[a] < 1 || H->n[a] > ((int64_t)1 << 31)) return STZ_ERR_CORRUPT;
  }
  if ((int64_t)H->b[0] * H->b[1] * H->b[2] * H->maxlen > 65535) return STZ_ERR_CORRUPT;
  if (H->nsub != 1 && H->nsub != 2 && H->nsub != 4 && H->nsub != 8) return STZ_ERR_CORRUPT;
  if (H->n[0] * H->n[1] > ((int64_t)1 << 40) / H->n[2]) return STZ_ERR_CORRUPT;
  if (H->ndim == 2 && H->n[0] != 1) return STZ_ERR_CORRUPT;
  if (H->ns != 1 + 7 * (H->L - 1)) return STZ_ERR_CORRUPT;
  if (H->total > comp_bytes) return STZ_ERR_CORRUPT;
  const uint64_t dir_end = kHeaderBytes + (uint64_t)H->ns * kDirEntryBytes;
  if (dir_end > H->total || avail < dir_end) return STZ_ERR_CORRUPT;
  for (int l = 1; l <= H->L; l++) H->two_eb[l] = rdf64(h + 144 + 8 * (l - 1));
  Geo g;
  make_geo(H->n, H->ndim, H->dtype, H->L, H->b, &g);
  const uint64_t ps = H->dtype == STZ_F32 ? 4 : 8;
  for (int s = 0; s < H->ns; s++) {
    const uint8_t* d = h + kHeaderBytes + (size_t)s * kDirEntryBytes;
    H->d[s].sect_off = rd64(d);
    H->d[s].nsym = rd64(d + 8);
    H->d[s].nch = rd32(d + 16);
    H->d[s].nlive = rd32(d + 20);
    H->d[s].pw = rd64(d + 24);
    H->d[s].nout = rd64(d + 32);
    const auto& e = H->d[s];
    if (e.nsym != (uint64_t)g.s[s].nsym || e.nch != (uint64_t)g.s[s].nchunks) return STZ_ERR_CORRUPT;
    if (e.nlive > (uint64_t)2 * H->R || (e.nsym > 0 && e.nlive == 0)) return STZ_ERR_CORRUPT;
    if (e.nout > e.nsym || e.pw > e.nsym * 24 + e.nch) return STZ_ERR_CORRUPT;
    if (e.sect_off % 8 || e.sect_off < dir_end || e.sect_off > H->total) return STZ_ERR_CORRUPT;
    SectHost sh = sect_host(e.nlive, e.nch, e.pw, e.nout, ps, H->nsub);
    if (sh.size > H->total - e.sect_off) return STZ_ERR_CORRUPT;
  }
  if (H->R != kRadius || H->maxlen > kMaxCodeLen) return STZ_ERR_ARG;
  {
    int64_t m1[3];  // the level-1 grid is indexed in 32 bits
    grid_extent(H->n, H->L, 1, m1);
    if (m1[0] * m1[1] * m1[2] >= ((int64_t)1 << 31)) return STZ_ERR_ARG;
  }
  {
    int64_t tv = 1;
    for (int a = 0; a < 3; a++) tv *= H->b[a] + 3;
    if (tv * (int64_t)ps > 160 * 1024 || (int64_t)H->b[0] * H->b[1] * H->b[2] > 4096)
      return STZ_ERR_ARG;
  }
  return STZ_OK;
}

static_assert(STZ_HEADER_MAX_BYTES == kHeaderBytes + kMaxStreams * kDirEntryBytes,
              "header bytes a serving loop keeps on the host");

static int read_hdr(const void* comp, size_t comp_bytes, int on_device, cudaStream_t st, Hdr* H) {
  if (!comp || comp_bytes < (size_t)kHeaderBytes) return STZ_ERR_CORRUPT;
  const size_t want = kHeaderBytes + (size_t)kMaxStreams * kDirEntryBytes;
  const size_t n = comp_bytes < want ? comp_bytes : want;
  uint8_t buf[kHeaderBytes + kMaxStreams * kDirEntryBytes];
  if (on_device) {
    const uint8_t* h = nullptr;
    const int rc = readback(comp, (int)n, 0, st, &h);
    if (rc != STZ_OK) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return STZ_ERR_CUDA;
    memcpy(buf, h, n);
  } else {
    memcpy(buf, comp, n);
  }
  return parse_hdr(buf, n, comp_bytes, H);
}

// Decode workspace plan for a region: level-1 grid, box grids of levels
// 2..k-1, code slots of the needed chunks, decode tables.
struct DecPlan {
  int k;
  int64_t OA[3], OB[3];                                // output box on G_k
  int64_t A[kMaxLevels + 1][3], B[kMaxLevels + 1][3];  // grid boxes on G_j (G_1 whole)
  int64_t N1A[3], N1B[3];                              // the part of G_1 the output needs
  int64_t tlo[kMaxLevels + 1][3], tcnt[kMaxLevels + 1][3];
  SlotMap sm[kMaxStreams];
  int64_t nslots;
  size_t dp, grid[kMaxLevels + 1], codes, lut, sub_olo, total;
};

// Coarse support of the G_j coordinates [a, b) along one axis, on G_{j-1}
// (extent M): a coordinate 2c + 1 is predicted from coarse c - 1 .. c + 2
// (the cubic reach, Eqs. 6-8; the boundary rules use a subset), a
// coordinate 2c is the copy of coarse c.  A range holding one even
// coordinate -- an axis-aligned slice on the lattice of the coarser level --
// therefore needs one coarse plane; any other range needs its widened hull.
static void coarse_support(int64_t a, int64_t b, int64_t M, int64_t* ca, int64_t* cb) {
  if (b - a == 1 && a % 2 == 0) {
    *ca = a / 2;
    *cb = a / 2 + 1;
  } else {
    *ca = imax(0, a / 2 - 1);
    *cb = imin(M, b / 2 + 2);
  }
}

// skip_l1: the caller supplies the decoded level-1 grid (no level-1 buffer,
// no level-1 code slots).
//
// Random access (Sec. 3.3): at each level j >= 2 only the points of the box
// [A[j], B[j]) are predicted, and of the level's 7 sub-block streams each
// decodes only the bricks holding its own points of that box.  A sub-block
// whose offset parity along some axis never occurs in the box (an
// axis-aligned slice at an even coordinate has no odd-z points) decodes no
// chunk at all: a z-slice at the finest level reads 3 of the 7 level-L
// streams, the 2D-slice decoding saving of Sec. 3.3.
static void plan_decode(const Geo& g, int k, const int64_t lo[3], const int64_t hi[3], DecPlan* P,
                        bool skip_l1 = false) {
  memset(P, 0, sizeof(*P));
  P->k = k;
  const int64_t sk = level_stride(g.L, k);
  for (int a = 0; a < 3; a++) {
    P->OA[a] = P->A[k][a] = cdiv(lo[a], sk);
    P->OB[a] = P->B[k][a] = cdiv(hi[a], sk);
  }
  for (int j = k; j >= 2; j--) {
    int64_t M[3];
    grid_extent(g.n, g.L, j - 1, M);
    for (int a = 0; a < 3; a++)
      coarse_support(P->A[j][a], P->B[j][a], M[a], &P->A[j - 1][a], &P->B[j - 1][a]);
  }
  {
    int64_t m1[3];
    grid_extent(g.n, g.L, 1, m1);
    for (int a = 0; a < 3; a++) {
      P->N1A[a] = P->A[1][a];
      P->N1B[a] = P->B[1][a];
      P->A[1][a] = 0;  // the level-1 grid buffer is always laid out whole
      P->B[1][a] = m1[a];
    }
  }
  // slots: level 1 whole, then for each level and sub-block the bricks over
  // that sub-block's points in the box
  int64_t nslots = 0;
  const StreamGeo& s0 = g.s[0];
  for (int a = 0; a < 3; a++) {
    P->sm[0].lo[a] = 0;
    P->sm[0].cnt[a] = skip_l1 ? 0 : s0.nb[a];
  }
  P->sm[0].base = 0;
  if (!skip_l1) nslots += s0.nchunks;
  for (int j = 2; j <= k; j++) {
    for (int a = 0; a < 3; a++) {
      const int64_t clo = P->A[j][a] / 2, chi = cdiv(P->B[j][a], 2);
      P->tlo[j][a] = clo / g.b[a];
      P->tcnt[j][a] = imax(0, cdiv(chi, g.b[a]) - P->tlo[j][a]);
    }
    for (int K = 1; K <= 7; K++) {
      const int sid = 1 + 7 * (j - 2) + (K - 1);
      const StreamGeo& sg = g.s[sid];
      SlotMap& sm = P->sm[sid];
      int64_t c = 1;
      for (int a = 0; a < 3; a++) {
        // cells c of the sub-block with 2c + o in [A, B)
        const int64_t o = sg.o[a];
        const int64_t c0 = imax(0, (P->A[j][a] - o + 1) >> 1);
        const int64_t c1 = imin(sg.e[a], (P->B[j][a] - o + 1) >> 1);
        if (c1 <= c0) {
          c = 0;
          break;
        }
        sm.lo[a] = c0 / g.b[a];
        sm.cnt[a] = cdiv(c1, g.b[a]) - sm.lo[a];
        c *= sm.cnt[a];
      }
      if (c == 0)
        for (int a = 0; a < 3; a++) sm.lo[a] = sm.cnt[a] = 0;
      sm.base = nslots;
      nslots += c;
    }
  }
  P->nslots = nslots;
  const size_t ps = g.dtype == STZ_F32 ? 4 : 8;
  size_t o = 0;
  P->dp = o;
  o += al256(sizeof(DevParams));
  for (int j = skip_l1 ? 2 : 1; j < (k > 1 ? k : 2); j++) {
    P->grid[j] = o;
    int64_t e[3] = {P->B[j][0] - P->A[j][0], P->B[j][1] - P->A[j][1], P->B[j][2] - P->A[j][2]};
    o += al256(ps * (size_t)vol(e));
  }
  P->codes = o;
  o += al256(2 * (size_t)(nslots * g.bvol));
  P->lut = o;
  o += al256(4 * (size_t)g.nstreams * kLutSize);
  // where each decoded chunk's sub-chunks start in their stream's outlier list
  P->sub_olo = o;
  o += al256(4 * (size_t)(kNSub + 1) * (size_t)(nslots > 0 ? nslots : 1));
  P->total = o;
}

// ------------------------------------------------------------ launch share
namespace {
thread_local int tl_share_num = 1, tl_share_den = 1;
}

void set_launch_share(int num, int den) {
  tl_share_num = num > 0 ? num : 1;
  tl_share_den = den > 0 ? den : 1;
}

int launch_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int v = (int)((int64_t)sms * tl_share_num / tl_share_den);
  return v > 0 ? v : 1;
}

namespace {
struct SmemLimit {
  const void* func;
  int dev, bytes;
};
constexpr int kSmemLimits = 512;  // kernel instances x devices, with room
std::mutex g_smem_mu;
SmemLimit g_smem[kSmemLimits];
int g_nsmem = 0;
}  // namespace

int allow_smem(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return STZ_OK;  // within the default limit
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return STZ_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  SmemLimit* e = nullptr;
  for (int i = 0; i < g_nsmem; i++)
    if (g_smem[i].func == func && g_smem[i].dev == dev) e = &g_smem[i];
  if (e && (size_t)e->bytes >= bytes) return STZ_OK;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
      cudaSuccess)
    return STZ_ERR_CUDA;
  if (!e && g_nsmem < kSmemLimits) {
    e = &g_smem[g_nsmem++];
    e->func = func;
    e->dev = dev;
  }
  if (e) e->bytes = (int)bytes;
  return STZ_OK;
}

// ------------------------------------------------------------- compression
// The three words a compression reports, gathered for one read-back:
// container bytes, payload words, status bits.
__global__ void k_result(const unsigned long long* __restrict__ total,
                         const unsigned long long* __restrict__ payload_words,
                         const uint32_t* __restrict__ status, unsigned long long* __restrict__ r) {
  if (threadIdx.x == 0) {
    r[0] = *total;
    r[1] = *payload_words;
    r[2] = *status;
  }
}

// Argument checks of stz_compress; fills the job (geometry, workspace plan).
int compress_check(const void* field_dev, const int64_t* dims, int ndim, int dtype, int eb_mode,
                   double eb, void* out_dev, size_t out_cap, void* ws_dev, size_t ws_bytes,
                   CompressJob* j, const stz_compress_opts* opts) {
  int64_t n[3];
  if (dims3(dims, ndim, n) != STZ_OK) return STZ_ERR_ARG;
  int L = kLevels, pred = kPredCubic;
  double ratio = 2.5;
  if (opts) {
    if (opts->levels != 0) L = opts->levels;
    pred = (int)opts->predictor;
    if (opts->eb_ratio != 0.0) ratio = opts->eb_ratio;
  }
  if (L < 1 || L > kMaxLevels) return STZ_ERR_ARG;
  if (pred != kPredCubic && pred != kPredLinear && pred != kPredDirect) return STZ_ERR_ARG;
  if (!(ratio >= 1.0 && ratio <= 64.0)) return STZ_ERR_ARG;
  if (dtype != STZ_F32 && dtype != STZ_F64) return STZ_ERR_ARG;
  if (eb_mode != STZ_EB_ABS && eb_mode != STZ_EB_REL) return STZ_ERR_ARG;
  if (!(eb > 0.0) || !isfinite(eb)) return STZ_ERR_ARG;
  if (!field_dev || !out_dev || !ws_dev) return STZ_ERR_ARG;
  if (((uintptr_t)field_dev % 16) || ((uintptr_t)out_dev % 8) || ((uintptr_t)ws_dev % 256))
    return STZ_ERR_ARG;
  memset(j, 0, sizeof(*j));
  make_geo(n, ndim, dtype, L, default_brick(ndim), &j->g);
  {
    // the level-1 grid (with L = 1 the whole field) is indexed in 32 bits
    int64_t m1[3];
    grid_extent(n, L, 1, m1);
    if (m1[0] * m1[1] * m1[2] >= ((int64_t)1 << 31)) return STZ_ERR_ARG;
  }
  if (ws_bytes < plan_compress(j->g).total) return STZ_ERR_CAPACITY;
  j->pred = pred;
  j->eb_ratio = ratio;
  j->field = field_dev;
  j->eb_mode = eb_mode;
  j->eb = eb;
  j->out = out_dev;
  j->out_cap = out_cap;
  j->ws = ws_dev;
  return STZ_OK;
}

// Queues every stage of one compression on st without waiting for it.
// no_coop: run the level-1 passes as plain launches (no cooperative launch),
// as needed inside a captured graph whose branches run concurrently.
// The compress arguments of level l (2..L) of job j.
void compress_level_args(const CompressJob& j, int l, LevelArgs* out) {
  const Geo& g = j.g;
  const WsPlan w = plan_compress(g);
  uint8_t* ws = (uint8_t*)j.ws;
  LevelArgs& a = *out;
  memset(&a, 0, sizeof(a));
  a.geo = g;
  a.level = l;
  a.pred = j.pred;
  a.dp = (DevParams*)(ws + w.dp);
  a.field = j.field;
  int64_t M[3], m[3];
  grid_extent(g.n, g.L, l - 1, M);
  grid_extent(g.n, g.L, l, m);
  a.coarse = ws + w.grid[l - 1];
  a.fine = l < g.L ? (void*)(ws + w.grid[l]) : nullptr;
  for (int d = 0; d < 3; d++) {
    a.clo[d] = 0;
    a.chi[d] = M[d];
    a.flo[d] = 0;
    a.fhi[d] = m[d];
    a.tlo[d] = 0;
    a.tcnt[d] = cdiv(M[d], g.b[d]);
  }
  a.codes = (uint16_t*)(ws + w.codes);
  a.chunk_outliers = (uint32_t*)(ws + w.chunk_out);
  a.hist = (uint32_t*)(ws + w.hist);
  a.status = &((DevParams*)(ws + w.dp))->status;
  for (int K = 1; K <= 7; K++) {
    const StreamGeo& sg = g.s[1 + 7 * (l - 2) + K - 1];
    for (int d = 0; d < 3; d++) {
      a.sm[K].lo[d] = 0;
      a.sm[K].cnt[d] = sg.nb[d];
    }
    a.sm[K].base = sg.chunk0;
  }
}

#define STZ_TRY(x)               \
  do {                           \
    const int rc_ = (x);         \
    if (rc_ != STZ_OK) return rc_; \
  } while (0)

// Compression up to level 1: the range pass (which also clears the
// histograms and the per-chunk outlier counts), the bounds, the level-1
// coder and level 1's histogram.
int compress_prologue(const CompressJob& j, bool no_coop, cudaStream_t st) {
  const Geo& g = j.g;
  const WsPlan w = plan_compress(g);
  uint8_t* ws = (uint8_t*)j.ws;
  DevParams* dp = (DevParams*)(ws + w.dp);
  uint16_t* codes = (uint16_t*)(ws + w.codes);
  uint32_t* hist = (uint32_t*)(ws + w.hist);
  uint32_t* chunk_out = (uint32_t*)(ws + w.chunk_out);
  {
    unsigned long long* part = (unsigned long long*)(ws + w.range_part);
    int nparts = 0;
    STZ_TRY(launch_range(j.field, g.dtype, j.eb_mode == STZ_EB_REL ? vol(g.n) : 0, part, &nparts,
                         hist, (int64_t)g.nstreams * kAlphabet, chunk_out, g.total_chunks, st));
    STZ_TRY(launch_params(dp, part, nparts, g.dtype, j.eb_mode, j.eb, g.L, kRadius, j.eb_ratio,
                          j.pred, st));
  }
  {
    BaseArgs a;
    memset(&a, 0, sizeof(a));
    a.geo = g;
    a.dp = dp;
    a.field = j.field;
    a.g1 = ws + w.grid[1];
    a.codes = codes;
    a.chunk_outliers = chunk_out;
    for (int d = 0; d < 3; d++) {
      a.sm.lo[d] = 0;
      a.sm.cnt[d] = g.s[0].nb[d];
    }
    a.sm.base = g.s[0].chunk0;
    STZ_TRY(no_coop ? launch_base_nocoop(a, false, st) : launch_base(a, false, st));
  }
  STZ_TRY(launch_stream_hist(g, 0, codes, hist, st));
  return STZ_OK;
}

// Levels 2..L of a compression, one level launch after another.
int compress_levels(const CompressJob& j, cudaStream_t st) {
  for (int l = 2; l <= j.g.L; l++) {
    LevelArgs a;
    compress_level_args(j, l, &a);
    STZ_TRY(launch_level(a, false, st));
  }
  return STZ_OK;
}

// The entropy stage and the container: codebooks, chunk bit counts, their
// scans, the section layout, the sections and the payload, the result word.
int compress_epilogue(const CompressJob& j, cudaStream_t st, CompressDev* d) {
  const Geo& g = j.g;
  const WsPlan w = plan_compress(g);
  uint8_t* ws = (uint8_t*)j.ws;
  DevParams* dp = (DevParams*)(ws + w.dp);
  uint16_t* codes = (uint16_t*)(ws + w.codes);
  uint32_t* hist = (uint32_t*)(ws + w.hist);
  uint32_t* chunk_out = (uint32_t*)(ws + w.chunk_out);
  uint32_t* chunk_words = (uint32_t*)(ws + w.chunk_words);
  uint16_t* lane_bits = (uint16_t*)(ws + w.lane_bits);
  unsigned long long* word_off = (unsigned long long*)(ws + w.word_off);
  unsigned long long* out_off = (unsigned long long*)(ws + w.out_off);
  uint16_t* enc = (uint16_t*)(ws + w.enc);
  BookDev* books = (BookDev*)(ws + w.books);
  LayoutDev* lay = (LayoutDev*)(ws + w.lay);
  uint8_t* out = (uint8_t*)j.out;
  STZ_TRY(launch_codebook(g, hist, enc, books, st));
  STZ_TRY(launch_chunk_words(g, codes, enc, chunk_words, lane_bits, st));
  STZ_TRY(launch_scan2(chunk_words, chunk_out, g.total_chunks,
                       (unsigned long long*)(ws + w.scan_sums), word_off, out_off, st));
  STZ_TRY(launch_layout(g, dp, j.eb_mode, word_off, out_off, books, lay, out, j.out_cap, st));
  STZ_TRY(launch_sections(g, lay, books, word_off, dp, out, st));
  STZ_TRY(launch_pack(g, codes, enc, lane_bits, word_off, lay->s, out, dp, j.field, chunk_out,
                      out_off, st));
  unsigned long long* res = (unsigned long long*)(ws + w.result);
  {
    ProfScope ps_("k_result", st);
    k_result<<<1, 32, 0, st>>>(&lay->total, word_off + g.total_chunks, &dp->status, res);
    STZ_TRY(cuda_ok(cudaGetLastError()));
  }
  d->total = &lay->total;
  d->payload_words = word_off + g.total_chunks;
  d->status = &dp->status;
  d->result = res;
  return STZ_OK;
}
#undef STZ_TRY

int compress_enqueue(const CompressJob& j, bool no_coop, cudaStream_t st, CompressDev* d) {
  int rc = compress_prologue(j, no_coop, st);
  if (rc == STZ_OK) rc = compress_levels(j, st);
  if (rc == STZ_OK) rc = compress_epilogue(j, st, d);
  return rc;
}

// Captured compressions, by their arguments: a repeated stz_compress replays
// one graph.  The graph holds the launch sequence with every pointer and size
// fixed; the field's current contents are read at each replay.
namespace {
struct CompKey {
  int dev, ndim, dtype, eb_mode, levels, pred;
  const void* field;
  int64_t dims[3];
  double eb, eb_ratio;
  void* out;
  size_t out_cap;
  void* ws;
  size_t ws_bytes;
};
struct CompGraph {
  CompKey key;
  cudaGraphExec_t exec;
  unsigned long long kernels;
  CompressDev d;
  unsigned long long last;
};
constexpr int kCompGraphs = 8;
std::mutex g_cg_mu;
CompGraph g_cg[kCompGraphs];
int g_ncg = 0;
unsigned long long g_cg_tick = 0;
cudaStream_t g_cap_stream[64];

unsigned long long graph_kernels(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
  cudaGraphNode_t* nodes = (cudaGraphNode_t*)malloc(sizeof(cudaGraphNode_t) * n);
  if (!nodes) return 0;
  unsigned long long k = 0;
  if (cudaGraphGetNodes(g, nodes, &n) == cudaSuccess)
    for (size_t i = 0; i < n; i++) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) k++;
    }
  free(nodes);
  return k;
}
}  // namespace

int compress_graph_launch(const CompressJob& j, const void* field, const int64_t dims[3], int ndim,
                          int dtype, int eb_mode, double eb, void* out, size_t out_cap, void* ws,
                          size_t ws_bytes, cudaStream_t st, CompressDev* d) {
  CompKey key;
  memset(&key, 0, sizeof(key));
  if (cudaGetDevice(&key.dev) != cudaSuccess || key.dev < 0 || key.dev >= 64) return STZ_ERR_CUDA;
  key.ndim = ndim;
  key.dtype = dtype;
  key.eb_mode = eb_mode;
  key.field = field;
  for (int a = 0; a < 3; a++) key.dims[a] = dims[a];
  key.eb = eb;
  key.levels = j.g.L;
  key.pred = j.pred;
  key.eb_ratio = j.eb_ratio;
  key.out = out;
  key.out_cap = out_cap;
  key.ws = ws;
  key.ws_bytes = ws_bytes;
  std::lock_guard<std::mutex> lk(g_cg_mu);
  CompGraph* hit = nullptr;
  for (int i = 0; i < g_ncg; i++)
    if (memcmp(&g_cg[i].key, &key, sizeof(key)) == 0) hit = &g_cg[i];
  if (!hit) {
    int slot;
    if (g_ncg < kCompGraphs) {
      slot = g_ncg++;
      g_cg[slot].exec = nullptr;
    } else {  // the least recently used entry makes room
      slot = 0;
      for (int i = 1; i < kCompGraphs; i++)
        if (g_cg[i].last < g_cg[slot].last) slot = i;
      if (g_cg[slot].exec) cudaGraphExecDestroy(g_cg[slot].exec);
      g_cg[slot].exec = nullptr;
    }
    cudaStream_t& cap = g_cap_stream[key.dev];
    if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
      cap = nullptr;
      return STZ_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    CompressDev dd;
    int rc = cuda_ok(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    if (rc != STZ_OK) return rc;
    // inside a graph the level-1 passes are plain launches (no cooperative one)
    rc = compress_enqueue(j, true, cap, &dd);
    const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    if (rc == STZ_OK && ce != cudaSuccess) rc = STZ_ERR_CUDA;
    if (rc != STZ_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      memset(&g_cg[slot].key, 0, sizeof(CompKey));  // never matches (null field)
      g_cg[slot].exec = nullptr;
      return rc;
    }
    CompGraph& c = g_cg[slot];
    c.key = key;
    c.d = dd;
    c.kernels = graph_kernels(graph);
    const cudaError_t ie = cudaGraphInstantiate(&c.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      c.exec = nullptr;
      memset(&c.key, 0, sizeof(c.key));
      return STZ_ERR_CUDA;
    }
    hit = &c;
  }
  hit->last = ++g_cg_tick;
  if (cudaGraphLaunch(hit->exec, st) != cudaSuccess) return STZ_ERR_CUDA;
  prof_count_launches(hit->kernels);
  *d = hit->d;
  return STZ_OK;
}

}  // namespace stz

using namespace stz;

// ------------------------------------------------------------------ kernels
// copy a box of the level-1 grid to the output (progressive/region at level 1)
template <typename T>
__global__ void k_copy_box(const T* __restrict__ src, T* __restrict__ dst, int64_t a0, int64_t a1,
                           int64_t a2, int64_t e0, int64_t e1, int64_t e2, int64_t m1,
                           int64_t m2) {
  const int64_t n = e0 * e1 * e2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t x = i % e2, y = (i / e2) % e1, z = i / (e1 * e2);
    dst[i] = src[((z + a0) * m1 + (y + a1)) * m2 + (x + a2)];
  }
}

namespace stz {
// a level-1 request of a batch: a box of the cached level-1 grid copied to
// the output
struct CopyJob {
  const void* src;
  void* dst;
  int64_t a[3], e[3], m1, m2;
};
}  // namespace stz

template <typename T>
__global__ void k_copy_boxes(const CopyJob* __restrict__ jobs) {
  const CopyJob& j = jobs[blockIdx.y];
  const int64_t n = j.e[0] * j.e[1] * j.e[2];
  const T* __restrict__ src = (const T*)j.src;
  T* __restrict__ dst = (T*)j.dst;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % j.e[2], y = (i / j.e[2]) % j.e[1], z = i / (j.e[1] * j.e[2]);
    dst[i] = src[((z + j.a[0]) * j.m1 + (y + j.a[1])) * j.m2 + (x + j.a[2])];
  }
}

extern "C" {

const char* stz_strerror(int code) {
  switch (code) {
    case STZ_OK: return "ok";
    case STZ_ERR_ARG: return "invalid argument or unsupported option";
    case STZ_ERR_CAPACITY: return "buffer too small";
    case STZ_ERR_CORRUPT: return "corrupt container";
    case STZ_ERR_CUDA: return "CUDA runtime error";
    case STZ_ERR_TIMEOUT: return "device wait timed out";
    case STZ_ERR_NOMEM: return "host allocation failed";
    default: return "unknown error";
  }
}

const char* stz_version(void) { return "stz-gb300 1.0 (sm_103a)"; }

size_t stz_compress_bound_ex(const int64_t* dims, int ndim, stz_dtype dtype, int levels) {
  int64_t n[3];
  if (levels == 0) levels = kLevels;
  if (dims3(dims, ndim, n) != STZ_OK || (dtype != STZ_F32 && dtype != STZ_F64) || levels < 1 ||
      levels > kMaxLevels)
    return 0;
  Geo g;
  make_geo(n, ndim, dtype, levels, default_brick(ndim), &g);
  return bound_of(g);
}

size_t stz_compress_bound(const int64_t* dims, int ndim, stz_dtype dtype) {
  return stz_compress_bound_ex(dims, ndim, dtype, kLevels);
}

size_t stz_workspace_size_ex(const int64_t* dims, int ndim, stz_dtype dtype, int levels) {
  int64_t n[3];
  if (levels == 0) levels = kLevels;
  if (dims3(dims, ndim, n) != STZ_OK || (dtype != STZ_F32 && dtype != STZ_F64) || levels < 1 ||
      levels > kMaxLevels)
    return 0;
  Geo g;
  make_geo(n, ndim, dtype, levels, default_brick(ndim), &g);
  WsPlan w = plan_compress(g);
  DecPlan P;
  int64_t lo[3] = {0, 0, 0};
  plan_decode(g, g.L, lo, g.n, &P);
  return w.total > P.total ? w.total : P.total;
}

size_t stz_workspace_size(const int64_t* dims, int ndim, stz_dtype dtype) {
  return stz_workspace_size_ex(dims, ndim, dtype, kLevels);
}

int stz_compress_ex(const void* field_dev, const int64_t* dims, int ndim, stz_dtype dtype,
                    stz_eb_mode eb_mode, double eb, const stz_compress_opts* opts,
                    void* out_dev, size_t out_cap, size_t* out_bytes, void* ws_dev,
                    size_t ws_bytes, void* stream) {
  if (!out_bytes) return STZ_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CompressJob j;
  int rc = compress_check(field_dev, dims, ndim, dtype, eb_mode, eb, out_dev, out_cap, ws_dev,
                          ws_bytes, &j, opts);
  if (rc != STZ_OK) return rc;
  CompressDev d;
  // repeated calls with the same arguments replay one captured graph (no
  // per-kernel launches); while the kernel timer is on, plain launches
  if (prof_enabled()) {
    rc = compress_enqueue(j, false, st, &d);
  } else {
    const int64_t nd[3] = {dims[0], dims[1], ndim == 3 ? dims[2] : 0};
    rc = compress_graph_launch(j, field_dev, nd, ndim, dtype, eb_mode, eb, out_dev, out_cap,
                               ws_dev, ws_bytes, st, &d);
  }
  if (rc != STZ_OK) return rc;
  const uint8_t* hres = nullptr;
  if ((rc = readback(d.result, 3 * (int)sizeof(unsigned long long), 0, st, &hres)) != STZ_OK)
    return rc;
  if ((rc = cuda_ok(cudaStreamSynchronize(st))) != STZ_OK) return rc;
  unsigned long long r[3];
  memcpy(r, hres, sizeof(r));
  *out_bytes = (size_t)r[0];
  prof_add_bytes("k_pack", 4.0 * (double)r[1]);
  if (r[2] & kStatTimeout) return STZ_ERR_TIMEOUT;
  if (r[2] & kStatCapacity) return STZ_ERR_CAPACITY;
  return STZ_OK;
}

int stz_compress(const void* field_dev, const int64_t* dims, int ndim, stz_dtype dtype,
                 stz_eb_mode eb_mode, double eb, void* out_dev, size_t out_cap,
                 size_t* out_bytes, void* ws_dev, size_t ws_bytes, void* stream) {
  return stz_compress_ex(field_dev, dims, ndim, dtype, eb_mode, eb, nullptr, out_dev, out_cap,
                         out_bytes, ws_dev, ws_bytes, stream);
}

int stz_info(const void* comp, size_t comp_bytes, int comp_on_device, stz_info_t* info) {
  if (!info) return STZ_ERR_ARG;
  Hdr H;
  int rc = read_hdr(comp, comp_bytes, comp_on_device, (cudaStream_t)0, &H);
  if (rc == STZ_ERR_CUDA || rc == STZ_ERR_CORRUPT) return rc;
  memset(info, 0, sizeof(*info));
  info->dtype = (stz_dtype)H.dtype;
  info->ndim = H.ndim;
  if (H.ndim == 3) {
    for (int a = 0; a < 3; a++) info->dims[a] = H.n[a];
  } else {
    info->dims[0] = H.n[1];
    info->dims[1] = H.n[2];
    info->dims[2] = 1;
  }
  info->levels = H.L;
  info->eb = H.eb;
  info->eb_mode = (stz_eb_mode)H.eb_mode;
  info->eb_abs = H.eb_abs;
  info->total_bytes = H.total;
  return rc;
}

// Parsed headers of recently decoded containers, by device, address and
// size.  A plain decode of a container seen before starts its launches at
// once from the cached header instead of waiting for a read-back; it copies
// the header bytes back beside its final status word and, if they differ
// from the cached ones (another container now sits at that address), decodes
// again with the fresh header.  A stale header cannot lead a decode outside
// its buffers: its sections lie within the same comp_bytes, and the output
// and workspace sizes are checked against the plan it gives.
namespace {
struct HdrCacheEntry {
  int dev;
  const void* ptr;
  size_t bytes, nraw;
  unsigned long long last;
  Hdr H;
  uint8_t raw[kHeaderBytes + kMaxStreams * kDirEntryBytes];
};
constexpr int kHdrCache = 16;
std::mutex g_hc_mu;
HdrCacheEntry g_hc[kHdrCache];
int g_nhc = 0;
unsigned long long g_hc_tick = 0;
}  // namespace

static bool hdr_cache_get(int dev, const void* ptr, size_t bytes, Hdr* H, uint8_t* raw,
                          size_t* nraw) {
  std::lock_guard<std::mutex> lk(g_hc_mu);
  for (int i = 0; i < g_nhc; i++) {
    HdrCacheEntry& e = g_hc[i];
    if (e.dev == dev && e.ptr == ptr && e.bytes == bytes) {
      e.last = ++g_hc_tick;
      *H = e.H;
      memcpy(raw, e.raw, e.nraw);
      *nraw = e.nraw;
      return true;
    }
  }
  return false;
}

static void hdr_cache_put(int dev, const void* ptr, size_t bytes, const Hdr& H, const uint8_t* raw,
                          size_t nraw) {
  std::lock_guard<std::mutex> lk(g_hc_mu);
  int slot = -1;
  for (int i = 0; i < g_nhc; i++)
    if (g_hc[i].dev == dev && g_hc[i].ptr == ptr && g_hc[i].bytes == bytes) slot = i;
  if (slot < 0 && g_nhc < kHdrCache) slot = g_nhc++;
  if (slot < 0) {
    slot = 0;
    for (int i = 1; i < g_nhc; i++)
      if (g_hc[i].last < g_hc[slot].last) slot = i;
  }
  HdrCacheEntry& e = g_hc[slot];
  e.dev = dev;
  e.ptr = ptr;
  e.bytes = bytes;
  e.H = H;
  e.nraw = nraw;
  memcpy(e.raw, raw, nraw);
  e.last = ++g_hc_tick;
}

// Captured decodes.  A plain decode seen twice with the same arguments and
// header bytes is captured as a graph on the second call and replayed from
// then on (one-off calls, such as random boxes, never pay for a capture).
namespace {
struct DecKey {
  int dev, level, whole;
  const void* comp;
  size_t comp_bytes;
  int64_t lo[3], hi[3];
  void* out;
  size_t out_cap;
  void* ws;
  size_t ws_bytes;
  size_t nraw;
  uint64_t rawhash;  // of the header bytes (compared first)
  uint8_t raw[STZ_HEADER_MAX_BYTES];
};
// equal keys: the small fields and the hash, then the header bytes
bool same_key(const DecKey& a, const DecKey& b) {
  return memcmp(&a, &b, offsetof(DecKey, raw)) == 0 && memcmp(a.raw, b.raw, a.nraw) == 0;
}
uint64_t hash_bytes(const uint8_t* p, size_t n) {  // FNV-1a over 8-byte words
  uint64_t h = 1469598103934665603ull;
  size_t i = 0;
  for (; i + 8 <= n; i += 8) {
    uint64_t w;
    memcpy(&w, p + i, 8);
    h = (h ^ w) * 1099511628211ull;
  }
  for (; i < n; i++) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}
struct DecGraph {
  DecKey key;
  cudaGraphExec_t exec;
  unsigned long long kernels, last;
};
struct DecSeen {
  DecKey key;
  unsigned long long last;
};
constexpr int kDecGraphs = 16, kDecSeen = 32;
std::mutex g_dg_mu;
DecGraph g_dg[kDecGraphs];  // captured decodes
DecSeen g_ds[kDecSeen];     // decodes seen once (keys only)
int g_ndg = 0, g_nds = 0;
unsigned long long g_dg_tick = 0;
}  // namespace

extern "C++" {
// This thread's side stream on the current device, with two events: a
// decode runs its finer streams' chunk decoding there beside level 1's
// passes.  Null when it cannot be created.
namespace {
struct Side {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
thread_local Side tl_side[64];
}  // namespace

static Side* side_stream() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  Side& sd = tl_side[dev];
  if (!sd.s) {
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
      if (st) cudaStreamDestroy(st);
      if (a) cudaEventDestroy(a);
      cudaGetLastError();
      return nullptr;
    }
    sd.s = st;
    sd.fork = a;
    sd.join = b;
  }
  return &sd;
}

template <typename F>
static int decode_graph_run(const DecKey& key, F& launch_all, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_dg_mu);
  const unsigned long long now = ++g_dg_tick;
  DecGraph* e = nullptr;
  for (int i = 0; i < g_ndg; i++)
    if (same_key(g_dg[i].key, key)) e = &g_dg[i];
  if (!e) {
    int seen = -1;
    for (int i = 0; i < g_nds; i++)
      if (same_key(g_ds[i].key, key)) seen = i;
    if (seen < 0) {  // first sight: remember the key, launch plainly
      int slot = 0;
      if (g_nds < kDecSeen) {
        slot = g_nds++;
      } else {
        for (int i = 1; i < kDecSeen; i++)
          if (g_ds[i].last < g_ds[slot].last) slot = i;
      }
      g_ds[slot].key = key;
      g_ds[slot].last = now;
      return launch_all(st, false);
    }
    // second sight: capture into the graph table
    g_ds[seen] = g_ds[--g_nds];
    int slot = 0;
    if (g_ndg < kDecGraphs) {
      slot = g_ndg++;
    } else {
      for (int i = 1; i < kDecGraphs; i++)
        if (g_dg[i].last < g_dg[slot].last) slot = i;
      if (g_dg[slot].exec) cudaGraphExecDestroy(g_dg[slot].exec);
    }
    e = &g_dg[slot];
    e->key = key;
    e->exec = nullptr;
    cudaStream_t& cap = g_cap_stream[key.dev];
    if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
      cap = nullptr;
      return STZ_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    int rc = cuda_ok(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    if (rc != STZ_OK) return rc;
    rc = launch_all(cap, true);
    const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    if (rc == STZ_OK && ce != cudaSuccess) rc = STZ_ERR_CUDA;
    if (rc == STZ_OK) {
      e->kernels = graph_kernels(graph);
      if (cudaGraphInstantiate(&e->exec, graph, 0) != cudaSuccess) {
        e->exec = nullptr;
        rc = STZ_ERR_CUDA;
      }
    }
    if (graph) cudaGraphDestroy(graph);
    if (rc != STZ_OK) {
      cudaGetLastError();
      memset(&e->key, 0, sizeof(DecKey));  // never matches (null container)
      return launch_all(st, false);        // capture failed: this call plainly
    }
  }
  e->last = now;
  if (cudaGraphLaunch(e->exec, st) != cudaSuccess) return STZ_ERR_CUDA;
  prof_count_launches(e->kernels);
  return STZ_OK;
}
}  // extern "C++"

// Options of a decode beyond the plain calls: a header parsed beforehand (no
// read-back from the device), a decoded level-1 grid to start from, and a
// device word that receives the status instead of a wait at the end.
struct DecOpts {
  const Hdr* hdr;
  const void* l1;
  uint32_t* status_out;
  bool no_cache;  // read the header back even when it is cached
  // allocate nothing on the host or the device: the header and the status
  // word come back by plain copies into this call's stack, the header cache
  // is not used, and the launches are never captured into a graph
  bool no_alloc;
};

static int decode_core(const void* comp_dev, size_t comp_bytes, const int64_t* lo_in,
                       const int64_t* hi_in, int level, int whole, void* out_dev, size_t out_cap,
                       int64_t* out_dims, void* ws_dev, size_t ws_bytes, cudaStream_t st,
                       const DecOpts& o) {
  const int level_in = level;
  if (!comp_dev || !out_dev || !ws_dev) return STZ_ERR_ARG;
  if (((uintptr_t)comp_dev % 8) || ((uintptr_t)ws_dev % 256)) return STZ_ERR_ARG;
  Hdr H;
  int rc = STZ_OK;
  // plain calls: the header from the cache (checked at the end), else read
  const size_t nraw = comp_bytes < (size_t)STZ_HEADER_MAX_BYTES ? comp_bytes
                                                                : (size_t)STZ_HEADER_MAX_BYTES;
  uint8_t raw[STZ_HEADER_MAX_BYTES];
  size_t nraw_cached = 0;
  int dev = -1;
  bool cached = false;
  if (o.hdr) {
    H = *o.hdr;
  } else if (o.no_alloc) {
    if (comp_bytes < (size_t)kHeaderBytes) return STZ_ERR_CORRUPT;
    if (cudaMemcpyAsync(raw, comp_dev, nraw, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return STZ_ERR_CUDA;
    rc = parse_hdr(raw, nraw, comp_bytes, &H);
  } else {
    if (cudaGetDevice(&dev) != cudaSuccess) return STZ_ERR_CUDA;
    cached = !o.no_cache && hdr_cache_get(dev, comp_dev, comp_bytes, &H, raw, &nraw_cached);
    if (!cached) {
      if (!comp_dev || comp_bytes < (size_t)kHeaderBytes) return STZ_ERR_CORRUPT;
      const uint8_t* h = nullptr;
      if ((rc = readback(comp_dev, (int)nraw, 0, st, &h)) != STZ_OK) return rc;
      if (cudaStreamSynchronize(st) != cudaSuccess) return STZ_ERR_CUDA;
      memcpy(raw, h, nraw);
      rc = parse_hdr(raw, nraw, comp_bytes, &H);
      if (rc == STZ_OK) hdr_cache_put(dev, comp_dev, comp_bytes, H, raw, nraw);
    }
  }
  if (rc != STZ_OK) return rc;
  // a return decided from a cached header before any launch: decide it again
  // from the header read back
#define STZ_EARLY(x)                                                                       \
  do {                                                                                     \
    if (cached) {                                                                          \
      DecOpts o2 = o;                                                                      \
      o2.no_cache = true;                                                                  \
      return decode_core(comp_dev, comp_bytes, lo_in, hi_in, level_in, whole, out_dev,     \
                         out_cap, out_dims, ws_dev, ws_bytes, st, o2);                     \
    }                                                                                      \
    return (x);                                                                            \
  } while (0)
  const bool have_l1 = o.l1 != nullptr;
  if (have_l1 && ((uintptr_t)o.l1 % (H.dtype == STZ_F32 ? 4 : 8))) STZ_EARLY(STZ_ERR_ARG);
  if (level == 0) level = H.L;
  if (level < 1 || level > H.L) STZ_EARLY(STZ_ERR_ARG);
  const size_t ps = H.dtype == STZ_F32 ? 4 : 8;
  if ((uintptr_t)out_dev % ps) STZ_EARLY(STZ_ERR_ARG);
  Geo g;
  make_geo(H.n, H.ndim, H.dtype, H.L, H.b, &g);
  int64_t lo[3] = {0, 0, 0}, hi[3] = {g.n[0], g.n[1], g.n[2]};
  if (!whole) {
    if (!lo_in || !hi_in) return STZ_ERR_ARG;
    if (H.ndim == 3) {
      for (int a = 0; a < 3; a++) {
        lo[a] = lo_in[a];
        hi[a] = hi_in[a];
      }
    } else {
      lo[1] = lo_in[0];
      hi[1] = hi_in[0];
      lo[2] = lo_in[1];
      hi[2] = hi_in[1];
    }
    for (int a = 0; a < 3; a++)
      if (lo[a] < 0 || hi[a] > g.n[a] || lo[a] >= hi[a]) STZ_EARLY(STZ_ERR_ARG);
  }
  DecPlan P;
  plan_decode(g, level, lo, hi, &P, have_l1);
  int64_t od[3];
  for (int a = 0; a < 3; a++) od[a] = imax(0, P.OB[a] - P.OA[a]);
  if (out_dims) {
    if (H.ndim == 3) {
      for (int a = 0; a < 3; a++) out_dims[a] = od[a];
    } else {
      out_dims[0] = od[1];
      out_dims[1] = od[2];
      out_dims[2] = 1;
    }
  }
  const int64_t npts = od[0] * od[1] * od[2];
  if (npts == 0) STZ_EARLY(STZ_OK);
  if ((size_t)npts * ps > out_cap) STZ_EARLY(STZ_ERR_CAPACITY);
  if (P.total > ws_bytes) STZ_EARLY(STZ_ERR_CAPACITY);
  uint8_t* ws = (uint8_t*)ws_dev;
  DevParams* dp = (DevParams*)(ws + P.dp);
  uint16_t* codes = (uint16_t*)(ws + P.codes);
  uint32_t* lut = (uint32_t*)(ws + P.lut);
  uint32_t* sub_olo = (uint32_t*)(ws + P.sub_olo);
  uint32_t* status = &dp->status;
  const uint8_t* comp = (const uint8_t*)comp_dev;
  // decode tables
  DecTables tb;
  memset(&tb, 0, sizeof(tb));
  for (int s = 0; s < H.ns; s++) {
    DecStream& d = tb.ds[s];
    SectHost sh = sect_host(H.d[s].nlive, H.d[s].nch, H.d[s].pw, H.d[s].nout, ps, H.nsub);
    d.sect = comp + H.d[s].sect_off;
    d.nlive = H.d[s].nlive;
    d.nchunks = H.d[s].nch;
    d.pw = H.d[s].pw;
    d.off_syms = sh.off_syms;
    d.off_lens = sh.off_lens;
    d.off_chunks = sh.off_chunks;
    d.off_subs = sh.off_subs;
    d.off_payload = sh.off_payload;
    d.nsub = H.nsub;
    d.nout = H.d[s].nout;
    d.off_opos = sh.off_opos;
    d.dense = dense_outliers(H.d[s].nout, H.d[s].nsym) ? 1 : 0;
  }
  const int ns_needed = 1 + 7 * (level - 1);
  int64_t nblocks = 0;
  double dec_bytes = 0.0;
  double job_bytes[kMaxStreams] = {};
  for (int s = have_l1 ? 1 : 0; s < ns_needed; s++) {
    if (g.s[s].nsym == 0) continue;
    const SlotMap& sm = P.sm[s];
    const int64_t c = sm.cnt[0] * sm.cnt[1] * sm.cnt[2];
    if (c == 0) continue;  // no point of this stream is needed: no table, no chunk
    tb.lut_sid[tb.nlut++] = s;
    DecChunkJob& jb = tb.jobs[tb.njobs++];
    jb.sid = s;
    for (int a = 0; a < 3; a++) {
      jb.lo[a] = sm.lo[a];
      jb.cnt[a] = sm.cnt[a];
    }
    jb.slot_base = sm.base;
    jb.nchunks_job = c;
    // the job's share of the stream's codes (written) and payload (read)
    if (H.d[s].nch > 0)
      job_bytes[tb.njobs - 1] = (2.0 * (double)H.d[s].nsym + 4.0 * (double)H.d[s].pw) *
                                (double)c / (double)H.d[s].nch;
    dec_bytes += job_bytes[tb.njobs - 1];
    jb.block0 = nblocks;
    nblocks += cdiv(c * H.nsub, kDecThreads);
  }
  tb.nblocks = nblocks;
#define STZ_TRY(x)               \
  do {                           \
    rc = (x);                    \
    if (rc != STZ_OK) return rc; \
  } while (0)
  // every launch of this decode, on stream st (no_coop: level 1 without the
  // cooperative launch, as inside a captured graph)
  auto launch_all = [&](cudaStream_t st, bool no_coop) -> int {
    static_assert(sizeof(DevParams) % 4 == 0, "DevParams is cleared in words");
    // the parameter words (status among them) are cleared by the table kernel
    if (tb.nlut > 0)
      STZ_TRY(launch_lut(tb, lut, (uint32_t*)dp, (int)(sizeof(DevParams) / 4), st));
    else
      STZ_TRY(zero_words(dp, (int64_t)(sizeof(DevParams) / 4), st));
    // Level 1's passes are a latency chain on a few SMs.  When the finer
    // streams' chunks make at least a full wave of the decoder, level 1's
    // chunks are decoded first and the finer ones on the side stream beside
    // level 1's passes, on a grid that leaves two SMs to them; the levels
    // above wait for both.
    Side* sd = nullptr;
    DecTables tb1, tbf;
    double b1 = 0.0, bf = 0.0;
    const int sms = launch_sms();
    if (!have_l1 && level >= 2) {
      tb1 = tb;
      tbf = tb;
      tb1.njobs = tbf.njobs = 0;
      tb1.nblocks = tbf.nblocks = 0;
      for (int q = 0; q < tb.njobs; q++) {
        DecTables& t = tb.jobs[q].sid == 0 ? tb1 : tbf;
        DecChunkJob jb = tb.jobs[q];
        jb.block0 = t.nblocks;
        t.nblocks += cdiv(jb.nchunks_job * H.nsub, kDecThreads);
        t.jobs[t.njobs++] = jb;
        (tb.jobs[q].sid == 0 ? b1 : bf) += job_bytes[q];
      }
      // (not for the no-allocation entry, which creates no stream)
      if (tb1.njobs > 0 && tbf.nblocks >= (int64_t)sms * decode_blocks_per_sm() && sms > 4 &&
          !o.no_alloc)
        sd = side_stream();
    }
    if (sd) {
      STZ_TRY(cuda_ok(cudaEventRecord(sd->fork, st)));
      STZ_TRY(launch_decode_chunks(g, tb1, lut, codes, sub_olo, status, b1, st));
      STZ_TRY(cuda_ok(cudaStreamWaitEvent(sd->s, sd->fork, 0)));
      STZ_TRY(launch_decode_chunks(g, tbf, lut, codes, sub_olo, status, bf, sd->s,
                                   (int64_t)(sms - 2) * decode_blocks_per_sm()));
      STZ_TRY(cuda_ok(cudaEventRecord(sd->join, sd->s)));
    } else {
      STZ_TRY(launch_decode_chunks(g, tb, lut, codes, sub_olo, status, dec_bytes, st));
    }
    const uint8_t* sec0 = comp + H.d[0].sect_off;
    SectHost sh0 = sect_host(H.d[0].nlive, H.d[0].nch, H.d[0].pw, H.d[0].nout, ps, H.nsub);
    uint8_t* g1buf = have_l1 ? (uint8_t*)o.l1 : ws + P.grid[1];
    if (!have_l1) {
      BaseArgs a;
      memset(&a, 0, sizeof(a));
      a.geo = g;
      a.dp = dp;
      a.g1 = g1buf;
      a.codes = codes;
      a.sm = P.sm[0];
      a.opos = (const uint32_t*)(sec0 + sh0.off_opos);
      a.oval = sec0 + sh0.off_oval;
      a.nout = (int64_t)H.d[0].nout;
      a.two_eb = H.two_eb[1];
      a.status = status;
      a.sub_olo = sub_olo;
      a.nsub = H.nsub;
      a.dense = tb.ds[0].dense;
      // the part of level 1 the output depends on: the output box itself, or
      // the coarse cells the level-2 box is predicted from
      int64_t m1[3];
      grid_extent(g.n, g.L, 1, m1);
      bool whole = true;
      for (int d = 0; d < 3; d++) {
        a.rlo[d] = level == 1 ? P.OA[d] : P.N1A[d];
        a.rhi[d] = level == 1 ? P.OB[d] : P.N1B[d];
        whole = whole && a.rlo[d] == 0 && a.rhi[d] == m1[d];
      }
      a.region = whole ? 0 : 1;
      STZ_TRY(no_coop ? launch_base_nocoop(a, true, st) : launch_base(a, true, st));
    }
    if (level == 1) {
      int64_t m1[3];
      grid_extent(g.n, g.L, 1, m1);
      const int blocks = (int)imin(cdiv(npts, 256), 4096);
      ProfScope ps_("k_copy_box", st);
      if (ps == 4)
        k_copy_box<float><<<blocks, 256, 0, st>>>((const float*)g1buf, (float*)out_dev, P.OA[0],
                                                  P.OA[1], P.OA[2], od[0], od[1], od[2], m1[1],
                                                  m1[2]);
      else
        k_copy_box<double><<<blocks, 256, 0, st>>>((const double*)g1buf, (double*)out_dev, P.OA[0],
                                                   P.OA[1], P.OA[2], od[0], od[1], od[2], m1[1],
                                                   m1[2]);
      STZ_TRY(cuda_ok(cudaGetLastError()));
    }
    if (sd) STZ_TRY(cuda_ok(cudaStreamWaitEvent(st, sd->join, 0)));
    for (int j = 2; j <= level; j++) {
      LevelArgs a;
      memset(&a, 0, sizeof(a));
      a.geo = g;
      a.level = j;
      a.pred = H.pred;
      a.dp = dp;
      a.coarse = (j == 2) ? (const void*)g1buf : (const void*)(ws + P.grid[j - 1]);
      a.fine = (j == level) ? out_dev : (void*)(ws + P.grid[j]);
      for (int d = 0; d < 3; d++) {
        a.clo[d] = P.A[j - 1][d];
        a.chi[d] = P.B[j - 1][d];
        a.flo[d] = P.A[j][d];
        a.fhi[d] = P.B[j][d];
        a.tlo[d] = P.tlo[j][d];
        a.tcnt[d] = P.tcnt[j][d];
      }
      a.codes = codes;
      for (int K = 1; K <= 7; K++) {
        const int sid = 1 + 7 * (j - 2) + K - 1;
        a.sm[K] = P.sm[sid];
        const uint8_t* sec = comp + H.d[sid].sect_off;
        SectHost sh = sect_host(H.d[sid].nlive, H.d[sid].nch, H.d[sid].pw, H.d[sid].nout, ps,
                                H.nsub);
        a.opos[K] = (const uint32_t*)(sec + sh.off_opos);
        a.oval[K] = sec + sh.off_oval;
        a.nout[K] = (int64_t)H.d[sid].nout;
      }
      a.two_eb = H.two_eb[j];
      a.status = status;
      a.sub_olo = sub_olo;
      a.nsub = H.nsub;
      for (int K = 1; K <= 7; K++) a.dense[K] = (uint8_t)tb.ds[1 + 7 * (j - 2) + K - 1].dense;
      STZ_TRY(launch_level(a, true, st));
    }
    return STZ_OK;
  };
  // plain calls repeated with the same arguments and header replay a graph
  if (!o.status_out && !o.hdr && !o.no_alloc && !prof_enabled()) {
    DecKey key;
    memset(&key, 0, sizeof(key));
    key.dev = dev;
    key.comp = comp_dev;
    key.comp_bytes = comp_bytes;
    key.level = level;
    key.whole = whole;
    for (int a = 0; a < 3; a++) {
      key.lo[a] = lo[a];
      key.hi[a] = hi[a];
    }
    key.out = out_dev;
    key.out_cap = out_cap;
    key.ws = ws_dev;
    key.ws_bytes = ws_bytes;
    key.nraw = nraw;
    key.rawhash = hash_bytes(raw, nraw);
    memcpy(key.raw, raw, nraw);
    STZ_TRY(decode_graph_run(key, launch_all, st));
  } else {
    STZ_TRY(launch_all(st, false));
  }
  if (o.status_out) {
    ProfScope ps_("k_readback", st);
    k_readback<<<1, 32, 0, st>>>((const uint8_t*)status, (uint8_t*)o.status_out, 4);
    STZ_TRY(cuda_ok(cudaGetLastError()));
    return STZ_OK;
  }
  if (o.no_alloc) {
    uint32_t hs = 0;
    STZ_TRY(cuda_ok(cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, st)));
    STZ_TRY(cuda_ok(cudaStreamSynchronize(st)));
    if (hs & kStatTimeout) return STZ_ERR_TIMEOUT;
    return (hs & kStatCorrupt) ? STZ_ERR_CORRUPT : STZ_OK;
  }
  // the status word, and for a cached header the header bytes beside it
  const uint8_t* hst = nullptr;
  const uint8_t* hhdr = nullptr;
  if (cached)
    STZ_TRY(readback2(status, 4, 0, comp_dev, (int)nraw, 64, st, &hst, &hhdr));
  else
    STZ_TRY(readback(status, 4, 0, st, &hst));
  STZ_TRY(cuda_ok(cudaStreamSynchronize(st)));
#undef STZ_TRY
  uint32_t hstat = 0;
  memcpy(&hstat, hst, 4);
  if (cached && (nraw != nraw_cached || memcmp(hhdr, raw, nraw) != 0)) {
    // another container at this address: decode again from its own header
    Hdr F;
    memcpy(raw, hhdr, nraw);
    rc = parse_hdr(raw, nraw, comp_bytes, &F);
    if (rc != STZ_OK) return rc;
    hdr_cache_put(dev, comp_dev, comp_bytes, F, raw, nraw);
    DecOpts o2 = o;
    o2.hdr = &F;
    return decode_core(comp_dev, comp_bytes, lo_in, hi_in, level, whole, out_dev, out_cap,
                       out_dims, ws_dev, ws_bytes, st, o2);
  }
  if (hstat & kStatTimeout) return STZ_ERR_TIMEOUT;
  return (hstat & kStatCorrupt) ? STZ_ERR_CORRUPT : STZ_OK;
#undef STZ_EARLY
}

static int decode_impl(const void* comp_dev, size_t comp_bytes, const int64_t* lo_in,
                       const int64_t* hi_in, int level, int whole, void* out_dev, size_t out_cap,
                       int64_t* out_dims, void* ws_dev, size_t ws_bytes, cudaStream_t st) {
  DecOpts o;
  memset(&o, 0, sizeof(o));
  return decode_core(comp_dev, comp_bytes, lo_in, hi_in, level, whole, out_dev, out_cap, out_dims,
                     ws_dev, ws_bytes, st, o);
}

// Box in the container's axis order (2D: y, x) to field coordinates (z, y, x).
static void box3(const Hdr& H, const int64_t* lo_in, const int64_t* hi_in, int64_t lo[3],
                 int64_t hi[3]) {
  if (H.ndim == 3) {
    for (int a = 0; a < 3; a++) {
      lo[a] = lo_in[a];
      hi[a] = hi_in[a];
    }
  } else {
    lo[0] = 0;
    hi[0] = 1;
    lo[1] = lo_in[0];
    hi[1] = hi_in[0];
    lo[2] = lo_in[1];
    hi[2] = hi_in[1];
  }
}

size_t stz_region_workspace_size(const void* hdr_host, size_t hdr_bytes, size_t comp_bytes,
                                 const int64_t* lo_in, const int64_t* hi_in, int level,
                                 int level1_given) {
  if (!hdr_host || !lo_in || !hi_in) return 0;
  Hdr H;
  if (parse_hdr((const uint8_t*)hdr_host, hdr_bytes, comp_bytes, &H) != STZ_OK) return 0;
  if (level < 1 || level > H.L) return 0;
  int64_t lo[3], hi[3];
  box3(H, lo_in, hi_in, lo, hi);
  Geo g;
  make_geo(H.n, H.ndim, H.dtype, H.L, H.b, &g);
  for (int a = 0; a < 3; a++)
    if (lo[a] < 0 || hi[a] > g.n[a] || lo[a] >= hi[a]) return 0;
  DecPlan P;
  plan_decode(g, level, lo, hi, &P, level1_given != 0);
  return P.total;
}

int stz_region_chunks(const void* hdr_host, size_t hdr_bytes, size_t comp_bytes,
                      const int64_t* lo_in, const int64_t* hi_in, int level, int level1_given,
                      int64_t* chunks, int max_streams) {
  if (!hdr_host || !lo_in || !hi_in || !chunks) return STZ_ERR_ARG;
  Hdr H;
  const int rc = parse_hdr((const uint8_t*)hdr_host, hdr_bytes, comp_bytes, &H);
  if (rc != STZ_OK) return rc;
  if (level < 1 || level > H.L || max_streams < H.ns) return STZ_ERR_ARG;
  int64_t lo[3], hi[3];
  box3(H, lo_in, hi_in, lo, hi);
  Geo g;
  make_geo(H.n, H.ndim, H.dtype, H.L, H.b, &g);
  for (int a = 0; a < 3; a++)
    if (lo[a] < 0 || hi[a] > g.n[a] || lo[a] >= hi[a]) return STZ_ERR_ARG;
  DecPlan P;
  plan_decode(g, level, lo, hi, &P, level1_given != 0);
  const int ns_needed = 1 + 7 * (level - 1);
  for (int s = 0; s < H.ns; s++) {
    const SlotMap& sm = P.sm[s];
    chunks[s] = (s < ns_needed && g.s[s].nsym > 0) ? sm.cnt[0] * sm.cnt[1] * sm.cnt[2] : 0;
  }
  return H.ns;
}

int stz_decompress_region_async(const void* comp_dev, size_t comp_bytes, const void* hdr_host,
                                size_t hdr_bytes, const void* level1_dev, const int64_t* lo,
                                const int64_t* hi, int level, void* out_dev, size_t out_cap,
                                int64_t* out_dims, void* ws_dev, size_t ws_bytes,
                                uint32_t* status_dev, void* stream) {
  if (!hdr_host || !status_dev || level < 1) return STZ_ERR_ARG;
  if ((uintptr_t)status_dev % 4) return STZ_ERR_ARG;
  Hdr H;
  const int rc = parse_hdr((const uint8_t*)hdr_host, hdr_bytes, comp_bytes, &H);
  if (rc != STZ_OK) return rc;
  DecOpts o;
  o.hdr = &H;
  o.l1 = level1_dev;
  o.status_out = status_dev;
  return decode_core(comp_dev, comp_bytes, lo, hi, level, 0, out_dev, out_cap, out_dims, ws_dev,
                     ws_bytes, (cudaStream_t)stream, o);
}

int stz_decompress_full(const void* comp_dev, size_t comp_bytes, void* out_dev, size_t out_cap,
                        void* ws_dev, size_t ws_bytes, void* stream) {
  return decode_impl(comp_dev, comp_bytes, nullptr, nullptr, 0, 1, out_dev, out_cap, nullptr,
                     ws_dev, ws_bytes, (cudaStream_t)stream);
}

int stz_decompress_progressive(const void* comp_dev, size_t comp_bytes, int level,
                               void* out_dev, size_t out_cap, int64_t* out_dims, void* ws_dev,
                               size_t ws_bytes, void* stream) {
  if (level < 1) return STZ_ERR_ARG;
  return decode_impl(comp_dev, comp_bytes, nullptr, nullptr, level, 1, out_dev, out_cap,
                     out_dims, ws_dev, ws_bytes, (cudaStream_t)stream);
}

int stz_decompress_region(const void* comp_dev, size_t comp_bytes, const int64_t* lo,
                          const int64_t* hi, int level, void* out_dev, size_t out_cap,
                          int64_t* out_dims, void* ws_dev, size_t ws_bytes, void* stream) {
  if (level < 1) return STZ_ERR_ARG;
  return decode_impl(comp_dev, comp_bytes, lo, hi, level, 0, out_dev, out_cap, out_dims, ws_dev,
                     ws_bytes, (cudaStream_t)stream);
}

// ------------------------------------------------------------ ROI selection
static int roi_geom(const int64_t* dims, int ndim, const int64_t* block, int64_t n[3],
                    int64_t b[3], int64_t* nunits) {
  if (!block || dims3(dims, ndim, n) != STZ_OK) return STZ_ERR_ARG;
  if (ndim == 3) {
    for (int a = 0; a < 3; a++) b[a] = block[a];
  } else {
    b[0] = 1;
    b[1] = block[0];
    b[2] = block[1];
  }
  int64_t nu = 1;
  for (int a = 0; a < 3; a++) {
    if (b[a] < 1) return STZ_ERR_ARG;
    nu *= cdiv(n[a], b[a]);
  }
  if (nu >= ((int64_t)1 << 31)) return STZ_ERR_ARG;
  *nunits = nu;
  return STZ_OK;
}

int64_t stz_roi_units(const int64_t* dims, int ndim, const int64_t* block) {
  int64_t n[3], b[3], nu;
  return roi_geom(dims, ndim, block, n, b, &nu) == STZ_OK ? nu : -1;
}

size_t stz_roi_workspace_size(const int64_t* dims, int ndim, const int64_t* block) {
  int64_t n[3], b[3], nu;
  if (roi_geom(dims, ndim, block, n, b, &nu) != STZ_OK) return 0;
  return 3 * al256(8 * (size_t)nu) + 256;
}

int stz_roi_select(const void* field_dev, const int64_t* dims, int ndim, stz_dtype dtype,
                   const int64_t* block, stz_roi_metric metric, stz_roi_mode mode, double value,
                   int64_t* sel_dev, size_t sel_cap, double* metric_dev, int64_t* nsel,
                   void* ws_dev, size_t ws_bytes, void* stream) {
  int64_t n[3], b[3], nu;
  if (roi_geom(dims, ndim, block, n, b, &nu) != STZ_OK) return STZ_ERR_ARG;
  if (dtype != STZ_F32 && dtype != STZ_F64) return STZ_ERR_ARG;
  if (metric != STZ_ROI_RANGE && metric != STZ_ROI_MAX) return STZ_ERR_ARG;
  if (mode != STZ_ROI_THRESHOLD && mode != STZ_ROI_TOP) return STZ_ERR_ARG;
  if (mode == STZ_ROI_TOP && !(value > 0.0 && value <= 1.0)) return STZ_ERR_ARG;
  if (!field_dev || !sel_dev || !nsel || !ws_dev) return STZ_ERR_ARG;
  const size_t ps = dtype == STZ_F32 ? 4 : 8;
  if (((uintptr_t)field_dev % ps) || ((uintptr_t)sel_dev % 8) || ((uintptr_t)ws_dev % 256) ||
      (metric_dev && ((uintptr_t)metric_dev % 8)))
    return STZ_ERR_ARG;
  if (sel_cap < (size_t)nu || ws_bytes < stz_roi_workspace_size(dims, ndim, block))
    return STZ_ERR_CAPACITY;
  int64_t k = 0;
  if (mode == STZ_ROI_TOP) {
    k = (int64_t)ceil(value * (double)nu);
    if (k > nu) k = nu;
  }
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* ws = (uint8_t*)ws_dev;
  const size_t a = al256(8 * (size_t)nu);
  unsigned long long* kmin = (unsigned long long*)ws;
  unsigned long long* kmax = (unsigned long long*)(ws + a);
  unsigned long long* mkey = (unsigned long long*)(ws + 2 * a);
  unsigned long long* cnt = (unsigned long long*)(ws + 3 * a);
  int rc = launch_roi(field_dev, dtype, n, b, metric, mode, value, k, kmin, kmax, mkey, metric_dev,
                      sel_dev, cnt, st);
  if (rc != STZ_OK) return rc;
  const uint8_t* h = nullptr;
  if ((rc = readback(cnt, 8, 0, st, &h)) != STZ_OK) return rc;
  if ((rc = cuda_ok(cudaStreamSynchronize(st))) != STZ_OK) return rc;
  unsigned long long c;
  memcpy(&c, h, 8);
  *nsel = (int64_t)c;
  return STZ_OK;
}

// ---------------------------------------------------------- batched serving
// decode-side description of stream s of a parsed container
static void dec_stream(const Hdr& H, const uint8_t* comp, int s, DecStream* d) {
  const size_t ps = H.dtype == STZ_F32 ? 4 : 8;
  SectHost sh = sect_host(H.d[s].nlive, H.d[s].nch, H.d[s].pw, H.d[s].nout, ps, H.nsub);
  memset(d, 0, sizeof(*d));
  d->sect = comp + H.d[s].sect_off;
  d->nlive = H.d[s].nlive;
  d->nchunks = H.d[s].nch;
  d->pw = H.d[s].pw;
  d->off_syms = sh.off_syms;
  d->off_lens = sh.off_lens;
  d->off_chunks = sh.off_chunks;
  d->off_subs = sh.off_subs;
  d->off_payload = sh.off_payload;
  d->nsub = H.nsub;
  d->nout = H.d[s].nout;
  d->off_opos = sh.off_opos;
  d->dense = dense_outliers(H.d[s].nout, H.d[s].nsym) ? 1 : 0;
}

size_t stz_decode_tables_size(const void* hdr_host, size_t hdr_bytes, size_t comp_bytes) {
  Hdr H;
  if (!hdr_host || parse_hdr((const uint8_t*)hdr_host, hdr_bytes, comp_bytes, &H) != STZ_OK)
    return 0;
  return sizeof(uint32_t) * (size_t)kLutSize * (size_t)H.ns;
}

int stz_decode_tables(const void* comp_dev, size_t comp_bytes, const void* hdr_host,
                      size_t hdr_bytes, void* tables_dev, size_t tables_bytes, void* stream) {
  if (!comp_dev || !hdr_host || !tables_dev || ((uintptr_t)tables_dev % 16)) return STZ_ERR_ARG;
  Hdr H;
  const int rc = parse_hdr((const uint8_t*)hdr_host, hdr_bytes, comp_bytes, &H);
  if (rc != STZ_OK) return rc;
  if (tables_bytes < sizeof(uint32_t) * (size_t)kLutSize * (size_t)H.ns) return STZ_ERR_CAPACITY;
  Geo g;
  make_geo(H.n, H.ndim, H.dtype, H.L, H.b, &g);
  DecTables tb;
  memset(&tb, 0, sizeof(tb));
  for (int s = 0; s < H.ns; s++) {
    dec_stream(H, (const uint8_t*)comp_dev, s, &tb.ds[s]);
    if (g.s[s].nsym > 0) tb.lut_sid[tb.nlut++] = s;
  }
  if (tb.nlut == 0) return STZ_OK;
  return launch_lut(tb, (uint32_t*)tables_dev, nullptr, 0, (cudaStream_t)stream);
}


namespace {
// The plan of one stz_decode_requests call: parsed fields, per-request decode
// plans and boxes, and the workspace layout (argument arenas, then one region
// per request decoded beyond level 1).
struct BatchPlan {
  std::vector<Hdr> H;
  std::vector<Geo> G;
  std::vector<DecPlan> P;
  std::vector<int64_t> npts;
  std::vector<size_t> req_off;
  int maxlevel = 1, dtype = 0, njobs = 0, ncopy = 0;
  size_t o_jobs = 0, o_copy = 0, o_level[kMaxLevels + 1] = {}, total = 0;
};
}  // namespace

static int plan_batch(int n, stz_region_request* reqs, const stz_served_field* fields, int nf,
                      BatchPlan* B) {
  if (n < 1 || nf < 1 || !reqs || !fields) return STZ_ERR_ARG;
  B->H.resize(nf);
  B->G.resize(nf);
  for (int f = 0; f < nf; f++) {
    const stz_served_field& F = fields[f];
    if (!F.comp_dev || !F.hdr_host || !F.level1_dev || !F.tables_dev) return STZ_ERR_ARG;
    if ((uintptr_t)F.comp_dev % 8) return STZ_ERR_ARG;
    const int rc = parse_hdr((const uint8_t*)F.hdr_host, F.hdr_bytes, F.comp_bytes, &B->H[f]);
    if (rc != STZ_OK) return rc;
    const Hdr& H = B->H[f];
    if (f == 0) B->dtype = H.dtype;
    if (H.dtype != B->dtype) return STZ_ERR_ARG;
    if ((uintptr_t)F.level1_dev % (H.dtype == STZ_F32 ? 4 : 8)) return STZ_ERR_ARG;
    make_geo(H.n, H.ndim, H.dtype, H.L, H.b, &B->G[f]);
  }
  const size_t ps = B->dtype == STZ_F32 ? 4 : 8;
  B->P.resize(n);
  B->npts.assign(n, 0);
  B->req_off.assign(n, 0);
  int nlev[kMaxLevels + 1] = {};
  for (int i = 0; i < n; i++) {
    stz_region_request& r = reqs[i];
    if (r.field < 0 || r.field >= nf) return STZ_ERR_ARG;
    const Hdr& H = B->H[r.field];
    const Geo& g = B->G[r.field];
    if (r.level < 1 || r.level > H.L || !r.out_dev || ((uintptr_t)r.out_dev % ps))
      return STZ_ERR_ARG;
    int64_t lo[3], hi[3];
    box3(H, r.lo, r.hi, lo, hi);
    for (int a = 0; a < 3; a++)
      if (lo[a] < 0 || hi[a] > g.n[a] || lo[a] >= hi[a]) return STZ_ERR_ARG;
    DecPlan& P = B->P[i];
    plan_decode(g, r.level, lo, hi, &P, true);
    int64_t od[3];
    for (int a = 0; a < 3; a++) od[a] = imax(0, P.OB[a] - P.OA[a]);
    if (H.ndim == 3) {
      for (int a = 0; a < 3; a++) r.out_dims[a] = od[a];
    } else {
      r.out_dims[0] = od[1];
      r.out_dims[1] = od[2];
      r.out_dims[2] = 1;
    }
    B->npts[i] = od[0] * od[1] * od[2];
    if ((size_t)B->npts[i] * ps > r.out_cap) return STZ_ERR_CAPACITY;
    if (B->npts[i] == 0) continue;
    if (r.level == 1) {
      B->ncopy++;
      continue;
    }
    B->maxlevel = r.level > B->maxlevel ? r.level : B->maxlevel;
    B->njobs += 7 * (r.level - 1);
    for (int j = 2; j <= r.level; j++) nlev[j]++;
  }
  size_t o = 0;
  B->o_jobs = o;
  o += al256(sizeof(DecJobMulti) * (size_t)(B->njobs > 0 ? B->njobs : 1));
  B->o_copy = o;
  o += al256(sizeof(CopyJob) * (size_t)(B->ncopy > 0 ? B->ncopy : 1));
  for (int j = 2; j <= B->maxlevel; j++) {
    B->o_level[j] = o;
    o += al256(level_multi_arena_bytes(nlev[j]));
  }
  for (int i = 0; i < n; i++) {
    if (B->npts[i] == 0 || reqs[i].level == 1) continue;
    B->req_off[i] = o;
    o += al256(B->P[i].total);
  }
  B->total = o;
  return STZ_OK;
}

size_t stz_decode_requests_workspace(int n, const stz_region_request* reqs,
                                     const stz_served_field* fields, int nfields) {
  if (n < 1 || !reqs) return 0;
  std::vector<stz_region_request> copy(reqs, reqs + n);  // out_dims are written
  BatchPlan B;
  return plan_batch(n, copy.data(), fields, nfields, &B) == STZ_OK ? B.total : 0;
}

int stz_decode_requests(int n, stz_region_request* reqs, const stz_served_field* fields,
                        int nfields, void* ws_dev, size_t ws_bytes, uint32_t* status_dev,
                        void* stream) {
  if (!ws_dev || !status_dev || ((uintptr_t)ws_dev % 256) || ((uintptr_t)status_dev % 4))
    return STZ_ERR_ARG;
  BatchPlan B;
  int rc = plan_batch(n, reqs, fields, nfields, &B);
  if (rc != STZ_OK) return rc;
  if (B.total > ws_bytes) return STZ_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* ws = (uint8_t*)ws_dev;
  const size_t ps = B.dtype == STZ_F32 ? 4 : 8;
  // every request's status word starts at zero; the kernels OR into it
  if ((rc = zero_words(status_dev, n, st)) != STZ_OK) return rc;
  // chunk jobs of all requests, and the level-1 copies
  std::vector<DecJobMulti> jobs;
  std::vector<CopyJob> copies;
  jobs.reserve(B.njobs);
  int64_t nblocks = 0, copy_max = 0;
  double dec_bytes = 0.0;
  for (int i = 0; i < n; i++) {
    const stz_region_request& r = reqs[i];
    if (B.npts[i] == 0) continue;
    const stz_served_field& F = fields[r.field];
    const Hdr& H = B.H[r.field];
    const Geo& g = B.G[r.field];
    const DecPlan& P = B.P[i];
    if (r.level == 1) {
      int64_t m1[3];
      grid_extent(g.n, g.L, 1, m1);
      CopyJob c;
      c.src = F.level1_dev;
      c.dst = r.out_dev;
      for (int a = 0; a < 3; a++) {
        c.a[a] = P.OA[a];
        c.e[a] = P.OB[a] - P.OA[a];
      }
      c.m1 = m1[1];
      c.m2 = m1[2];
      copies.push_back(c);
      copy_max = imax(copy_max, B.npts[i]);
      continue;
    }
    uint8_t* base = ws + B.req_off[i];
    for (int sid = 1; sid < 1 + 7 * (r.level - 1); sid++) {
      if (g.s[sid].nsym == 0) continue;
      const SlotMap& sm = P.sm[sid];
      const int64_t c = sm.cnt[0] * sm.cnt[1] * sm.cnt[2];
      if (c == 0) continue;
      DecJobMulti m;
      memset(&m, 0, sizeof(m));
      m.job.sid = sid;
      for (int a = 0; a < 3; a++) {
        m.job.lo[a] = sm.lo[a];
        m.job.cnt[a] = sm.cnt[a];
        m.b[a] = g.b[a];
      }
      m.job.slot_base = sm.base;
      m.job.nchunks_job = c;
      m.job.block0 = nblocks;
      nblocks += cdiv(c * H.nsub, kDecThreads);
      dec_stream(H, (const uint8_t*)F.comp_dev, sid, &m.ds);
      m.sg = g.s[sid];
      m.bvol = g.bvol;
      m.lut = (const uint32_t*)F.tables_dev + (int64_t)sid * kLutSize;
      m.codes = (uint16_t*)(base + P.codes);
      m.sub_olo = (uint32_t*)(base + P.sub_olo);
      m.status = status_dev + i;
      if (H.d[sid].nch > 0)
        dec_bytes += (2.0 * (double)H.d[sid].nsym + 4.0 * (double)H.d[sid].pw) * (double)c /
                     (double)H.d[sid].nch;
      jobs.push_back(m);
    }
  }
#define STZ_TRY(x)               \
  do {                           \
    rc = (x);                    \
    if (rc != STZ_OK) return rc; \
  } while (0)
  if (!copies.empty()) {
    CopyJob* dcopy = (CopyJob*)(ws + B.o_copy);
    STZ_TRY(cuda_ok(cudaMemcpyAsync(dcopy, copies.data(), sizeof(CopyJob) * copies.size(),
                                    cudaMemcpyHostToDevice, st)));
    const dim3 grid((unsigned)imin(cdiv(copy_max, 256), 256), (unsigned)copies.size());
    ProfScope ps_("k_copy_box", st);
    if (ps == 4) k_copy_boxes<float><<<grid, 256, 0, st>>>(dcopy);
    else k_copy_boxes<double><<<grid, 256, 0, st>>>(dcopy);
    STZ_TRY(cuda_ok(cudaGetLastError()));
  }
  if (!jobs.empty()) {
    DecJobMulti* djobs = (DecJobMulti*)(ws + B.o_jobs);
    STZ_TRY(cuda_ok(cudaMemcpyAsync(djobs, jobs.data(), sizeof(DecJobMulti) * jobs.size(),
                                    cudaMemcpyHostToDevice, st)));
    STZ_TRY(launch_decode_chunks_multi(djobs, (int)jobs.size(), nblocks, dec_bytes, st));
  }
  // each finer level of every request: one launch of each level kernel
  std::vector<LevelArgs> la;
  for (int j = 2; j <= B.maxlevel; j++) {
    la.clear();
    for (int i = 0; i < n; i++) {
      const stz_region_request& r = reqs[i];
      if (B.npts[i] == 0 || r.level < j) continue;
      const stz_served_field& F = fields[r.field];
      const Hdr& H = B.H[r.field];
      const DecPlan& P = B.P[i];
      uint8_t* base = ws + B.req_off[i];
      LevelArgs a;
      memset(&a, 0, sizeof(a));
      a.geo = B.G[r.field];
      a.level = j;
      a.pred = H.pred;
      a.dp = (const DevParams*)(base + P.dp);
      a.coarse = j == 2 ? F.level1_dev : (const void*)(base + P.grid[j - 1]);
      a.fine = j == r.level ? r.out_dev : (void*)(base + P.grid[j]);
      for (int d = 0; d < 3; d++) {
        a.clo[d] = P.A[j - 1][d];
        a.chi[d] = P.B[j - 1][d];
        a.flo[d] = P.A[j][d];
        a.fhi[d] = P.B[j][d];
        a.tlo[d] = P.tlo[j][d];
        a.tcnt[d] = P.tcnt[j][d];
      }
      a.codes = (uint16_t*)(base + P.codes);
      for (int K = 1; K <= 7; K++) {
        const int sid = 1 + 7 * (j - 2) + K - 1;
        a.sm[K] = P.sm[sid];
        const uint8_t* sec = (const uint8_t*)F.comp_dev + H.d[sid].sect_off;
        SectHost sh = sect_host(H.d[sid].nlive, H.d[sid].nch, H.d[sid].pw, H.d[sid].nout, ps,
                                H.nsub);
        a.opos[K] = (const uint32_t*)(sec + sh.off_opos);
        a.oval[K] = sec + sh.off_oval;
        a.nout[K] = (int64_t)H.d[sid].nout;
        a.dense[K] = dense_outliers(H.d[sid].nout, H.d[sid].nsym) ? 1 : 0;
      }
      a.two_eb = H.two_eb[j];
      a.status = status_dev + i;
      a.sub_olo = (const uint32_t*)(base + P.sub_olo);
      a.nsub = H.nsub;
      if (level_multi_ok(a)) la.push_back(a);
      else STZ_TRY(launch_level(a, true, st));  // other bricks or predictors: on its own
    }
    if (!la.empty()) STZ_TRY(launch_level_multi(la.data(), (int)la.size(), ws + B.o_level[j], st));
  }
#undef STZ_TRY
  return STZ_OK;
}

// ------------------------------------------------ region decode, no allocation
// The scratch of stz_decompress_region_noalloc: one file-scope array in the
// library's device memory.  Host code sees only a host-side stand-in under
// this name, so its device address is looked up per device (with that
// device current) and passed to the kernels like any workspace.
static __device__ __align__(256) unsigned char g_noalloc_scratch[STZ_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices];
}  // namespace

static int noalloc_scratch(void** ptr) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return STZ_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return STZ_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *ptr = g_noalloc_ptr[dev];
  return STZ_OK;
}

int stz_decompress_region_noalloc(const void* comp_dev, size_t comp_bytes, const int64_t* lo,
                                  const int64_t* hi, int level, void* out_dev, size_t out_cap,
                                  int64_t* out_dims, void* stream) {
  if (level < 1) return STZ_ERR_ARG;
  void* ws = nullptr;
  const int rc = noalloc_scratch(&ws);
  if (rc != STZ_OK) return rc;
  // decode_core rejects a plan larger than the array before it queues work
  // and clears the device parameters (status word) at its start
  DecOpts o;
  memset(&o, 0, sizeof(o));
  o.no_alloc = true;
  return decode_core(comp_dev, comp_bytes, lo, hi, level, 0, out_dev, out_cap, out_dims, ws,
                     STZ_NOALLOC_SCRATCH_BYTES, (cudaStream_t)stream, o);
}

}  // extern "C"
