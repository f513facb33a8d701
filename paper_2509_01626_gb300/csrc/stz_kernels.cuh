// stz_kernels.cuh -- host-side launchers of the STZ kernels (one .cu each).
#pragma once

#include <cuda.h>

#include <vector>

#include "stz_common.cuh"

namespace stz {

// ---- stz_range.cu: value range and error-bound constants ----
// Per-block min / max keys over the finite values of the field (n = 0: none)
// into part[2 b], part[2 b + 1], b < *nparts (at most kRangeMaxBlocks); the
// same launch zero-fills the word ranges (z0, nz0) and (z1, nz1).
constexpr int kRangeMaxBlocks = 2048;
int launch_range(const void* field, int dtype, int64_t n, unsigned long long* part, int* nparts,
                 uint32_t* z0, int64_t nz0, uint32_t* z1, int64_t nz1, cudaStream_t s);
// Reduces the range partials (relative mode) and writes the whole of *dp:
// range, eb_abs, per-level bounds (eb_l = eb_abs / ratio^(L-l), the power
// formed by repeated multiplication), quantizer constants, the predictor
// and status 0.
int launch_params(DevParams* dp, const unsigned long long* part, int nparts, int dtype,
                  int eb_mode, double eb, int L, int R, double ratio, int pred,
                  cudaStream_t s);

// ---- stz_base.cu: level 1 (SZ3-style axis passes) ----
struct BaseArgs {
  Geo geo;
  const DevParams* dp;
  const void* field;          // compress: the input field
  void* g1;                   // level-1 grid (compact), reconstruction
  uint16_t* codes;            // code buffer (slots)
  uint32_t* chunk_outliers;   // compress: outliers per chunk (global chunk index)
  SlotMap sm;                 // slots of stream 0
  const uint32_t* opos;       // decode: outliers of stream 0
  const void* oval;
  int64_t nout;
  double two_eb;              // decode: 2 eb_1 in the field precision
  uint32_t* status;           // decode: corrupt flag
  const uint32_t* sub_olo;    // decode: first outlier index per (slot, sub-chunk)
  int nsub;                   // decode: sub-chunks per chunk
  int dense;                  // decode: sub_olo holds stream 0's ranges
  int region;                 // decode: only the box [rlo, rhi) of the level-1 grid is needed
  int64_t rlo[3], rhi[3];
};
int launch_base(const BaseArgs& a, bool decode, cudaStream_t s);
// the coarse single-block phase, then one plain launch per remaining pass (no
// cooperative launch: for graphs whose branches run concurrently)
int launch_base_nocoop(const BaseArgs& a, bool decode, cudaStream_t s);

// ---- stz_level.cu: levels 2..L (multi-dimensional cubic prediction) ----
struct LevelArgs {
  Geo geo;
  int level;                  // l >= 2
  int pred;                   // kPredCubic / kPredLinear / kPredDirect
  const DevParams* dp;
  const void* field;          // compress: input field
  const void* coarse;         // G_{l-1} reconstruction, box [clo, chi)
  int64_t clo[3], chi[3];
  void* fine;                 // G_l output, box [flo, fhi); may be null (compress, l = L)
  int64_t flo[3], fhi[3];
  uint16_t* codes;
  uint32_t* chunk_outliers;   // compress
  uint32_t* hist;             // compress: histograms of the 7 streams (2R bins each)
  SlotMap sm[8];              // index = sub-block 1..7
  const uint32_t* opos[8];    // decode: outliers per sub-block stream
  const void* oval[8];
  int64_t nout[8];
  double two_eb;              // decode
  uint32_t* status;
  const uint32_t* sub_olo;    // decode: first outlier index per (slot, sub-chunk)
  int nsub;                   // decode: sub-chunks per chunk
  uint8_t dense[8];           // decode: sub_olo holds sub-block K's ranges
  int64_t tlo[3], tcnt[3];    // tiles (bricks of cells) to process
};
int launch_level(const LevelArgs& a, bool decode, cudaStream_t s);
// The decode of level a.level for many requests in one launch of each of the
// interior and boundary kernels (the batched served form).  Every request
// must pass level_multi_ok and share the level and dtype.  arena_dev: device
// memory of level_multi_arena_bytes(n) bytes that receives the arguments (a
// copy queued on s; the host array may be reused on return).
bool level_multi_ok(const LevelArgs& a);
size_t level_multi_arena_bytes(int n);
int launch_level_multi(const LevelArgs* h, int n, uint8_t* arena_dev, cudaStream_t s);

// The level stages (2..L) of many fields of one dtype in one persistent
// launch over (field, level, tile) work items (the batched form of
// compression).  h[r]: the compress arguments of one (field, level) group;
// every group passes level_queue_ok, and a group of level l > 2 has its
// field's level l-1 among the others (same code buffer).  schedule: 0 every
// field's level 2 first, then level 3, ...; 1 field by field in the order of
// h.  gran: interior tiles per work item (1..64).  blocks_per_sm: 0 for the
// occupancy limit.  arena_dev: 256-byte aligned device memory of
// level_queue_arena_bytes(n) bytes.  plan_level_queue fills the plan on the
// host; write_level_queue queues the copy of its arguments into the arena
// (not inside a stream capture: the source is pageable); run_level_queue
// zeroes the queue's counters and launches the kernel (capturable).
struct ShellGeo;
struct QueueGroup {
  int64_t ntile;   // interior tiles of the group (0: none)
  int64_t nshell;  // boundary cells
  uint32_t items;  // work items: ceil(ntile / gran) + ceil(nshell / 256)
  int dep;         // the group whose items must all be done first (-1: none)
  int pair, vec;   // fast_tile's paired accesses; 16-byte tile copies
  int tma;         // the coarse tile by one TMA copy (tensor map tmaps[group])
};
struct QueueSeg {
  int64_t first;  // first work item
  int group;
  int kind;       // 0: interior tiles, 1: boundary cells
};
struct LevelQueue {
  const LevelArgs* args;
  const ShellGeo* shs;
  const QueueGroup* groups;
  const QueueSeg* segs;
  const CUtensorMap* tmaps;   // per group (used where groups[g].tma)
  int nseg;
  uint32_t* done;             // completed items per group
  unsigned long long* claim;  // next item to claim
  uint32_t* abort;            // set by a block whose wait ran out
  int64_t total;
  int gran;
};
struct LevelQueuePlan {
  std::vector<uint8_t> buf;  // the arena's contents
  uint8_t* arena;
  void* counters;            // the words run_level_queue zeroes
  int64_t counter_words;
  LevelQueue qa;
  size_t smem;
  int64_t grid;              // 0: nothing to do
  bool f64;
  double bytes;
};
bool level_queue_ok(const LevelArgs& a);
size_t level_queue_arena_bytes(int n);
int plan_level_queue(const LevelArgs* h, int n, int schedule, int gran, int blocks_per_sm,
                     uint8_t* arena_dev, LevelQueuePlan* P);
int write_level_queue(const LevelQueuePlan& P, cudaStream_t s);
int run_level_queue(const LevelQueuePlan& P, cudaStream_t s);

// ---- stz_huffman.cu: histograms, codebooks, chunk coding ----
// histogram of stream 0 from its slots
int launch_stream_hist(const Geo& g, int sid, const uint16_t* codes, uint32_t* hist,
                       cudaStream_t s);
// codebook per stream: enc[s][sym] = code << 4 | len; book = nlive, syms, lens
struct BookDev {
  uint32_t nlive;
  uint16_t sym[kAlphabet];
  uint8_t len[kAlphabet];
};
// the codebooks of streams s0 .. s0 + ns - 1 (ns < 0: through the last)
int launch_codebook(const Geo& g, const uint32_t* hist, uint16_t* enc, BookDev* books,
                    cudaStream_t s, int s0 = 0, int ns = -1);
// payload words per chunk, and the bits of each 64-symbol lane run of a chunk
// (32 u16 per chunk) for the packing pass
int launch_chunk_words(const Geo& g, const uint16_t* codes, const uint16_t* enc,
                       uint32_t* chunk_words, uint16_t* lane_bits, cudaStream_t s);
// exclusive scans of two n-entry u32 arrays into (n+1)-entry u64 arrays;
// sums: 2 * ceil(n / 4096) scratch entries
int launch_scan2(const uint32_t* a, const uint32_t* b, int64_t n, unsigned long long* sums,
                 unsigned long long* oa, unsigned long long* ob, cudaStream_t s);
// pack every chunk's codes into the container payload and list its outliers
struct SectDev;  // stz_container.cu
int launch_pack(const Geo& g, const uint16_t* codes, const uint16_t* enc,
                const uint16_t* lane_bits, const unsigned long long* word_off,
                const SectDev* sect, uint8_t* out,
                const DevParams* dp, const void* field, const uint32_t* chunk_outliers,
                const unsigned long long* out_off, cudaStream_t s);

// decode tables: lut[s][i] = sym | len << 11 for the top-12-bit window i
// (len 0: no code starts with i)
struct DecStream {
  const uint8_t* sect;        // section start in the container
  uint64_t nlive, nchunks, pw, nout;
  int dense;                  // sub_olo ranges recorded (dense_outliers)
  uint64_t off_syms, off_lens, off_chunks, off_subs, off_payload, off_opos;
  int nsub;
};
// entropy-decode the chunks of bricks [lo, lo+cnt) of each stream into slots
struct DecChunkJob {
  int sid;                    // stream
  int64_t lo[3], cnt[3];      // brick range
  int64_t slot_base;          // slot index of the first brick
  int64_t nchunks_job;        // cnt0*cnt1*cnt2
  int64_t block0;             // first thread block of this job
};
struct DecTables {
  DecStream ds[kMaxStreams];  // indexed by stream
  int lut_sid[kMaxStreams];   // streams whose decode table is built
  int nlut;
  DecChunkJob jobs[kMaxStreams];
  int njobs;
  int64_t nblocks;            // thread blocks of the chunk decoder
};
// decode tables of the streams tb.lut_sid[0 .. nlut) (nlut > 0); block 0 also
// zero-fills the nclear words at clear
int launch_lut(const DecTables& tb, uint32_t* lut, uint32_t* clear, int nclear,
               cudaStream_t s);
// bytes: the launch's algorithmic bytes (payload read, codes written).
// For streams with outliers, sub_olo[slot * (kNSub + 1) + u] receives where
// sub-chunk u of each decoded chunk starts in the stream's outlier list
// (u = nsub: where the chunk ends).
// max_grid > 0: at most that many thread blocks, striding over the work
int launch_decode_chunks(const Geo& g, const DecTables& tb, const uint32_t* lut,
                         uint16_t* codes, uint32_t* sub_olo, uint32_t* status, double bytes,
                         cudaStream_t s, int64_t max_grid = 0);
// blocks of the chunk decoder resident per SM
int decode_blocks_per_sm();

// Chunk jobs of many decodes in one launch (the batched served form); jobs
// in device memory, ascending block0, each with its own table and outputs.
struct DecJobMulti {
  DecChunkJob job;
  DecStream ds;
  StreamGeo sg;
  int32_t b[3];
  int64_t bvol;
  const uint32_t* lut;        // the stream's decode table (kLutSize entries)
  uint16_t* codes;
  uint32_t* sub_olo;
  uint32_t* status;
};
int launch_decode_chunks_multi(const DecJobMulti* jobs_dev, int njobs, int64_t nblocks,
                               double bytes, cudaStream_t s);

// ---- stz_container.cu: layout, header, sections, outliers ----
struct SectDev {
  unsigned long long sect_off, off_syms, off_lens, off_chunks, off_subs, off_payload, off_opos,
      off_oval, size;
  unsigned long long pw, nout, nlive, word0, out0;
};
struct LayoutDev {
  unsigned long long total;
  SectDev s[kMaxStreams];
};
int launch_layout(const Geo& g, const DevParams* dp, int eb_mode,
                  const unsigned long long* word_off, const unsigned long long* out_off,
                  const BookDev* books, LayoutDev* lay, uint8_t* out, size_t cap,
                  cudaStream_t s);
int launch_sections(const Geo& g, const LayoutDev* lay, const BookDev* books,
                    const unsigned long long* word_off, const DevParams* dp, uint8_t* out,
                    cudaStream_t s);

// ---- stz_api.cu: one compression as a queue of launches ----
struct CompressJob {
  Geo g;
  const void* field;
  int eb_mode;
  double eb;
  int pred;          // predictor of levels 2..L
  double eb_ratio;   // adaptive-bound ratio
  void* out;
  size_t out_cap;
  void* ws;
};
// device words a queued compression leaves behind
struct CompressDev {
  const unsigned long long* total;          // container bytes
  const unsigned long long* payload_words;  // payload words of all chunks
  const uint32_t* status;                   // kStat* bits
  const unsigned long long* result;         // the three above, gathered (k_result)
};
int compress_check(const void* field_dev, const int64_t* dims, int ndim, int dtype, int eb_mode,
                   double eb, void* out_dev, size_t out_cap, void* ws_dev, size_t ws_bytes,
                   CompressJob* j, const stz_compress_opts* opts = nullptr);
int compress_enqueue(const CompressJob& j, bool no_coop, cudaStream_t st, CompressDev* d);
// compress_enqueue in its three stages: up to level 1 (range, bounds, level-1
// coder and histogram); levels 2..L (one level launch after another); the
// entropy stage and the container.  compress_level_args: the arguments of
// level l of job j (for the batched form's work queue, which runs the levels
// of many fields in one launch instead of compress_levels).
int compress_prologue(const CompressJob& j, bool no_coop, cudaStream_t st);
int compress_levels(const CompressJob& j, cudaStream_t st);
int compress_epilogue(const CompressJob& j, cudaStream_t st, CompressDev* d);
void compress_level_args(const CompressJob& j, int l, LevelArgs* out);
// stz_compress's launch sequence as a graph captured once per argument tuple
// and replayed
int compress_graph_launch(const CompressJob& j, const void* field, const int64_t dims[3], int ndim,
                          int dtype, int eb_mode, double eb, void* out, size_t out_cap, void* ws,
                          size_t ws_bytes, cudaStream_t st, CompressDev* d);

// ---- stz_roi.cu: ROI selection (Sec. 3.3) ----
// kmin / kmax / mkey: one u64 per unit each; sel: the selection, ascending;
// nsel: its size; k: units kept in top mode
int launch_roi(const void* field, int dtype, const int64_t n[3], const int64_t b[3], int metric,
               int mode, double value, int64_t k, unsigned long long* kmin,
               unsigned long long* kmax, unsigned long long* mkey, double* metric_out,
               int64_t* sel, unsigned long long* nsel, cudaStream_t s);

// SMs that one launch sizes a persistent grid for: all of them, unless the
// calling thread set a share (the batched form runs several fields' kernels
// side by side and gives each a part of the GPU).
int launch_sms();
// zero fill of device words by a kernel
int launch_zero_words(uint32_t* p, int64_t nwords, cudaStream_t s);
void set_launch_share(int num, int den);

// Lets kernel `func` take `bytes` of dynamic shared memory on the current
// device.  The function's limit only ever rises: a graph captured earlier
// with a larger launch keeps a valid limit when a later call needs less.
// STZ_OK or STZ_ERR_CUDA.
int allow_smem(const void* func, size_t bytes);

}  // namespace stz
