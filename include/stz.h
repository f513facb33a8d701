/*
 * stz.h -- C ABI of the GB300 (sm_103a) implementation of the STZ streaming
 * lossy compressor's hot path ("STZ: A High Quality and High Speed Streaming
 * Lossy Compression Framework for Scientific Data", SC'25).
 *
 * Every step of compression and decompression runs in hand-written CUDA
 * kernels on the device; the host only validates arguments, sizes launches
 * and reads back a few bytes.  The library allocates no device memory:
 * callers pass device buffers (typically from PyTorch) for the field, the
 * output and a workspace, and a CUDA stream (cast to void*; NULL = legacy
 * default stream).  All pointers named *_dev are device pointers.
 *
 * Layout conventions
 *   - A field is a C-order array of float (STZ_F32) or double (STZ_F64).
 *   - dims[] lists the extents slowest first: {nz, ny, nx} for ndim = 3,
 *     {ny, nx} for ndim = 2 (dims[2] ignored).
 *   - Boxes are half-open [lo, hi) in field coordinates, slowest first, in the
 *     same order as dims (2D: only lo[0..1], hi[0..1] are read).
 *   - Level l of L has stride s_l = 2^(L-l): level 1 is the coarsest grid,
 *     level L the full field (Sec. 3.2, three-level partition; L = 3).
 *
 * Errors: every call returns STZ_OK (0) or a negative code; stz_strerror()
 * names it.  Device-side checks (corrupt containers) are read back before a
 * decompression call returns, so no call leaves a fault behind.
 *
 * Threading: calls on different workspaces may run concurrently on different
 * streams.  A workspace must not be shared by two calls in flight.
 */
#ifndef STZ_H
#define STZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { STZ_F32 = 0, STZ_F64 = 1 } stz_dtype;

/* STZ_EB_ABS: |x - x'| <= eb.  STZ_EB_REL: |x - x'| <= eb * (max - min) over
 * the finite values (a zero range falls back to eb as an absolute bound). */
typedef enum { STZ_EB_ABS = 0, STZ_EB_REL = 1 } stz_eb_mode;

enum {
  STZ_OK = 0,
  STZ_ERR_ARG = -1,       /* invalid argument or unsupported container option */
  STZ_ERR_CAPACITY = -2,  /* output or workspace too small; needed size returned */
  STZ_ERR_CORRUPT = -3,   /* container fails validation */
  STZ_ERR_CUDA = -4,      /* a CUDA runtime call failed */
  STZ_ERR_TIMEOUT = -5,   /* a bounded device wait ran out */
  STZ_ERR_NOMEM = -6      /* host allocation failed */
};

/* Name of an error code (static string). */
const char* stz_strerror(int code);

/* Library version string, e.g. "stz-gb300 1.0 (sm_103a)". */
const char* stz_version(void);

/*
 * Worst-case container size for a field of these dims and dtype (all points
 * outliers, longest codes).  0 on invalid arguments.
 */
size_t stz_compress_bound(const int64_t* dims, int ndim, stz_dtype dtype);

/*
 * Workspace bytes that suffice for stz_compress and for every decompression
 * call on a container of a field with these dims and dtype.
 */
size_t stz_workspace_size(const int64_t* dims, int ndim, stz_dtype dtype);

/*
 * Compress (Sec. 3.1-3.2: hierarchical partition into L = 3 levels, SZ3-style
 * interpolation of level 1, multi-dimensional cubic prediction of levels 2
 * and 3 (Eqs. 6-8) with the adaptive bound eb_l = eb_{l+1} / 2.5
 * (Sec. 3.1 opt. 5), linear-scale quantization with outliers, and Huffman
 * coding of each sub-block's codes in independently decodable chunks).
 *
 *   field_dev     input field (device), ndim/dims/dtype as above
 *   eb_mode, eb   error bound (eb > 0, finite)
 *   out_dev       output container (device), capacity out_cap bytes;
 *                 stz_compress_bound() always suffices
 *   out_bytes     receives the container size (also on STZ_ERR_CAPACITY:
 *                 the size that would have been needed)
 *   ws_dev        workspace (device), ws_bytes >= stz_workspace_size()
 *   stream        cudaStream_t
 *
 * Blocks the calling thread once, at the end, to read the size back.
 * The container is bit-identical to the CPU oracle's for the same input.
 * Size limit (here and for every decompression call): the level-1 grid,
 * ceil(dims / 2^(L-1)) per axis, has fewer than 2^31 points, else STZ_ERR_ARG.
 */
int stz_compress(const void* field_dev, const int64_t* dims, int ndim, stz_dtype dtype,
                 stz_eb_mode eb_mode, double eb, void* out_dev, size_t out_cap,
                 size_t* out_bytes, void* ws_dev, size_t ws_bytes, void* stream);

/*
 * Options of stz_compress_ex (NULL or zeroed fields: the method as the paper
 * defines it -- three levels, cubic prediction, adaptive bound ratio 2.5).
 *
 *   levels     L, 1..6 (0: 3).  Sec. 3.2: three levels; more for very large
 *              fields ("4-level (or higher)" for e.g. 4096^3), fewer for small
 *              ones.  Level 1 is the stride-2^(L-1) grid.
 *   predictor  prediction of levels 2..L, the ablation of Sec. 3.1 (Fig. 2):
 *              STZ_PRED_CUBIC (opt. 4, Eqs. 6-8; the method), STZ_PRED_LINEAR
 *              (opt. 2, multi-linear Eqs. 3-5), STZ_PRED_DIRECT (opt. 1,
 *              Eq. 1: the coarse point of the cell).  The two ablation
 *              predictors run in a general (slower) kernel.
 *   eb_ratio   adaptive bound of Sec. 3.1 opt. 5: eb_l = eb_{l+1} / eb_ratio,
 *              in [1, 64] (0: 2.5; 1: the same bound on every level).
 *
 * The container records all three; every decompression call reads them.
 */
typedef enum { STZ_PRED_CUBIC = 0, STZ_PRED_LINEAR = 1, STZ_PRED_DIRECT = 2 } stz_predictor;

typedef struct {
  int levels;
  stz_predictor predictor;
  double eb_ratio;
} stz_compress_opts;

/* stz_compress_bound / stz_workspace_size for a given level count L (0: 3);
 * the workspace then suffices for every decompression of such a container. */
size_t stz_compress_bound_ex(const int64_t* dims, int ndim, stz_dtype dtype, int levels);
size_t stz_workspace_size_ex(const int64_t* dims, int ndim, stz_dtype dtype, int levels);

/* stz_compress with options (opts may be NULL); ws_bytes >=
 * stz_workspace_size_ex(dims, ndim, dtype, opts->levels).  Out-of-range
 * options return STZ_ERR_ARG. */
int stz_compress_ex(const void* field_dev, const int64_t* dims, int ndim, stz_dtype dtype,
                    stz_eb_mode eb_mode, double eb, const stz_compress_opts* opts,
                    void* out_dev, size_t out_cap, size_t* out_bytes, void* ws_dev,
                    size_t ws_bytes, void* stream);

/* Header of a container (host or device memory; comp_on_device selects). */
typedef struct {
  stz_dtype dtype;
  int ndim;
  int64_t dims[3];   /* slowest first; 2D: {ny, nx, 1} */
  int levels;        /* L */
  double eb;         /* bound given to stz_compress */
  stz_eb_mode eb_mode;
  double eb_abs;     /* absolute bound of the finest level */
  uint64_t total_bytes;
} stz_info_t;

int stz_info(const void* comp, size_t comp_bytes, int comp_on_device, stz_info_t* info);

/*
 * Full decompression: the whole field at full resolution, out_cap >= number
 * of points times the element size.  Each level is reconstructed from the
 * coarser one (Sec. 3.3; "L2 pre./rec." of Table 5 fused into one pass).
 */
int stz_decompress_full(const void* comp_dev, size_t comp_bytes, void* out_dev, size_t out_cap,
                        void* ws_dev, size_t ws_bytes, void* stream);

/*
 * Progressive decompression to level `level` (1..L; Sec. 3.3): only levels
 * 1..level are decoded; the output is the stride-2^(L-level) grid, out_dims
 * = ceil(dims / 2^(L-level)) (slowest first; 2D: out_dims[2] = 1).
 */
int stz_decompress_progressive(const void* comp_dev, size_t comp_bytes, int level,
                               void* out_dev, size_t out_cap, int64_t* out_dims, void* ws_dev,
                               size_t ws_bytes, void* stream);

/*
 * Random-access decompression of the box [lo, hi) at level `level`
 * (Sec. 3.3, Fig. 5): every level-1 chunk is entropy-decoded, but only the
 * level-1 interpolation passes the box depends on are run; at each finer
 * level only the chunks and predictions the box needs (its points plus the
 * interpolation support) are decoded, and of a level's 7 sub-block streams
 * only those with points in that support (an axis-aligned slice skips the
 * others: the 2D-slice decoding saving of Sec. 3.3).  The output is the
 * box's points whose coordinates are multiples of 2^(L-level), C order;
 * out_dims receives its shape.  The values
 * are bitwise those of the full decode.  The box must be non-empty and inside
 * the field (STZ_ERR_ARG otherwise); it may contain no lattice point, then
 * out_dims has a zero.
 */
int stz_decompress_region(const void* comp_dev, size_t comp_bytes, const int64_t* lo,
                          const int64_t* hi, int level, void* out_dev, size_t out_cap,
                          int64_t* out_dims, void* ws_dev, size_t ws_bytes, void* stream);

/*
 * Batched form: compress n fields of any shapes and dtypes in one call.
 * Each field's container is bit-identical to stz_compress's for the same
 * field and bound (same stages and kernels); the call only arranges their
 * launches: fields spread over `lanes` concurrent streams (largest first onto
 * the least loaded lane), persistent kernels sized for SMs / sm_share_den,
 * and with use_graph = 1 the whole batch captured once as a CUDA graph that
 * later calls with the same job list replay with one graph launch (up to 8
 * job lists are cached per process).  The paper compresses one field at a
 * time (Sec. 4); this form has no counterpart there.
 *
 *   jobs[i]     one field: field_dev, dims/ndim/dtype, eb_mode/eb and its own
 *               out_dev/out_cap and ws_dev/ws_bytes (>= stz_workspace_size),
 *               all as for stz_compress; no two jobs may share a workspace
 *   sizes_dev   device array of n u64 (8-byte aligned): receives the
 *               container size of field i, with bit 63 set when out_cap was
 *               too small (the low bits then hold the size needed) and bit 62
 *               set when a bounded wait for an asynchronous copy ran out
 *               (STZ_ERR_TIMEOUT of stz_compress)
 *   opts        NULL for defaults (lanes 4, sm_share_den 1, no graph)
 *   stream      the caller's stream; the batch is ordered after the work
 *               queued on it before the call, and work queued after the call
 *               waits for the whole batch
 *
 * Asynchronous: nothing is waited for.  Arguments are checked for every job
 * before any work is queued (STZ_ERR_ARG / STZ_ERR_CAPACITY for a workspace
 * that is too small).  Calls from several host threads are serialised.
 */
typedef struct {
  const void* field_dev;
  int64_t dims[3];
  int ndim;
  stz_dtype dtype;
  stz_eb_mode eb_mode;
  double eb;
  void* out_dev;
  size_t out_cap;
  void* ws_dev;
  size_t ws_bytes;
} stz_field_job;

typedef struct {
  int lanes;         /* concurrent streams, 1..32 (0: 4) */
  int sm_share_den;  /* persistent grids sized for SMs / den, 1..64 (0: 1) */
  int use_graph;     /* 1: capture once, replay as one graph launch */
  /* The work-queue arrangement (persistent = 1): every 3D field with the
   * default predictor runs its level stages 2..L inside ONE persistent launch
   * per dtype, whose blocks claim (field, level, tile) work items in schedule
   * order from a counter (an item of level l waits, on the device, for its
   * field's level l-1); fields' stages up to level 1 and after the levels run
   * on the lanes before and after it.  Other fields (2D, ablation predictors)
   * run the per-field path on the lanes meanwhile. */
  int persistent;      /* 1: the work queue; needs ws_dev */
  int schedule;        /* 0: every field's level 2, then level 3, ...; 1: field by field */
  int tiles_per_item;  /* interior brick tiles per work item, 1..64 (0: 1) */
  int blocks_per_sm;   /* blocks of the queue kernel per SM (0: as many as fit) */
  void* ws_dev;        /* persistent: 256-byte aligned device memory of */
  size_t ws_bytes;     /*   stz_compress_batch_workspace_size() bytes */
} stz_batch_opts;

/* Workspace of the work-queue arrangement of stz_compress_batch for these
 * jobs (0 on invalid jobs). */
size_t stz_compress_batch_workspace_size(int n, const stz_field_job* jobs);

int stz_compress_batch(int n, const stz_field_job* jobs, unsigned long long* sizes_dev,
                       const stz_batch_opts* opts, void* stream);

/* ---- ROI selection (Sec. 3.3, last paragraph) ----
 * The paper's module that helps users pick the regions of interest to
 * decompress: per slice or block of a field, the value range (suits
 * interfaces between fluids) or the maximum (suits over-density halos), then
 * the units whose metric reaches a threshold or the top x% of units.  It is
 * meant for a progressive (coarse) decode of a field: the selected units,
 * scaled by the level's stride, are boxes for stz_decompress_region.
 *
 * A unit is a block of block[] points, slowest axis first ({bz, by, bx};
 * 2D: {by, bx}), clipped at the field's edge; units are numbered in raster
 * order of (z / bz, y / by, x / bx).  A slice along an axis is the block of
 * extent 1 along that axis spanning the others.
 *
 *   metric   STZ_ROI_RANGE: max - min of the unit's finite values (one
 *            correctly rounded double subtraction); STZ_ROI_MAX: the
 *            maximum.  A unit without a finite value has the metric -inf.
 *            Non-finite values are ignored; -0 orders below +0.
 *   mode     STZ_ROI_THRESHOLD: units with metric >= value;
 *            STZ_ROI_TOP: the ceil(value * nunits) units (0 < value <= 1,
 *            the product in double) with the largest metrics, equal metrics
 *            taken by lower unit index.
 *   sel_dev      device int64[sel_cap >= nunits]: the selected unit indices,
 *                ascending
 *   metric_dev   device double[nunits] receiving every unit's metric, or NULL
 *   nsel         host: the number of selected units
 *   ws_dev       device workspace of stz_roi_workspace_size() bytes
 *
 * Waits on the host once, at the end, for nsel.  The result equals the CPU
 * oracle's bit for bit.  Units must number fewer than 2^31. */
typedef enum { STZ_ROI_RANGE = 0, STZ_ROI_MAX = 1 } stz_roi_metric;
typedef enum { STZ_ROI_THRESHOLD = 0, STZ_ROI_TOP = 1 } stz_roi_mode;

/* Number of units (-1 on invalid arguments). */
int64_t stz_roi_units(const int64_t* dims, int ndim, const int64_t* block);
size_t stz_roi_workspace_size(const int64_t* dims, int ndim, const int64_t* block);
int stz_roi_select(const void* field_dev, const int64_t* dims, int ndim, stz_dtype dtype,
                   const int64_t* block, stz_roi_metric metric, stz_roi_mode mode, double value,
                   int64_t* sel_dev, size_t sel_cap, double* metric_dev, int64_t* nsel,
                   void* ws_dev, size_t ws_bytes, void* stream);

/* ---- serving support (no counterpart in the paper) ----
 * A serving loop keeps containers resident and answers many region requests
 * without waiting on the host per request: it parses each container's header
 * once (the first STZ_HEADER_MAX_BYTES bytes, or the whole container if
 * shorter, copied to the host), decodes each field's level-1 grid once with
 * stz_decompress_progressive(level 1) and keeps it, and then issues
 * stz_decompress_region_async for each request on a stream of its own. */
#define STZ_HEADER_MAX_BYTES 1984

/* Workspace bytes a region decode of [lo, hi) at `level` needs, given the
 * header bytes; level1_given != 0 when the level-1 grid will be supplied.
 * 0 on invalid arguments or a corrupt header. */
size_t stz_region_workspace_size(const void* hdr_host, size_t hdr_bytes, size_t comp_bytes,
                                 const int64_t* lo, const int64_t* hi, int level,
                                 int level1_given);

/*
 * Plan of a region decode, on the host only (no device work): for each
 * stream of the container (0 = level 1, 1 + 7(l-2) + (k-1) = level l
 * sub-block k), the number of its chunks that stz_decompress_region (or the
 * _async form, with level1_given as there) entropy-decodes for the box
 * [lo, hi) at `level`.  Sec. 3.3: a level-l point depends only on nearby
 * points of level l-1, so a box needs few chunks, and an axis-aligned slice
 * needs none of the sub-blocks whose points it does not hold (3 of the 7
 * finest-level streams for a z-slice at an even z).  hdr_host as for
 * stz_region_workspace_size; chunks has room for max_streams entries.
 * Returns the container's stream count, or STZ_ERR_ARG / STZ_ERR_CORRUPT.
 */
int stz_region_chunks(const void* hdr_host, size_t hdr_bytes, size_t comp_bytes,
                      const int64_t* lo, const int64_t* hi, int level, int level1_given,
                      int64_t* chunks, int max_streams);

/*
 * Region decode (as stz_decompress_region: Sec. 3.3 random access, values
 * bitwise those of the full decode) that never waits on the host:
 *   hdr_host, hdr_bytes  host copy of the container's first bytes (see above)
 *   level1_dev           the field's decoded level-1 grid (output of
 *                        stz_decompress_progressive at level 1, device), or
 *                        NULL to decode the level-1 passes the box needs
 *   status_dev           device u32 that receives 0, or a nonzero status when
 *                        the container proved corrupt during the decode
 * Arguments are checked on the host (STZ_ERR_ARG / STZ_ERR_CAPACITY /
 * STZ_ERR_CORRUPT for a bad header) before any work is queued on `stream`.
 * Calls on different streams with different workspaces may overlap.
 */
int stz_decompress_region_async(const void* comp_dev, size_t comp_bytes, const void* hdr_host,
                                size_t hdr_bytes, const void* level1_dev, const int64_t* lo,
                                const int64_t* hi, int level, void* out_dev, size_t out_cap,
                                int64_t* out_dims, void* ws_dev, size_t ws_bytes,
                                uint32_t* status_dev, void* stream);

/*
 * Region decompression without any allocation, for callers that cannot
 * obtain memory at the point of the call: a plug-in (an I/O library filter,
 * a visualisation reader) that its host application hands only the
 * compressed input and the output buffer, or a latency-critical path that
 * must not pay cudaMalloc's implicit device synchronisation.  The paper has
 * no counterpart; it is an addition of this library.
 *
 * Same arguments, output and errors as stz_decompress_region, minus the
 * workspace: the scratch comes from one array of STZ_NOALLOC_SCRATCH_BYTES
 * in the library's device memory, which every GPU that loads the library
 * holds until the process exits (with CUDA's lazy module loading it is
 * reserved on a device when the library's kernels are first loaded there,
 * at the latest by this call's first use on that device).  A call whose
 * decode needs more scratch than that returns STZ_ERR_CAPACITY before any
 * work is queued (all level-1 chunks are decoded into it, so this covers
 * fields up to about 512^3 f32 with boxes up to about 128^3).
 *
 * Allocates nothing, on the host or the device: no cudaMalloc, cudaFree,
 * cudaHostAlloc or graph instantiation.  The header and the final status
 * word come back by plain copies into the call's own stack, and the kernels
 * are launched one by one (other decode calls cache parsed headers, use a
 * pinned per-thread read-back buffer and replay repeated calls as graphs;
 * this one does none of that).  Only with kernel timing switched on
 * (stz_profile_enable) does the library's timer create CUDA events.
 *
 * The first call on a device looks up that array's device address (with
 * the device current); make that first call before any stream capture on
 * the device.  The calling thread must have the stream's device current.
 * The call waits on the host for the header and for the final status.
 * All calls share the one array and it keeps the last call's contents
 * (each call clears what must start at zero): calls whose work overlaps on
 * the GPU -- on different streams, or from different host threads -- race
 * and give wrong results.  Issue them on one stream, one after another.
 */
#define STZ_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int stz_decompress_region_noalloc(const void* comp_dev, size_t comp_bytes, const int64_t* lo,
                                  const int64_t* hi, int level, void* out_dev, size_t out_cap,
                                  int64_t* out_dims, void* stream);

/* ---- batched serving: many region requests in a fixed number of launches ----
 * (no counterpart in the paper).  A serving loop that keeps fields resident
 * decodes every admitted request of an iteration with one call: the chunk
 * decoding of all of them is one kernel launch, each finer level's
 * prediction one launch of the interior and one of the boundary kernel, and
 * the level-1 copies one launch -- whatever the number of requests.  Each
 * result is bitwise that of stz_decompress_region.
 *
 * Per field, once: its level-1 grid (stz_decompress_progressive at level 1)
 * and its decode tables (stz_decode_tables). */
size_t stz_decode_tables_size(const void* hdr_host, size_t hdr_bytes, size_t comp_bytes);
int stz_decode_tables(const void* comp_dev, size_t comp_bytes, const void* hdr_host,
                      size_t hdr_bytes, void* tables_dev, size_t tables_bytes, void* stream);

typedef struct {
  const void* comp_dev;     /* the container (device) */
  size_t comp_bytes;
  const void* hdr_host;     /* host copy of its first bytes (STZ_HEADER_MAX_BYTES) */
  size_t hdr_bytes;
  const void* level1_dev;   /* its decoded level-1 grid */
  const void* tables_dev;   /* its decode tables (stz_decode_tables) */
} stz_served_field;

typedef struct {
  int field;                /* index into the fields array */
  int level;                /* 1..L */
  int64_t lo[3], hi[3];     /* the box, axis order as for stz_decompress_region */
  void* out_dev;            /* output (device), out_cap bytes */
  size_t out_cap;
  int64_t out_dims[3];      /* receives the output shape */
} stz_region_request;

/* Workspace bytes of stz_decode_requests for these requests (0 on invalid
 * arguments). */
size_t stz_decode_requests_workspace(int n, const stz_region_request* reqs,
                                     const stz_served_field* fields, int nfields);

/*
 * Decode n region requests on `stream` without waiting on the host.  All
 * fields must have the same dtype.  status_dev: device u32[n], receives 0 or
 * a nonzero status per request (corrupt container).  Arguments are checked
 * for every request before any work is queued (STZ_ERR_ARG /
 * STZ_ERR_CAPACITY / STZ_ERR_CORRUPT for a bad header).  The call copies
 * the launch arguments to the workspace from host memory it owns; the
 * workspace must not be in use by another call in flight.
 */
int stz_decode_requests(int n, stz_region_request* reqs, const stz_served_field* fields,
                        int nfields, void* ws_dev, size_t ws_bytes, uint32_t* status_dev,
                        void* stream);

/* ---- tracing (no counterpart in the paper, which reports wall times only) ----
 * Every kernel launch of the library is counted.  With profiling enabled an
 * event pair is recorded around each launch on its stream; stz_profile_read
 * waits for those events and returns, per kernel name, the number of timed
 * launches, their summed device time and their summed algorithmic bytes
 * (what the launches must read and write at the least: inputs once, outputs
 * once; 0 for kernels without such a figure).  Off by default. */
typedef struct {
  char name[48];
  unsigned long long launches;
  double total_ms;
  double algo_bytes;
} stz_kernel_time;

unsigned long long stz_launch_count(void);
void stz_profile_enable(int on);
void stz_profile_reset(void);
/* Fills up to max_entries entries; returns the number of kernel names seen. */
int stz_profile_read(stz_kernel_time* out, int max_entries);

#ifdef __cplusplus
}
#endif
#endif
