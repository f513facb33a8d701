// stz_batch.cu -- the batched form of compression (stz_compress_batch): many
// fields of uneven shape and dtype compressed in one call, with no host
// synchronisation between them.  Each field runs the same stages and kernels
// as stz_compress, so its container is bit-identical to the single-field
// call; what changes is how the launches are arranged on the GPU:
//   - fields are spread over `lanes` streams, largest first onto the least
//     loaded lane, so the latency-bound stages of small fields (level-1
//     passes, codebooks, scans) overlap with the bandwidth-bound stages of
//     large ones;
//   - each field's persistent kernels size their grids for a share of the
//     SMs, so side-by-side fields do not queue behind one another;
//   - with use_graph the whole fork/join of lanes is captured once as one
//     CUDA graph and replayed by a single cudaGraphLaunch on later calls with
//     the same jobs (graphs are cached by the job list);
//   - each field's container size lands in a device array, so the caller
//     reads all sizes with one copy.
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "stz_kernels.cuh"
#include "stz_prof.cuh"

namespace stz {

__global__ void k_batch_size(const unsigned long long* __restrict__ total,
                             const uint32_t* __restrict__ status,
                             unsigned long long* __restrict__ out) {
  if (threadIdx.x == 0) {
    unsigned long long v = *total;
    if (*status & kStatCapacity) v |= 1ull << 63;
    if (*status & kStatTimeout) v |= 1ull << 62;
    *out = v;
  }
}

namespace {

constexpr int kMaxLanes = 32;
constexpr int kMaxDevices = 64;
constexpr size_t kGraphCacheSize = 8;

struct Lanes {
  bool ready = false;
  cudaStream_t cap = nullptr;  // origin stream of captures
  cudaStream_t s[kMaxLanes] = {};
  cudaEvent_t fork = nullptr, join[kMaxLanes] = {};
  cudaEvent_t pro[kMaxLanes] = {};  // work queue: a lane's prologues queued
  cudaEvent_t lev[2] = {};          // work queue: the level launch of a dtype done
};

struct CachedGraph {
  std::vector<unsigned char> key;
  int dev;
  cudaGraphExec_t exec;
  unsigned long long kernels;
  unsigned long long last_use;
};

std::mutex g_mu;
Lanes g_lanes[kMaxDevices];
std::vector<CachedGraph> g_graphs;
unsigned long long g_tick = 0;

int lanes_of(int dev, Lanes** out) {
  Lanes& L = g_lanes[dev];
  if (!L.ready) {
    if (cudaStreamCreateWithFlags(&L.cap, cudaStreamNonBlocking) != cudaSuccess) return STZ_ERR_CUDA;
    if (cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming) != cudaSuccess) return STZ_ERR_CUDA;
    for (int i = 0; i < kMaxLanes; i++) {
      if (cudaStreamCreateWithFlags(&L.s[i], cudaStreamNonBlocking) != cudaSuccess)
        return STZ_ERR_CUDA;
      if (cudaEventCreateWithFlags(&L.join[i], cudaEventDisableTiming) != cudaSuccess)
        return STZ_ERR_CUDA;
      if (cudaEventCreateWithFlags(&L.pro[i], cudaEventDisableTiming) != cudaSuccess)
        return STZ_ERR_CUDA;
    }
    for (int d = 0; d < 2; d++)
      if (cudaEventCreateWithFlags(&L.lev[d], cudaEventDisableTiming) != cudaSuccess)
        return STZ_ERR_CUDA;
    L.ready = true;
  }
  *out = &L;
  return STZ_OK;
}

struct ShareGuard {
  ShareGuard(int den) { set_launch_share(1, den); }
  ~ShareGuard() { set_launch_share(1, 1); }
};

// Fork from `origin` onto the lanes, queue every field, join back.
int enqueue_all(const std::vector<CompressJob>& jobs, const std::vector<int>& order,
                const std::vector<int>& lane_of, unsigned long long* sizes_dev, int lanes, int share_den, bool no_coop,
                cudaStream_t origin, Lanes& L) {
  int rc;
  if ((rc = cuda_ok(cudaEventRecord(L.fork, origin))) != STZ_OK) return rc;
  for (int i = 0; i < lanes; i++)
    if ((rc = cuda_ok(cudaStreamWaitEvent(L.s[i], L.fork, 0))) != STZ_OK) return rc;
  {
    ShareGuard share(share_den);
    for (int f : order) {
      cudaStream_t st = L.s[lane_of[(size_t)f]];
      CompressDev d;
      if ((rc = compress_enqueue(jobs[(size_t)f], no_coop, st, &d)) != STZ_OK) return rc;
      ProfScope ps_("k_batch_size", st);
      k_batch_size<<<1, 32, 0, st>>>(d.total, d.status, sizes_dev + f);
      if ((rc = cuda_ok(cudaGetLastError())) != STZ_OK) return rc;
    }
  }
  for (int i = 0; i < lanes; i++) {
    if ((rc = cuda_ok(cudaEventRecord(L.join[i], L.s[i]))) != STZ_OK) return rc;
    if ((rc = cuda_ok(cudaStreamWaitEvent(origin, L.join[i], 0))) != STZ_OK) return rc;
  }
  return STZ_OK;
}

// ---- the work-queue arrangement ----
// A field whose level stages suit the queue kernel: 3D, every level on the
// fast kernels' brick and predictor.
bool queue_eligible(const CompressJob& j) {
  if (j.g.ndim != 3 || j.g.L < 2) return false;
  for (int l = 2; l <= j.g.L; l++) {
    LevelArgs a;
    compress_level_args(j, l, &a);
    if (!level_queue_ok(a)) return false;
  }
  return true;
}

// The level groups of the eligible fields of one dtype, in the order of
// `order` (largest field first), each field's levels ascending.
void queue_groups(const std::vector<CompressJob>& jobs, const std::vector<int>& order,
                  const std::vector<char>& elig, int dtype, std::vector<LevelArgs>* h) {
  h->clear();
  for (int f : order) {
    const CompressJob& j = jobs[(size_t)f];
    if (!elig[(size_t)f] || j.g.dtype != dtype) continue;
    for (int l = 2; l <= j.g.L; l++) {
      LevelArgs a;
      compress_level_args(j, l, &a);
      h->push_back(a);
    }
  }
}

size_t al256b(size_t v) { return (v + 255) & ~(size_t)255; }

// workspace of the queue arrangement: one arena per dtype
size_t queue_ws_bytes(const std::vector<CompressJob>& jobs, const std::vector<char>& elig,
                      size_t* off_f64) {
  int ng[2] = {0, 0};
  for (size_t f = 0; f < jobs.size(); f++)
    if (elig[f]) ng[jobs[f].g.dtype == STZ_F64 ? 1 : 0] += jobs[f].g.L - 1;
  const size_t a0 = ng[0] ? al256b(level_queue_arena_bytes(ng[0])) : 0;
  const size_t a1 = ng[1] ? al256b(level_queue_arena_bytes(ng[1])) : 0;
  if (off_f64) *off_f64 = a0;
  return a0 + a1;
}

struct QueueParts {
  LevelQueuePlan plan[2];  // f32, f64
};

int plan_queues(const std::vector<CompressJob>& jobs, const std::vector<int>& order,
                const std::vector<char>& elig, const stz_batch_opts& o, QueueParts* Q) {
  size_t off64 = 0;
  const size_t need = queue_ws_bytes(jobs, elig, &off64);
  if (need > 0 && (!o.ws_dev || ((uintptr_t)o.ws_dev & 255))) return STZ_ERR_ARG;
  if (o.ws_bytes < need) return STZ_ERR_CAPACITY;
  const int gran = o.tiles_per_item > 0 ? o.tiles_per_item : 1;
  for (int d = 0; d < 2; d++) {
    std::vector<LevelArgs> h;
    queue_groups(jobs, order, elig, d == 0 ? STZ_F32 : STZ_F64, &h);
    uint8_t* arena = (uint8_t*)o.ws_dev + (d == 0 ? 0 : off64);
    const int rc = plan_level_queue(h.data(), (int)h.size(), o.schedule, gran, o.blocks_per_sm,
                                    arena, &Q->plan[d]);
    if (rc != STZ_OK) return rc;
  }
  return STZ_OK;
}

// The work-queue arrangement: prologues of the eligible fields on the lanes,
// the queue launches (f32 on lane 0, f64 on lane 1) once every lane's
// prologues are done, the other fields' whole compressions on their lanes
// meanwhile, then each eligible field's epilogue after its dtype's queue.
int enqueue_queue(const std::vector<CompressJob>& jobs, const std::vector<int>& order,
                  const std::vector<int>& lane_of, const std::vector<char>& elig,
                  const QueueParts& Q, unsigned long long* sizes_dev, int lanes, int share_den,
                  bool no_coop, cudaStream_t origin, Lanes& L) {
  int rc;
  if ((rc = cuda_ok(cudaEventRecord(L.fork, origin))) != STZ_OK) return rc;
  for (int i = 0; i < lanes; i++)
    if ((rc = cuda_ok(cudaStreamWaitEvent(L.s[i], L.fork, 0))) != STZ_OK) return rc;
  {
    ShareGuard share(share_den);
    for (int f : order)
      if (elig[(size_t)f])
        if ((rc = compress_prologue(jobs[(size_t)f], no_coop, L.s[lane_of[(size_t)f]])) != STZ_OK)
          return rc;
  }
  for (int i = 0; i < lanes; i++)
    if ((rc = cuda_ok(cudaEventRecord(L.pro[i], L.s[i]))) != STZ_OK) return rc;
  cudaStream_t qs[2] = {L.s[0], L.s[lanes > 1 ? 1 : 0]};
  bool ran[2] = {false, false};
  for (int d = 0; d < 2; d++) {
    if (Q.plan[d].grid == 0) continue;
    for (int i = 0; i < lanes; i++)
      if (L.s[i] != qs[d])
        if ((rc = cuda_ok(cudaStreamWaitEvent(qs[d], L.pro[i], 0))) != STZ_OK) return rc;
    if ((rc = run_level_queue(Q.plan[d], qs[d])) != STZ_OK) return rc;
    if ((rc = cuda_ok(cudaEventRecord(L.lev[d], qs[d]))) != STZ_OK) return rc;
    ran[d] = true;
  }
  ShareGuard share(share_den);
  // fields outside the queue: their whole compression on their lanes
  for (int f : order) {
    if (elig[(size_t)f]) continue;
    cudaStream_t st = L.s[lane_of[(size_t)f]];
    CompressDev dd;
    if ((rc = compress_enqueue(jobs[(size_t)f], no_coop, st, &dd)) != STZ_OK) return rc;
    ProfScope ps_("k_batch_size", st);
    k_batch_size<<<1, 32, 0, st>>>(dd.total, dd.status, sizes_dev + f);
    if ((rc = cuda_ok(cudaGetLastError())) != STZ_OK) return rc;
  }
  // the queued fields' entropy stages, after their dtype's level launch
  std::vector<char> waited((size_t)lanes * 2, 0);
  for (int f : order) {
    if (!elig[(size_t)f]) continue;
    const int ln = lane_of[(size_t)f];
    const int d = jobs[(size_t)f].g.dtype == STZ_F64 ? 1 : 0;
    cudaStream_t st = L.s[ln];
    if (ran[d] && !waited[(size_t)ln * 2 + d] && st != qs[d]) {
      if ((rc = cuda_ok(cudaStreamWaitEvent(st, L.lev[d], 0))) != STZ_OK) return rc;
      waited[(size_t)ln * 2 + d] = 1;
    }
    CompressDev dd;
    if ((rc = compress_epilogue(jobs[(size_t)f], st, &dd)) != STZ_OK) return rc;
    ProfScope ps_("k_batch_size", st);
    k_batch_size<<<1, 32, 0, st>>>(dd.total, dd.status, sizes_dev + f);
    if ((rc = cuda_ok(cudaGetLastError())) != STZ_OK) return rc;
  }
  for (int i = 0; i < lanes; i++) {
    if ((rc = cuda_ok(cudaEventRecord(L.join[i], L.s[i]))) != STZ_OK) return rc;
    if ((rc = cuda_ok(cudaStreamWaitEvent(origin, L.join[i], 0))) != STZ_OK) return rc;
  }
  return STZ_OK;
}

unsigned long long count_kernels(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  unsigned long long k = 0;
  for (size_t i = 0; i < n; i++) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) k++;
  }
  return k;
}

}  // namespace
}  // namespace stz

using namespace stz;

extern "C" size_t stz_compress_batch_workspace_size(int n, const stz_field_job* jobs_in) {
  if (n < 1 || !jobs_in) return 0;
  std::vector<CompressJob> jobs((size_t)n);
  std::vector<char> elig((size_t)n, 0);
  for (int f = 0; f < n; f++) {
    const stz_field_job& J = jobs_in[f];
    if (compress_check(J.field_dev, J.dims, J.ndim, J.dtype, J.eb_mode, J.eb, J.out_dev,
                       J.out_cap, J.ws_dev, J.ws_bytes, &jobs[(size_t)f]) != STZ_OK)
      return 0;
    elig[(size_t)f] = queue_eligible(jobs[(size_t)f]) ? 1 : 0;
  }
  return queue_ws_bytes(jobs, elig, nullptr);
}

extern "C" int stz_compress_batch(int n, const stz_field_job* jobs_in,
                                  unsigned long long* sizes_dev, const stz_batch_opts* opts,
                                  void* stream) {
  if (n < 1 || !jobs_in || !sizes_dev) return STZ_ERR_ARG;
  if ((uintptr_t)sizes_dev % 8) return STZ_ERR_ARG;
  stz_batch_opts o;  // member by member: padding bytes stay zero (o is part of a cache key)
  memset(&o, 0, sizeof(o));
  if (opts) {
    o.lanes = opts->lanes;
    o.sm_share_den = opts->sm_share_den;
    o.use_graph = opts->use_graph;
    o.persistent = opts->persistent;
    o.schedule = opts->schedule;
    o.tiles_per_item = opts->tiles_per_item;
    o.blocks_per_sm = opts->blocks_per_sm;
    o.ws_dev = opts->ws_dev;
    o.ws_bytes = opts->ws_bytes;
  }
  if (o.persistent && (o.schedule < 0 || o.schedule > 1 || o.tiles_per_item < 0 ||
                       o.tiles_per_item > 64 || o.blocks_per_sm < 0))
    return STZ_ERR_ARG;
  int lanes = o.lanes > 0 ? o.lanes : 4;
  if (lanes > kMaxLanes) return STZ_ERR_ARG;
  if (lanes > n) lanes = n;
  const int share_den = o.sm_share_den > 0 ? o.sm_share_den : 1;
  if (share_den > 64) return STZ_ERR_ARG;
  std::vector<CompressJob> jobs((size_t)n);
  for (int f = 0; f < n; f++) {
    const stz_field_job& J = jobs_in[f];
    const int rc = compress_check(J.field_dev, J.dims, J.ndim, J.dtype, J.eb_mode, J.eb,
                                  J.out_dev, J.out_cap, J.ws_dev, J.ws_bytes, &jobs[(size_t)f]);
    if (rc != STZ_OK) return rc;
  }
  // largest field first onto the least loaded lane
  std::vector<int> order((size_t)n), lane_of((size_t)n);
  for (int f = 0; f < n; f++) order[(size_t)f] = f;
  auto pts = [&](int f) {
    const Geo& g = jobs[(size_t)f].g;
    return (double)g.n[0] * g.n[1] * g.n[2] * (g.dtype == STZ_F64 ? 2.0 : 1.0);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pts(a) > pts(b); });
  std::vector<double> load((size_t)lanes, 0.0);
  for (int f : order) {
    int best = 0;
    for (int i = 1; i < lanes; i++)
      if (load[(size_t)i] < load[(size_t)best]) best = i;
    lane_of[(size_t)f] = best;
    load[(size_t)best] += pts(f);
  }
  cudaStream_t origin = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return STZ_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  Lanes* L = nullptr;
  int rc = lanes_of(dev, &L);
  if (rc != STZ_OK) return rc;
  // the work queue: its plans, and the copy of its arguments into the batch
  // workspace (queued on the caller's stream, outside any capture)
  std::vector<char> elig((size_t)n, 0);
  QueueParts Q;
  if (o.persistent) {
    for (int f = 0; f < n; f++) elig[(size_t)f] = queue_eligible(jobs[(size_t)f]) ? 1 : 0;
    if ((rc = plan_queues(jobs, order, elig, o, &Q)) != STZ_OK) return rc;
    for (int d = 0; d < 2; d++)
      if ((rc = write_level_queue(Q.plan[d], origin)) != STZ_OK) return rc;
  }
  auto enqueue = [&](bool no_coop, cudaStream_t org) {
    return o.persistent ? enqueue_queue(jobs, order, lane_of, elig, Q, sizes_dev, lanes,
                                        share_den, no_coop, org, *L)
                        : enqueue_all(jobs, order, lane_of, sizes_dev, lanes, share_den, no_coop,
                                      org, *L);
  };
  // side-by-side lanes never use the cooperative level-1 launch: its grid
  // barrier needs every block resident while other fields hold SMs
  if (!o.use_graph) return enqueue(lanes > 1 || o.persistent, origin);
  // graph: look the job list up, else capture it once on the origin stream
  std::vector<unsigned char> key(sizeof(stz_field_job) * (size_t)n + sizeof(o) + 2 * sizeof(int) +
                                 sizeof(void*));
  {
    unsigned char* k = key.data();
    for (int f = 0; f < n; f++) {  // member by member: padding bytes stay zero
      stz_field_job c;
      memset(&c, 0, sizeof(c));
      const stz_field_job& J = jobs_in[f];
      c.field_dev = J.field_dev;
      memcpy(c.dims, J.dims, sizeof(c.dims));
      c.ndim = J.ndim;
      c.dtype = J.dtype;
      c.eb_mode = J.eb_mode;
      c.eb = J.eb;
      c.out_dev = J.out_dev;
      c.out_cap = J.out_cap;
      c.ws_dev = J.ws_dev;
      c.ws_bytes = J.ws_bytes;
      memcpy(k, &c, sizeof(c));
      k += sizeof(c);
    }
    memcpy(k, &o, sizeof(o));
    k += sizeof(o);
    memcpy(k, &n, sizeof(int));
    k += sizeof(int);
    memcpy(k, &dev, sizeof(int));
    k += sizeof(int);
    memcpy(k, &sizes_dev, sizeof(void*));
  }
  CachedGraph* hit = nullptr;
  for (auto& c : g_graphs)
    if (c.dev == dev && c.key == key) hit = &c;
  if (!hit) {
    if (g_graphs.size() >= kGraphCacheSize) {
      auto old = std::min_element(g_graphs.begin(), g_graphs.end(),
                                  [](const CachedGraph& a, const CachedGraph& b) {
                                    return a.last_use < b.last_use;
                                  });
      cudaGraphExecDestroy(old->exec);
      g_graphs.erase(old);
    }
    cudaGraph_t graph = nullptr;
    if ((rc = cuda_ok(cudaStreamBeginCapture(L->cap, cudaStreamCaptureModeThreadLocal))) != STZ_OK)
      return rc;
    rc = enqueue(true, L->cap);
    const cudaError_t ce = cudaStreamEndCapture(L->cap, &graph);
    if (rc == STZ_OK && ce != cudaSuccess) rc = STZ_ERR_CUDA;
    if (rc != STZ_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc;
    }
    CachedGraph c;
    c.key = key;
    c.dev = dev;
    c.kernels = count_kernels(graph);
    c.last_use = 0;
    const cudaError_t ie = cudaGraphInstantiate(&c.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return STZ_ERR_CUDA;
    g_graphs.push_back(c);
    hit = &g_graphs.back();
  }
  hit->last_use = ++g_tick;
  if ((rc = cuda_ok(cudaGraphLaunch(hit->exec, origin))) != STZ_OK) return rc;
  prof_count_launches(hit->kernels);
  return STZ_OK;
}
