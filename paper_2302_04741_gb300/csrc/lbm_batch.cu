// lbm_batch.cu -- batches of contexts stepped by one launch per step
// (lbm_batch_* in include/lbm.h), with CUDA-graph replay and an autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lbm_ctx.h"

struct lbm_batch {
  int lat = 0, precision = 0, force_order = 2;
  const lbm::LatticeOps* ops = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0, nsm = 0;
  std::vector<lbm_ctx*> members;
  int cap = 0;
  lbm::BatchGrid* d_grids = nullptr;
  int* d_prefix = nullptr;  // cap + 1
  int* d_header = nullptr;  // 2
  lbm::BatchGrid* h_grids = nullptr;  // pinned staging
  int* h_prefix = nullptr;
  int* h_header = nullptr;
  cudaEvent_t staged = nullptr;  // last upload from the staging buffers
  bool dirty = true;
  int bx = 128, spt = 1, ctas = 0;
  int stage = 0;  // 1: halo-staged kernel (FP32-shifted, one site per thread)
  int graph_steps = 0;
  cudaGraphExec_t graph = nullptr;
  std::string err;
};

namespace {

int bfail(lbm_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  else lbm::set_global_error(buf);
  return code;
}

#define BCUDA(b, call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail(b, LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
  } while (0)

void drop_graph(lbm_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

// CTAs of a batch launch: LBM_BATCH_WAVES times the resident capacity, each
// striding over the tiles.  Queued CTAs let the block scheduler start a new
// CTA whenever one finishes, as in a plain launch: on GB300 16 waves gave the
// ragged 64-grid mix 0.91 of the HBM roofline instead of 0.84 with one wave
// (a strictly persistent grid), and 24 mixed D3Q39 boxes +4 %; 64 waves were
// slower again.  A tuning hook (LBM_NVCC_DEFINES).
#ifndef LBM_BATCH_WAVES
#define LBM_BATCH_WAVES 16
#endif
int set_ctas(lbm_batch* b) {
  int bps = 0;
  if (b->stage) BCUDA(b, b->ops->batch_staged_occupancy(b->force_order, b->bx, &bps));
  else BCUDA(b, b->ops->batch_occupancy(b->precision, b->force_order, b->spt, b->bx, &bps));
  if (bps < 1) return bfail(b, LBM_EINVAL, "batch kernel does not fit with block %d", b->bx);
  b->ctas = bps * b->nsm * LBM_BATCH_WAVES;
  return LBM_OK;
}

// Uploads the member table (parameters, buffers, parities, tile prefix).
int upload(lbm_batch* b) {
  BCUDA(b, cudaEventSynchronize(b->staged));  // staging buffers free again
  const int TW = b->bx * b->spt;
  long long tiles = 0;
  const int n = (int)b->members.size();
  size_t bytes = 0;  // the launch's working set: both buffers of every member
  for (int g = 0; g < n; ++g)
    bytes += 2 * (size_t)b->members[g]->Q * b->members[g]->N * b->members[g]->elem;
  const int evict_first = lbm::l2_evict_first_for(bytes, b->device);
  for (int g = 0; g < n; ++g) {
    lbm_ctx* c = b->members[g];
    lbm::BatchGrid& G = b->h_grids[g];
    G.p = c->p;
    G.p.l2_evict_first = evict_first;
    G.f[0] = c->f[0];
    G.f[1] = c->f[1];
    G.cur = c->cur;
    b->h_prefix[g] = (int)tiles;
    tiles += ((long long)c->N + TW - 1) / TW;
  }
  if (tiles >= (1LL << 31)) return bfail(b, LBM_EINVAL, "batch has too many tiles");
  b->h_prefix[n] = (int)tiles;
  b->h_header[0] = n;
  b->h_header[1] = (int)tiles;
  if (n) BCUDA(b, cudaMemcpyAsync(b->d_grids, b->h_grids, sizeof(lbm::BatchGrid) * n,
                                  cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemcpyAsync(b->d_prefix, b->h_prefix, sizeof(int) * (n + 1), cudaMemcpyHostToDevice,
                           b->stream));
  BCUDA(b, cudaMemcpyAsync(b->d_header, b->h_header, sizeof(int) * 2, cudaMemcpyHostToDevice,
                           b->stream));
  BCUDA(b, cudaEventRecord(b->staged, b->stream));
  b->dirty = false;
  return LBM_OK;
}

int launch(lbm_batch* b, int k) {
  if (b->stage) {
    BCUDA(b, b->ops->batch_step_staged(b->force_order, b->d_grids, b->d_prefix, b->d_header, k, b->ctas,
                                       b->bx, b->stream));
    return LBM_OK;
  }
  BCUDA(b, b->ops->batch_step(b->precision, b->force_order, b->spt, b->d_grids, b->d_prefix,
                              b->d_header, k, b->ctas, b->bx, b->stream));
  return LBM_OK;
}

int build_graph(lbm_batch* b) {
  cudaGraph_t g = nullptr;
  BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int rc = LBM_OK;
  for (int k = 0; k < b->graph_steps && rc == LBM_OK; ++k) rc = launch(b, k);
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (rc != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// Autotuner cache: (lattice, precision, order, grid shapes) -> (block, sites
// per thread, staging).
struct TuneChoice {
  int bx, spt, stage;
};
std::mutex g_tune_mutex;
std::map<std::string, TuneChoice> g_tune_cache;

std::string tune_key(const lbm_batch* b) {
  std::vector<std::string> shapes;
  for (auto* c : b->members)
    shapes.push_back(std::to_string(c->nx) + "x" + std::to_string(c->ny) + "x" + std::to_string(c->nz) +
                     (c->p.wall ? "w" : "p"));
  std::sort(shapes.begin(), shapes.end());
  std::string k = std::to_string(b->lat) + "/" + std::to_string(b->precision) + "/" +
                  std::to_string(b->force_order);
  for (auto& s : shapes) k += "/" + s;
  return k;
}

}  // namespace

namespace lbm {
void batch_mark_dirty(lbm_batch* b) {
  if (b) b->dirty = true;
}
int batch_detach(lbm_batch* b, lbm_ctx* c) { return lbm_batch_remove(b, c); }
}  // namespace lbm

extern "C" {

int lbm_batch_create(lbm_lattice lat, int precision, int force_order, void* stream, int capacity,
                     lbm_batch** out) {
  if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  const lbm::LatticeOps* ops = lat == LBM_D2Q37 ? &lbm::ops_d2q37()
                                                : (lat == LBM_D3Q39 ? &lbm::ops_d3q39() : nullptr);
  if (!ops) return bfail(nullptr, LBM_EINVAL, "unknown lattice %d", (int)lat);
  if (precision != LBM_FP32_SHIFTED && precision != LBM_FP16_SCALED)
    return bfail(nullptr, LBM_EINVAL, "batches serve FP32-shifted and FP16-scaled storage");
  if (force_order < 0 || force_order > 2) return bfail(nullptr, LBM_EINVAL, "bad force_order");
  if (capacity < 1 || capacity > (1 << 20)) return bfail(nullptr, LBM_EINVAL, "bad capacity %d", capacity);
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return bfail(nullptr, LBM_ENOMEM, "out of host memory");
  b->lat = lat;
  b->precision = precision;
  b->force_order = force_order;
  b->ops = ops;
  b->stream = (cudaStream_t)stream;
  b->cap = capacity;
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
  bool ok = cudaMalloc(&b->d_grids, sizeof(lbm::BatchGrid) * capacity) == cudaSuccess &&
            cudaMalloc(&b->d_prefix, sizeof(int) * (capacity + 1)) == cudaSuccess &&
            cudaMalloc(&b->d_header, sizeof(int) * 2) == cudaSuccess &&
            cudaMallocHost(&b->h_grids, sizeof(lbm::BatchGrid) * capacity) == cudaSuccess &&
            cudaMallocHost(&b->h_prefix, sizeof(int) * (capacity + 1)) == cudaSuccess &&
            cudaMallocHost(&b->h_header, sizeof(int) * 2) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_batch_destroy(b);
    return bfail(nullptr, LBM_ENOMEM, "cannot allocate the batch table");
  }
  cudaEventRecord(b->staged, b->stream);
  int rc = set_ctas(b);
  if (rc) {
    std::string msg = b->err;
    lbm_batch_destroy(b);
    return bfail(nullptr, rc, "%s", msg.c_str());
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_add(lbm_batch* b, lbm_ctx* c) {
  if (!b || !c) return bfail(b, LBM_EINVAL, "batch and ctx are required");
  if (c->batch) return bfail(b, LBM_ESTATE, "ctx is already in a batch");
  if (!c->initialised) return bfail(b, LBM_ESTATE, "ctx is not initialised");
  if (c->lat != b->lat || c->opt.precision != b->precision || c->fo != b->force_order)
    return bfail(b, LBM_EINVAL, "ctx lattice / precision / force order differ from the batch");
  if (c->solid) return bfail(b, LBM_EINVAL, "ctx has solid sites (plain step kernel only)");
  if (c->slab) return bfail(b, LBM_EINVAL, "ctx is a slab (stepped with halo exchanges, not in batches)");
  if (c->stream != b->stream) return bfail(b, LBM_EINVAL, "ctx must use the batch's stream");
  if (c->device != b->device) return bfail(b, LBM_EINVAL, "ctx lives on another device");
  if ((int)b->members.size() >= b->cap) return bfail(b, LBM_ENOMEM, "batch is full (%d)", b->cap);
  b->members.push_back(c);
  c->batch = b;
  b->dirty = true;
  return LBM_OK;
}

int lbm_batch_remove(lbm_batch* b, lbm_ctx* c) {
  if (!b || !c) return bfail(b, LBM_EINVAL, "batch and ctx are required");
  auto it = std::find(b->members.begin(), b->members.end(), c);
  if (it == b->members.end()) return bfail(b, LBM_EINVAL, "ctx is not in this batch");
  b->members.erase(it);
  c->batch = nullptr;
  b->dirty = true;
  return LBM_OK;
}

int lbm_batch_size(const lbm_batch* b) { return b ? (int)b->members.size() : 0; }

int lbm_batch_set_config(lbm_batch* b, int block_x, int sites_per_thread, int graph_steps) {
  if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
  if (block_x < 32 || block_x > 256 || block_x % 32)
    return bfail(b, LBM_EINVAL, "block_x must be a multiple of 32 in [32, 256]");
  if (sites_per_thread != 1 && sites_per_thread != 2)
    return bfail(b, LBM_EINVAL, "sites_per_thread must be 1 or 2");
  if (b->stage && sites_per_thread != 1)
    return bfail(b, LBM_EINVAL, "the halo-staged kernel steps one site per thread");
  if (graph_steps < 0 || graph_steps % 2) return bfail(b, LBM_EINVAL, "graph_steps must be even and >= 0");
  const bool changed = block_x != b->bx || sites_per_thread != b->spt || graph_steps != b->graph_steps;
  b->bx = block_x;
  b->spt = sites_per_thread;
  b->graph_steps = graph_steps;
  if (changed) {
    drop_graph(b);
    b->dirty = true;
    return set_ctas(b);
  }
  return LBM_OK;
}

int lbm_batch_get_config(const lbm_batch* b, int* block_x, int* sites_per_thread, int* graph_steps) {
  if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
  if (block_x) *block_x = b->bx;
  if (sites_per_thread) *sites_per_thread = b->spt;
  if (graph_steps) *graph_steps = b->graph_steps;
  return LBM_OK;
}

int lbm_batch_set_staging(lbm_batch* b, int staged) {
  if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
  if (staged != 0 && staged != 1) return bfail(b, LBM_EINVAL, "staged must be 0 or 1");
  if (staged && b->precision != LBM_FP32_SHIFTED)
    return bfail(b, LBM_EINVAL, "halo staging serves FP32-shifted storage (4-byte populations)");
  if (staged && b->spt != 1) return bfail(b, LBM_EINVAL, "halo staging needs sites_per_thread 1");
  if (staged == b->stage) return LBM_OK;
  const int old = b->stage;
  b->stage = staged;
  drop_graph(b);
  const int rc = set_ctas(b);
  if (rc) b->stage = old;
  return rc;
}

int lbm_batch_get_staging(const lbm_batch* b, int* staged) {
  if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
  if (staged) *staged = b->stage;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n) {
  if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
  if (n < 0) return bfail(b, LBM_EINVAL, "n must be >= 0");
  if (b->members.empty() || n == 0) return LBM_OK;
  BCUDA(b, cudaSetDevice(b->device));
  if (b->dirty) {
    int rc = upload(b);
    if (rc) return rc;
  }
  int done = 0;
  if (b->graph_steps > 0) {
    if (!b->graph && n >= b->graph_steps) {
      int rc = build_graph(b);
      if (rc) return rc;
    }
    for (; n - done >= b->graph_steps; done += b->graph_steps)
      BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
  }
  for (int k = 0; done < n; ++k, ++done) {
    int rc = launch(b, k);
    if (rc) return rc;
  }
  for (auto* c : b->members) {
    c->cur ^= (n & 1);
    c->steps += n;
  }
  if (n & 1) b->dirty = true;
  return LBM_OK;
}

int lbm_batch_tune(lbm_batch* b, int trial_steps, int* block_x, int* sites_per_thread) {
  if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
  if (trial_steps < 2 || trial_steps % 2) return bfail(b, LBM_EINVAL, "trial_steps must be even and >= 2");
  if (b->members.empty()) return bfail(b, LBM_ESTATE, "batch is empty");
  const std::string key = tune_key(b);
  TuneChoice best_c{0, 0, 0};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) best_c = it->second;
  }
  const int G = b->graph_steps;
  if (!best_c.bx) {
    // candidates: block 64 / 128 / 256 x one or two sites per thread, plus
    // the halo-staged kernel (one site per thread) for FP32-shifted storage
    std::vector<TuneChoice> cands;
    for (int bx : {64, 128, 256}) {
      for (int spt : {1, 2}) cands.push_back({bx, spt, 0});
      if (b->precision == LBM_FP32_SHIFTED) cands.push_back({bx, 1, 1});
    }
    cudaEvent_t e0, e1;
    BCUDA(b, cudaEventCreate(&e0));
    BCUDA(b, cudaEventCreate(&e1));
    float best = 1e30f;
    for (const TuneChoice& c : cands) {
      int rc = lbm_batch_set_staging(b, 0);
      if (!rc) rc = lbm_batch_set_config(b, c.bx, c.spt, 0);
      if (!rc) rc = lbm_batch_set_staging(b, c.stage);
      if (!rc) rc = lbm_batch_step(b, 2);  // warm-up
      if (!rc) rc = cudaEventRecord(e0, b->stream) == cudaSuccess ? LBM_OK : LBM_ECUDA;
      if (!rc) rc = lbm_batch_step(b, trial_steps);
      if (!rc) rc = cudaEventRecord(e1, b->stream) == cudaSuccess ? LBM_OK : LBM_ECUDA;
      if (!rc) rc = cudaEventSynchronize(e1) == cudaSuccess ? LBM_OK : LBM_ECUDA;
      float ms = 0.f;
      if (!rc) rc = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess ? LBM_OK : LBM_ECUDA;
      if (rc) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc == LBM_ECUDA ? bfail(b, rc, "tuning trial failed") : rc;
      }
      if (ms < best) {
        best = ms;
        best_c = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best_c;
  }
  int rc = lbm_batch_set_staging(b, 0);
  if (!rc) rc = lbm_batch_set_config(b, best_c.bx, best_c.spt, G);
  if (!rc) rc = lbm_batch_set_staging(b, best_c.stage);
  if (rc) return rc;
  if (block_x) *block_x = best_c.bx;
  if (sites_per_thread) *sites_per_thread = best_c.spt;
  return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) {
  if (!b) return lbm_last_error(nullptr);
  return b->err.empty() ? "no error" : b->err.c_str();
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto* c : b->members) c->batch = nullptr;
  drop_graph(b);
  cudaFree(b->d_grids);
  cudaFree(b->d_prefix);
  cudaFree(b->d_header);
  if (b->h_grids) cudaFreeHost(b->h_grids);
  if (b->h_prefix) cudaFreeHost(b->h_prefix);
  if (b->h_header) cudaFreeHost(b->h_header);
  if (b->staged) cudaEventDestroy(b->staged);
  cudaGetLastError();
  delete b;
}

}  // extern "C"
