// lbm_ctx.h -- the context object behind the opaque lbm_ctx of include/lbm.h
// (private to the library's translation units).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/lbm.h"
#include "lbm_launch.cuh"

struct lbm_batch;

namespace lbm {
// Whether population loads should be evict-first in L2 (ld_pop_policy): the
// working set of a step, `bytes` (both population buffers of every grid the
// launch steps), is below 1.5 times the device's L2 size.
inline int l2_evict_first_for(size_t bytes, int device) {
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device) != cudaSuccess || l2 <= 0) {
    cudaGetLastError();
    return 0;
  }
  return bytes <= (size_t)l2 * 3 / 2 ? 1 : 0;
}
}  // namespace lbm

struct lbm_ctx {
  int lat = 0, D = 0, Q = 0, nx = 0, ny = 0, nz = 0;
  int N = 0;
  double tau = 0.0;
  lbm_options opt{};
  bool overlap = false;        // step kernels launched as programmatic dependents
  int fo = 2;                  // kernel force-order code: opt.force_order, or 3 for
                               // order 2 with the sigma-bar terms
  const lbm::LatticeOps* ops = nullptr;
  size_t elem = 0;             // bytes per stored population value
  void* f[2] = {nullptr, nullptr};
  int cur = 0;                 // f[cur] holds the current post-collision state
  double* gtab = nullptr;      // force table / field
  float* gtab_f = nullptr;     // its float copy (float kernels)
  unsigned char* solid = nullptr;  // solid-site flags (lbm_set_solid), N bytes
  double* wall_th = nullptr;   // wall temperature - 1 per site, N doubles
  float* wall_th_f = nullptr;  // its float copy
  double* part = nullptr;      // conservation partials (CONS_SLOT doubles per block)
  unsigned* bad = nullptr;     // bad-site counts per block
  double* dres = nullptr;      // final reduction result (when hres is not mapped)
  unsigned* ticket = nullptr;  // last-block ticket of the conservation pass
  unsigned* dmax = nullptr;    // FP16 init: max |d/w| bits
  double* hres = nullptr;      // pinned host copy of the result
  double* tmp = nullptr;       // (2 + 2D) * N doubles, lazily allocated
  int nblk_cons = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  lbm::StepParams p{};
  bool initialised = false;
  long long steps = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  size_t bytes = 0;
  int device = 0;
  int* derr = nullptr;         // device flag set by a bounded wait that ran out
  bool use_tma = false;        // TMA-staged step kernel
  CUtensorMap tmap[2];         // tensor maps of f[0], f[1]
  int tma_grid = 0, tma_stages = 0;
  bool use_async = false;      // prefetching persistent step kernel
  int async_grid = 0;
  bool use_wave = false;       // several steps per launch (wavefront order)
  int wave_grid = 0;
  unsigned* wave_sync = nullptr;  // item counter + per-line done counts
  lbm_batch* batch = nullptr;  // batch this context is a member of
  // slab of a grid split along its last axis (lbm_create_slab): the context
  // holds global layers [a_begin, a_end) of that axis after gb ghost layers
  // and before ga ghost layers (3 each, or 0 at a wall); p.a0 = gb and
  // p.na = a_end - a_begin select the layers the kernels step
  bool slab = false;
  int a_begin = 0, a_end = 0, n_axis = 0, gb = 0, ga = 0;
  std::string err;
};

namespace lbm {
// Error reporting shared by the ABI translation units: stores the message on
// the context (or the global slot when ctx is NULL) and returns code.
int ctx_fail(lbm_ctx* c, int code, const char* fmt, ...);
// Batch hooks used by the context entry points.
void batch_mark_dirty(lbm_batch* b);
int batch_detach(lbm_batch* b, lbm_ctx* c);
}  // namespace lbm
