// lbm_abi.cu -- the C ABI declared in include/lbm.h: context management,
// argument validation, device memory, launches on the context's stream.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_launch.cuh"

using lbm::StepParams;

#include "lbm_ctx.h"

namespace {

std::string g_create_error = "no error";

int vfail(lbm_ctx* c, int code, const char* fmt, va_list ap) {
  char buf[512];
  vsnprintf(buf, sizeof buf, fmt, ap);
  if (c) c->err = buf;
  else g_create_error = buf;
  return code;
}

int fail(lbm_ctx* c, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  int rc = vfail(c, code, fmt, ap);
  va_end(ap);
  return rc;
}

#define LBM_CUDA(ctx, call)                                                                   \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, LBM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                  __FILE__, __LINE__);                                                        \
  } while (0)

const lbm::LatticeOps* ops_of(int lat) {
  if (lat == LBM_D2Q37) return &lbm::ops_d2q37();
  if (lat == LBM_D3Q39) return &lbm::ops_d3q39();
  return nullptr;
}

template <class L>
void info_of(int* D, int* Q, double* c, int* e, double* w) {
  if (D) *D = L::D;
  if (Q) *Q = L::Q;
  if (c) *c = L::c;
  for (int i = 0; i < L::Q; ++i) {
    if (e)
      for (int a = 0; a < 3; ++a) e[3 * i + a] = L::e[i][a];
    if (w) w[i] = L::w[i];
  }
}

// The FP16 codec factors of the context's lattice for its current scale.
void fp16_factors(lbm_ctx* c) {
  if (c->lat == LBM_D2Q37) lbm::set_fp16_factors<lbm::D2Q37>(c->p);
  else lbm::set_fp16_factors<lbm::D3Q39>(c->p);
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A pointer kernels can dereference for `ptr`: device and managed memory as
// is, page-locked host memory through its mapped device address (kernels then
// read or write host memory directly over the host link, overlapped with their
// arithmetic, instead of a staging copy); nullptr for pageable host memory.
template <class T>
T* device_view(T* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return ptr;
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<T*>(a.devicePointer);
  return nullptr;
}

int ensure_tmp(lbm_ctx* c) {
  if (c->tmp) return LBM_OK;
  const size_t n = (size_t)(2 + 2 * c->D) * c->N;
  if (cudaMalloc(&c->tmp, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LBM_ENOMEM, "cannot allocate %zu bytes of moment buffers", n * sizeof(double));
  }
  c->bytes += n * sizeof(double);
  return LBM_OK;
}

void drop_graphs(lbm_ctx* c) {
  for (auto& g : c->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    else
      cudaGetLastError();
  }
  return fn;
}

// Tensor maps (x, y, [z,] direction) of both population buffers for the
// TMA-staged kernel.  Returns false when the grid does not qualify.
template <int P>
bool make_tensor_maps(lbm_ctx* c, std::string* why) {
  using G = lbm::TmaGeom<P>;
  const size_t es = G::ES;
  if ((c->nx * es) % 16 || ((size_t)c->N * es) % 16) {
    *why = "nx * element size is not a multiple of 16 bytes";
    return false;
  }
  auto enc = tensor_map_encoder();
  if (!enc) {
    *why = "cuTensorMapEncodeTiled is unavailable";
    return false;
  }
  const CUtensorMapDataType dt = P == lbm::P_FP16S ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  for (int k = 0; k < 2; ++k) {
    CUresult r;
    if (c->D == 2) {
      cuuint64_t dims[3] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, (cuuint64_t)c->Q};
      cuuint64_t strides[2] = {c->nx * es, (cuuint64_t)c->N * es};
      cuuint32_t box[3] = {(cuuint32_t)G::RW, 1, 1};
      cuuint32_t estr[3] = {1, 1, 1};
      r = enc(&c->tmap[k], dt, 3, c->f[k], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
      cuuint64_t dims[4] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, (cuuint64_t)c->nz, (cuuint64_t)c->Q};
      cuuint64_t strides[3] = {c->nx * es, (cuuint64_t)c->nx * c->ny * es, (cuuint64_t)c->N * es};
      cuuint32_t box[4] = {(cuuint32_t)G::RW, 1, 1, 1};
      cuuint32_t estr[4] = {1, 1, 1, 1};
      r = enc(&c->tmap[k], dt, 4, c->f[k], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) {
      *why = "cuTensorMapEncodeTiled rejected the layout";
      return false;
    }
  }
  return true;
}

// Chooses the step kernel; false with *why when the TMA kernel was required
// but cannot be used.
bool setup_step_kernel(lbm_ctx* c, std::string* why) {
  c->use_tma = false;
  c->use_async = false;
  c->use_wave = false;
  if (c->opt.kernel == LBM_KERNEL_WAVE) {
    if (c->opt.precision != LBM_FP32_SHIFTED && c->opt.precision != LBM_FP16_SCALED) {
      *why = "the wavefront kernel serves FP32-shifted and FP16-scaled storage";
      return false;
    }
    if (c->fo > 2) {
      *why = "the sigma-bar terms run in the plain step kernel only";
      return false;
    }
    int bps = 0, nsm = 0;
    cudaError_t e = c->ops->wave_occupancy(c->opt.precision, c->fo, &bps);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess || bps < 1) {
      cudaGetLastError();
      *why = "the wavefront kernel does not fit on this device";
      return false;
    }
    const int nA = c->D == 2 ? c->ny : c->nz;
    if (!c->wave_sync) {
      if (cudaMalloc(&c->wave_sync, sizeof(unsigned) * (1 + (size_t)nA)) != cudaSuccess) {
        cudaGetLastError();
        *why = "cannot allocate the wavefront counters";
        return false;
      }
      c->bytes += sizeof(unsigned) * (1 + (size_t)nA);
    }
    c->wave_grid = bps * nsm;
    c->use_wave = true;
    return true;
  }
  if (c->opt.kernel == LBM_KERNEL_PREFETCH) {
    if (c->opt.precision != LBM_FP32_SHIFTED) {
      *why = "the prefetching kernel serves FP32-shifted storage only";
      return false;
    }
    int bps = 0, nsm = 0;
    cudaError_t e = c->ops->async_occupancy(c->fo, c->opt.block_x, &bps);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess || bps < 1) {
      cudaGetLastError();
      *why = "the prefetching kernel does not fit with this block size";
      return false;
    }
    const long long tiles = (long long)((c->nx + c->opt.block_x - 1) / c->opt.block_x) * c->ny * c->nz;
    c->async_grid = (int)std::min<long long>(tiles, (long long)nsm * bps);
    c->use_async = true;
    return true;
  }
  // AUTO runs the plain kernel: on GB300 the TMA-staged variant measured ~2x
  // slower (its 12 resident warps per SM cannot hide the collision phase);
  // it stays available on request and to the autotuner.
  if (c->opt.kernel != LBM_KERNEL_TMA) return true;
  const int P = c->opt.precision;
  bool ok = false;
  if (P == LBM_FP32_SHIFTED) ok = make_tensor_maps<lbm::P_FP32S>(c, why);
  else if (P == LBM_FP16_SCALED) ok = make_tensor_maps<lbm::P_FP16S>(c, why);
  else *why = "the TMA-staged kernel serves FP32 and FP16 storage only";
  if (ok) {
    int bps = 0, nsm = 0;
    c->tma_stages = c->opt.tma_stages > 0 ? c->opt.tma_stages : 3;
    cudaError_t e = c->ops->tma_prepare(P, c->tma_stages, &bps);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess || bps < 1) {
      cudaGetLastError();
      *why = "the TMA-staged kernel does not fit on this device with these stages";
      ok = false;
    } else {
      const long long tiles = (long long)((c->nx + lbm::TMA_W - 1) / lbm::TMA_W) * c->ny * c->nz;
      c->tma_grid = (int)std::min<long long>(tiles, (long long)nsm * bps);
    }
  }
  c->use_tma = ok;
  return ok || c->opt.kernel == LBM_KERNEL_AUTO;
}

// n steps of the wavefront kernel: launches of at most as many steps as keep
// the item count below 2^31, each after zeroing its counters.
int launch_wave_steps(lbm_ctx* c, int n) {
  const int nA = c->D == 2 ? c->ny : c->nz;
  const long long per_step = (long long)((c->nx + lbm::WAVE_BX - 1) / lbm::WAVE_BX) * c->ny * c->nz;
  const int kmax = (int)std::max<long long>(1, ((1LL << 31) - 1) / per_step);
  while (n > 0) {
    const int k = std::min(n, kmax);
    LBM_CUDA(c, cudaMemsetAsync(c->wave_sync, 0, sizeof(unsigned) * (1 + (size_t)nA), c->stream));
    cudaError_t e = c->ops->step_wave(c->opt.precision, c->fo, c->f[c->cur], c->f[c->cur ^ 1], c->p,
                                      k, c->wave_sync, c->wave_grid, c->stream);
    if (e != cudaSuccess) return fail(c, LBM_ECUDA, "wavefront launch failed: %s", cudaGetErrorString(e));
    c->cur ^= k & 1;
    n -= k;
  }
  return LBM_OK;
}

int launch_one_step(lbm_ctx* c) {
  cudaError_t e;
  if (c->use_tma)
    e = c->ops->step_tma(c->opt.precision, c->fo, &c->tmap[c->cur], c->f[c->cur],
                         c->f[c->cur ^ 1], c->p, c->tma_grid, c->tma_stages, c->stream);
  else if (c->use_async)
    e = c->ops->step_async(c->fo, c->f[c->cur], c->f[c->cur ^ 1], c->p, c->async_grid,
                           c->opt.block_x, c->stream);
  else
    e = c->ops->step(c->opt.fp64_arith == LBM_ARITH_FLOAT_PAIR ? (int)lbm::P_FP64DF : c->opt.precision,
                     c->fo, c->f[c->cur], c->f[c->cur ^ 1], c->p, c->opt.block_x, c->overlap, c->stream);
  if (e != cudaSuccess) return fail(c, LBM_ECUDA, "step launch failed: %s", cudaGetErrorString(e));
  c->cur ^= 1;
  return LBM_OK;
}

// Graph of graph_steps steps starting from buffer parity `par` (even length,
// so the parity is restored).
int build_graph(lbm_ctx* c, int par) {
  cudaGraph_t g = nullptr;
  const int saved = c->cur;
  c->cur = par;
  LBM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int rc = LBM_OK;
  if (c->use_wave) rc = launch_wave_steps(c, c->opt.graph_steps);
  else
    for (int k = 0; k < c->opt.graph_steps && rc == LBM_OK; ++k) rc = launch_one_step(c);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  c->cur = saved;
  if (rc != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(c, LBM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->graph[par], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, LBM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_options_size(void) { return sizeof(lbm_options); }

void lbm_default_options(lbm_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = LBM_FP64;
  o->force_order = 2;
  o->include_sigma = 0;
  for (int a = 0; a < 3; ++a) {
    o->bc[a] = LBM_PERIODIC;
    o->T_lo[a] = 1.0;
    o->T_hi[a] = 1.0;
  }
  o->stream = nullptr;
  o->block_x = 0;
  o->graph_steps = 0;
  o->kernel = LBM_KERNEL_AUTO;
  o->tma_stages = 0;
  o->mu = 0.0;
  o->overlap_steps = -1;
}

int lbm_lattice_info(lbm_lattice lat, int* D, int* Q, double* c, int* e, double* w) {
  if (lat == LBM_D2Q37) info_of<lbm::D2Q37>(D, Q, c, e, w);
  else if (lat == LBM_D3Q39) info_of<lbm::D3Q39>(D, Q, c, e, w);
  else return fail(nullptr, LBM_EINVAL, "unknown lattice %d", (int)lat);
  return LBM_OK;
}

}  // extern "C"

namespace {
// A slab of the last axis (lbm_create_slab): global layers [a_begin, a_end).
struct SlabSpec {
  int a_begin, a_end;
};

int create_impl(lbm_lattice lat, int nx, int ny, int nz, double tau, const lbm_gfield* g,
                const lbm_options* opt, const SlabSpec* slab, lbm_ctx** out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  const lbm::LatticeOps* ops = ops_of(lat);
  if (!ops) return fail(nullptr, LBM_EINVAL, "unknown lattice %d", (int)lat);
  lbm_options o;
  if (opt) o = *opt;
  else lbm_default_options(&o);
  const int D = ops->D;
  if (D == 2 && nz != 1) return fail(nullptr, LBM_EINVAL, "D2Q37 needs nz == 1 (got %d)", nz);
  if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_EINVAL, "grid %dx%dx%d is empty", nx, ny, nz);
  const long long N = (long long)nx * ny * nz;
  if (N >= (1LL << 31)) return fail(nullptr, LBM_EINVAL, "grid has %lld >= 2^31 sites", N);
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(nullptr, LBM_EINVAL, "tau-hat must be > 1/2 (got %g)", tau);
  if (o.precision < LBM_FP64 || o.precision > LBM_FP16_SCALED)
    return fail(nullptr, LBM_EINVAL, "unknown precision %d", o.precision);
  if (o.force_order < 0 || o.force_order > 2)
    return fail(nullptr, LBM_EINVAL, "force_order must be 0, 1 or 2 (got %d)", o.force_order);
  if (o.include_sigma && o.force_order == 2 &&
      (o.kernel == LBM_KERNEL_TMA || o.kernel == LBM_KERNEL_PREFETCH || o.kernel == LBM_KERNEL_WAVE))
    return fail(nullptr, LBM_EINVAL, "the sigma-bar terms run in the plain step kernel only");
  const int n[3] = {nx, ny, nz};
  int wall = lbm::W_NONE;
  for (int a = 0; a < 3; ++a) {
    const int b = a < D ? o.bc[a] : LBM_PERIODIC;
    if (b < LBM_PERIODIC || b > LBM_THERMAL_WALL) return fail(nullptr, LBM_EINVAL, "bad bc[%d] = %d", a, b);
    if (b != LBM_PERIODIC) {
      if (a != D - 1) return fail(nullptr, LBM_EINVAL, "walls are supported on the last axis only (axis %d)", D - 1);
      if (n[a] < 6) return fail(nullptr, LBM_EINVAL, "a walled axis needs >= 6 sites (got %d)", n[a]);
      wall = b == LBM_BOUNCE_BACK ? lbm::W_BOUNCE : lbm::W_THERMAL;
    } else if (a < D && n[a] < 3) {
      return fail(nullptr, LBM_EINVAL, "a periodic axis needs >= 3 sites (axis %d has %d)", a, n[a]);
    }
  }
  if (o.block_x == 0) {
    // 128 threads, narrowed (down to one warp) while the row tiles would
    // leave SMs idle: small grids are latency bound per block, not HBM bound
    o.block_x = 128;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
      while (o.block_x > 32 && (long long)((nx + o.block_x - 1) / o.block_x) * ny * nz < 2LL * nsm)
        o.block_x /= 2;
    }
    cudaGetLastError();
  }
  if (o.block_x < 32 || o.block_x > 256 || o.block_x % 32)
    return fail(nullptr, LBM_EINVAL, "block_x must be a multiple of 32 in [32, 256] (got %d)", o.block_x);
  if (o.graph_steps < 0 || o.graph_steps % 2)
    return fail(nullptr, LBM_EINVAL, "graph_steps must be even and >= 0 (got %d)", o.graph_steps);
  if (o.kernel < LBM_KERNEL_AUTO || o.kernel > LBM_KERNEL_WAVE)
    return fail(nullptr, LBM_EINVAL, "unknown kernel choice %d", o.kernel);
  if (!(o.mu >= 0.0) || !std::isfinite(o.mu)) return fail(nullptr, LBM_EINVAL, "mu must be >= 0");
  if (o.overlap_steps < -1 || o.overlap_steps > 1)
    return fail(nullptr, LBM_EINVAL, "overlap_steps must be -1, 0 or 1 (got %d)", o.overlap_steps);
  if (o.fp64_arith != LBM_ARITH_DOUBLE) {
    if (o.fp64_arith != LBM_ARITH_FLOAT_PAIR)
      return fail(nullptr, LBM_EINVAL, "fp64_arith must be LBM_ARITH_DOUBLE or LBM_ARITH_FLOAT_PAIR");
    if (o.precision != LBM_FP64) return fail(nullptr, LBM_EINVAL, "fp64_arith needs LBM_FP64 storage");
    if (o.storage_probe != 0) return fail(nullptr, LBM_EINVAL, "fp64_arith and storage_probe exclude each other");
    if (o.kernel != LBM_KERNEL_AUTO && o.kernel != LBM_KERNEL_PLAIN)
      return fail(nullptr, LBM_EINVAL, "fp64_arith runs in the plain step kernel only");
  }
  if (o.storage_probe != 0) {
    if (o.storage_probe != LBM_FP32_SHIFTED && o.storage_probe != LBM_FP16_SCALED)
      return fail(nullptr, LBM_EINVAL, "storage_probe must be 0, LBM_FP32_SHIFTED or LBM_FP16_SCALED");
    if (o.precision != LBM_FP64)
      return fail(nullptr, LBM_EINVAL, "storage_probe needs LBM_FP64 storage");
    if (o.kernel != LBM_KERNEL_AUTO && o.kernel != LBM_KERNEL_PLAIN)
      return fail(nullptr, LBM_EINVAL, "storage_probe runs in the plain step kernel only");
  }
  if (o.tma_stages != 0 && (o.tma_stages < 2 || o.tma_stages > 8))
    return fail(nullptr, LBM_EINVAL, "tma_stages must be 0 or 2..8 (got %d)", o.tma_stages);
  lbm_gfield gf{};
  gf.kind = LBM_G_UNIFORM;
  if (g) gf = *g;
  if (gf.kind < LBM_G_UNIFORM || gf.kind > LBM_G_FIELD) return fail(nullptr, LBM_EINVAL, "bad force kind %d", gf.kind);
  if (gf.kind == LBM_G_SINE && (gf.wave_axis < 0 || gf.wave_axis >= D))
    return fail(nullptr, LBM_EINVAL, "bad wave_axis %d", gf.wave_axis);
  if (gf.kind == LBM_G_FIELD && !gf.field) return fail(nullptr, LBM_EINVAL, "force field is NULL");
  // slab: the buffer holds the slab's layers plus 3 ghost layers on each side
  // that is not a wall (the pull reaches 3 layers along every axis)
  const int A = D - 1, nAg = n[A];
  int gb = 0, ga = 0, na = nAg, a_begin = 0;
  if (slab) {
    if (slab->a_begin < 0 || slab->a_end > nAg || slab->a_end - slab->a_begin < 3)
      return fail(nullptr, LBM_EINVAL, "slab layers [%d, %d) must lie in [0, %d) and number at least 3",
                  slab->a_begin, slab->a_end, nAg);
    if (o.kernel != LBM_KERNEL_AUTO && o.kernel != LBM_KERNEL_PLAIN)
      return fail(nullptr, LBM_EINVAL, "slabs run in the plain step kernel");
    if (o.graph_steps != 0)
      return fail(nullptr, LBM_EINVAL, "slabs are stepped one step at a time (graph_steps must be 0)");
    if (o.storage_probe != 0) return fail(nullptr, LBM_EINVAL, "slabs take no storage probe");
    const bool periodic = wall == lbm::W_NONE;
    gb = (periodic || slab->a_begin > 0) ? 3 : 0;
    ga = (periodic || slab->a_end < nAg) ? 3 : 0;
    na = slab->a_end - slab->a_begin;
    a_begin = slab->a_begin;
  }
  const int nb = na + gb + ga;  // buffer layers along the last axis
  const int bny = D == 2 ? nb : ny, bnz = D == 3 ? nb : nz;
  const long long S = D == 2 ? (long long)nx : (long long)nx * ny;  // sites per layer
  const long long NB = S * nb;
  if (NB >= (1LL << 31)) return fail(nullptr, LBM_EINVAL, "slab buffer has %lld >= 2^31 sites", NB);

  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return fail(nullptr, LBM_ENOMEM, "out of host memory");
  c->lat = lat; c->D = D; c->Q = ops->Q; c->nx = nx; c->ny = bny; c->nz = bnz; c->N = (int)NB;
  c->slab = slab != nullptr;
  c->a_begin = a_begin; c->a_end = a_begin + na; c->n_axis = nAg; c->gb = gb; c->ga = ga;
  c->tau = tau; c->opt = o; c->ops = ops;
  c->fo = o.include_sigma && o.force_order == 2 ? 3 : o.force_order;
  // measured on GB300: +1.3 to +2 % (graphs) and +7 % (plain launches) on
  // 524 k sites; on grids of a few thousand sites the sign varied between
  // runs (-10 % to +10 %), so those keep plain stream order by default
  c->overlap = o.overlap_steps == 1 || (o.overlap_steps < 0 && N >= LBM_OVERLAP_MIN_SITES);
  c->elem = o.precision == LBM_FP64 ? 8 : (o.precision == LBM_FP32_SHIFTED ? 4 : 2);
  cudaGetDevice(&c->device);
  auto bail = [&](int rc) {
    const std::string msg = c->err;
    lbm_destroy(c);
    g_create_error = msg;
    return rc;
  };
  if (o.stream) {
    c->stream = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreate(&c->stream) != cudaSuccess) {
      cudaGetLastError();
      fail(c, LBM_ECUDA, "cudaStreamCreate failed");
      return bail(LBM_ECUDA);
    }
    c->own_stream = true;
  }
  const size_t fbytes = (size_t)c->Q * NB * c->elem;
  for (int k = 0; k < 2; ++k) {
    if (cudaMalloc(&c->f[k], fbytes) != cudaSuccess) {
      cudaGetLastError();
      fail(c, LBM_ENOMEM, "cannot allocate %zu bytes of populations", fbytes);
      return bail(LBM_ENOMEM);
    }
    c->bytes += fbytes;
  }
  // parameters
  StepParams& p = c->p;
  p.nx = nx; p.ny = bny; p.nz = bnz; p.N = (int)NB; p.wall = wall;
  p.a0 = gb;
  p.na = na;
  p.omega = 1.0 / tau;
  p.gkind = gf.kind; p.gaxis = gf.wave_axis;
  for (int a = 0; a < 3; ++a) p.g0[a] = a < D ? gf.g0[a] : 0.0;
  p.omega_f = (float)p.omega;
  p.mu_f = (float)o.mu;
  p.mu = p.mu_f > 0.0f ? o.mu : 0.0;  // the same switch in both precisions
  if (p.mu == 0.0) p.mu_f = 0.0f;
  for (int a = 0; a < 3; ++a) p.g0_f[a] = (float)p.g0[a];
  p.h_scale = 1.0f; p.h_inv_scale = 1.0f;
  fp16_factors(c);
  p.l2_evict_first = lbm::l2_evict_first_for(2 * fbytes, c->device);
  p.storage_probe = o.storage_probe;
  if (wall != lbm::W_NONE) {
    if (lat == LBM_D2Q37) lbm::wall_tables<lbm::D2Q37>(p, o.T_lo[D - 1], o.T_hi[D - 1]);
    else lbm::wall_tables<lbm::D3Q39>(p, o.T_lo[D - 1], o.T_hi[D - 1]);
  }
  // table length along the wave axis: the buffer's layers on a slab's last axis
  const int bn[3] = {nx, bny, bnz};
  if (gf.kind == LBM_G_SINE) {
    const int nw = n[gf.wave_axis], nt = bn[gf.wave_axis];
    const int off = gf.wave_axis == A ? a_begin - gb : 0;  // global index of table entry 0
    double* h = (double*)std::malloc(sizeof(double) * nt);
    if (!h) { fail(c, LBM_ENOMEM, "out of host memory"); return bail(LBM_ENOMEM); }
    for (int k = 0; k < nt; ++k) h[k] = std::sin(2.0 * M_PI * (((off + k) % nw + nw) % nw) / nw);
    cudaError_t e = cudaMalloc(&c->gtab, sizeof(double) * nt);
    if (e == cudaSuccess) e = cudaMemcpy(c->gtab, h, sizeof(double) * nt, cudaMemcpyHostToDevice);
    std::free(h);
    if (e != cudaSuccess) { cudaGetLastError(); fail(c, LBM_ECUDA, "force table upload failed"); return bail(LBM_ECUDA); }
    c->bytes += sizeof(double) * nt;
  } else if (gf.kind == LBM_G_FIELD) {
    // the caller's field covers the grid (a slab's own layers); the buffer's
    // ghost layers are never read and stay zero
    const size_t gbytes = sizeof(double) * D * NB;
    const size_t nuser = (size_t)S * na;
    cudaError_t e = cudaMalloc(&c->gtab, gbytes);
    if (e == cudaSuccess) e = cudaMemset(c->gtab, 0, gbytes);
    for (int k = 0; k < D && e == cudaSuccess; ++k)
      e = cudaMemcpy(c->gtab + (size_t)k * NB + (size_t)gb * S, gf.field + (size_t)k * nuser,
                     sizeof(double) * nuser, cudaMemcpyDefault);
    if (e != cudaSuccess) { cudaGetLastError(); fail(c, LBM_ECUDA, "force field upload failed"); return bail(LBM_ECUDA); }
    c->bytes += gbytes;
  }
  p.gtab = c->gtab;
  if (c->gtab) {  // float copy of the force table for the float kernels
    const size_t cnt = gf.kind == LBM_G_SINE ? (size_t)bn[gf.wave_axis] : (size_t)D * NB;
    float* ft = nullptr;
    double* h = (double*)std::malloc(sizeof(double) * cnt);
    float* hf = (float*)std::malloc(sizeof(float) * cnt);
    cudaError_t e = (h && hf) ? cudaMemcpy(h, c->gtab, sizeof(double) * cnt, cudaMemcpyDeviceToHost)
                              : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) {
      for (size_t k = 0; k < cnt; ++k) hf[k] = (float)h[k];
      e = cudaMalloc(&ft, sizeof(float) * cnt);
    }
    if (e == cudaSuccess) e = cudaMemcpy(ft, hf, sizeof(float) * cnt, cudaMemcpyHostToDevice);
    std::free(h);
    std::free(hf);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(ft);
      fail(c, LBM_ECUDA, "float force table upload failed");
      return bail(LBM_ECUDA);
    }
    c->gtab_f = ft;
    c->bytes += sizeof(float) * cnt;
    p.gtab_f = ft;
  }
  // reduction scratch: a grid-stride pass of at most 4 blocks per SM
  {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    const long long tiles = (long long)((nx + 127) / 128) * (D == 2 ? na : (long long)ny * na);
    c->nblk_cons = (int)std::min<long long>(tiles, (long long)LBM_CONSERVED_BLOCKS * (nsm > 0 ? nsm : 1));
  }
  const size_t pb = sizeof(double) * lbm::CONS_SLOT * c->nblk_cons;
  if (cudaMalloc(&c->part, pb) != cudaSuccess || cudaMalloc(&c->bad, sizeof(unsigned) * c->nblk_cons) != cudaSuccess ||
      cudaMalloc(&c->dres, sizeof(double) * (2 * lbm::NCONS + 2)) != cudaSuccess ||
      cudaMalloc(&c->dmax, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&c->ticket, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->ticket, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&c->hres, sizeof(double) * (2 * lbm::NCONS + 2)) != cudaSuccess) {
    cudaGetLastError();
    fail(c, LBM_ENOMEM, "cannot allocate reduction scratch");
    return bail(LBM_ENOMEM);
  }
  c->bytes += pb + sizeof(unsigned) * c->nblk_cons + sizeof(double) * (2 * lbm::NCONS + 2) + 2 * sizeof(unsigned);
  if (cudaMalloc(&c->derr, sizeof(int)) != cudaSuccess || cudaMemset(c->derr, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    fail(c, LBM_ENOMEM, "cannot allocate the error flag");
    return bail(LBM_ENOMEM);
  }
  c->bytes += sizeof(int);
  p.err = c->derr;
  {
    std::string why;
    if (!setup_step_kernel(c, &why)) {
      fail(c, LBM_EINVAL, "TMA-staged kernel unavailable: %s", why.c_str());
      return bail(LBM_EINVAL);
    }
  }
  *out = c;
  return LBM_OK;
}

// ---- halo exchange of slabs
// One halo message: the planes (a layer of one population) that the
// neighbour's own sites pull from its ghost layers.  A site pulls
// f*_i(x - e_i), so a neighbour above reads population i with e_iA > 0 from
// its ghost layer g (0 = farthest, 2 = adjacent to its own layers) when
// e_iA >= 3 - g, and a neighbour below reads population i with e_iA < 0 from
// its ghost layer h (0 = adjacent) when -e_iA >= h + 1.
constexpr int kMaxHaloPlanes = 32;
struct HaloPlanes {
  int n;
  long long src[kMaxHaloPlanes], dst[kMaxHaloPlanes];  // element offsets of each plane
};

// dir 1: the message to the neighbour above (its lower ghosts), dir 0: to the
// neighbour below (its upper ghosts); (g, i) in message order.
int halo_list(const lbm_ctx* c, int dir, int* layer, int* pop) {
  int e[39 * 3];
  lbm_lattice_info((lbm_lattice)c->lat, nullptr, nullptr, nullptr, e, nullptr);
  const int A = c->D - 1;
  int n = 0;
  for (int g = 0; g < 3; ++g)
    for (int i = 0; i < c->Q; ++i) {
      const int eA = e[3 * i + A];
      const bool take = dir == 1 ? eA >= 3 - g : -eA >= g + 1;
      if (take) {
        layer[n] = g;
        pop[n] = i;
        ++n;
      }
    }
  return n;
}

size_t layer_sites(const lbm_ctx* c) { return (size_t)(c->D == 2 ? c->nx : c->nx * c->ny); }

// Plane offsets for sending dir's message out of `from` (its own layers) and
// writing it into `to`'s ghost layers; either side may be a contiguous
// message instead (from == nullptr: source is the message, to == nullptr:
// destination is the message).
HaloPlanes halo_planes(const lbm_ctx* ref, int dir, const lbm_ctx* from, const lbm_ctx* to) {
  int layer[kMaxHaloPlanes * 2], pop[kMaxHaloPlanes * 2];
  HaloPlanes hp{};
  hp.n = halo_list(ref, dir, layer, pop);
  const long long S = (long long)layer_sites(ref);
  for (int k = 0; k < hp.n; ++k) {
    const int g = layer[k], i = pop[k];
    // source layer in `from`: the top three own layers (dir 1) or the bottom three (dir 0)
    hp.src[k] = from ? (long long)i * from->N +
                           (long long)(dir == 1 ? from->gb + (from->a_end - from->a_begin) - 3 + g : from->gb + g) * S
                     : (long long)k * S;
    // destination ghost layer in `to`: below its own layers (dir 1) or above (dir 0)
    hp.dst[k] = to ? (long long)i * to->N +
                         (long long)(dir == 1 ? g : to->gb + (to->a_end - to->a_begin) + g) * S
                   : (long long)k * S;
  }
  return hp;
}

template <class T>
__global__ void __launch_bounds__(256) k_halo_copy(const T* __restrict__ src, T* __restrict__ dst,
                                                   const HaloPlanes hp, long long S) {
  const int k = blockIdx.y;
  const T* s = src + hp.src[k];
  T* d = dst + hp.dst[k];
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < S; j += (long long)gridDim.x * blockDim.x)
    d[j] = s[j];
}

cudaError_t launch_halo(const void* src, void* dst, const HaloPlanes& hp, size_t S, size_t elem,
                        cudaStream_t st) {
  if (hp.n == 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min<size_t>((S + 255) / 256, 1024), (unsigned)hp.n);
  if (elem == 8) k_halo_copy<unsigned long long><<<grid, 256, 0, st>>>((const unsigned long long*)src, (unsigned long long*)dst, hp, (long long)S);
  else if (elem == 4) k_halo_copy<unsigned><<<grid, 256, 0, st>>>((const unsigned*)src, (unsigned*)dst, hp, (long long)S);
  else k_halo_copy<unsigned short><<<grid, 256, 0, st>>>((const unsigned short*)src, (unsigned short*)dst, hp, (long long)S);
  return cudaGetLastError();
}

// v <- half(float(v) * factor) over n halves (factor a power of two).
__global__ void k_rescale_half(unsigned short* __restrict__ f, size_t n, float factor) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x)
    f[j] = __half_as_ushort(__float2half_rn(__half2float(__ushort_as_half(f[j])) * factor));
}

// Sites of the caller's arrays: the whole grid, or a slab's own layers.
size_t user_sites(const lbm_ctx* c) {
  return c->slab ? (size_t)(c->D == 2 ? c->nx : c->nx * c->ny) * (c->a_end - c->a_begin) : (size_t)c->N;
}
// Offset of a slab's first own site in its buffer (0 without a slab).
size_t user_offset(const lbm_ctx* c) {
  return c->slab ? (size_t)(c->D == 2 ? c->nx : c->nx * c->ny) * c->gb : 0;
}
// rows x n doubles between a caller array (row stride n_user) and a buffer
// laid out like the context (row stride N, own sites from user_offset)
cudaError_t copy_rows(lbm_ctx* c, double* dst, const double* src, int rows, bool to_user) {
  const size_t nu = user_sites(c), nb = (size_t)c->N, off = user_offset(c);
  if (to_user)
    return cudaMemcpy2DAsync(dst, nu * sizeof(double), src + off, nb * sizeof(double), nu * sizeof(double), rows,
                             cudaMemcpyDefault, c->stream);
  return cudaMemcpy2DAsync(dst + off, nb * sizeof(double), src, nu * sizeof(double), nu * sizeof(double), rows,
                           cudaMemcpyDefault, c->stream);
}
}  // namespace

extern "C" {

int lbm_create(lbm_lattice lat, int nx, int ny, int nz, double tau, const lbm_gfield* g,
               const lbm_options* opt, lbm_ctx** out) {
  return create_impl(lat, nx, ny, nz, tau, g, opt, nullptr, out);
}

int lbm_create_slab(lbm_lattice lat, int nx, int ny, int nz, int a_begin, int a_end, double tau,
                    const lbm_gfield* g, const lbm_options* opt, lbm_ctx** out) {
  const SlabSpec s{a_begin, a_end};
  return create_impl(lat, nx, ny, nz, tau, g, opt, &s, out);
}

int lbm_init(lbm_ctx* c, const double* rho, const double* u, const double* T) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (!rho || !u || !T) return fail(c, LBM_EINVAL, "rho, u and T are required");
  LBM_CUDA(c, cudaSetDevice(c->device));
  const size_t N = (size_t)c->N;
  const double *drho = device_view(rho), *du = device_view(u), *dT = device_view(T);
  const bool dev = drho && du && dT && !c->slab;
  if (c->slab) {
    int rc = ensure_tmp(c);
    if (rc) return rc;
    double* t = c->tmp;
    LBM_CUDA(c, copy_rows(c, t, rho, 1, false));
    LBM_CUDA(c, copy_rows(c, t + N, u, c->D, false));
    LBM_CUDA(c, copy_rows(c, t + (1 + c->D) * N, T, 1, false));
    drho = t; du = t + N; dT = t + (1 + c->D) * N;
  } else if (!dev) {
    int rc = ensure_tmp(c);
    if (rc) return rc;
    double* t = c->tmp;
    LBM_CUDA(c, cudaMemcpyAsync(t, rho, N * sizeof(double), cudaMemcpyDefault, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync(t + N, u, c->D * N * sizeof(double), cudaMemcpyDefault, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync(t + (1 + c->D) * N, T, N * sizeof(double), cudaMemcpyDefault, c->stream));
    drho = t; du = t + N; dT = t + (1 + c->D) * N;
  }
  c->cur = 0;
  if (c->opt.precision == LBM_FP16_SCALED || c->opt.storage_probe == LBM_FP16_SCALED) {
    LBM_CUDA(c, cudaMemsetAsync(c->dmax, 0, sizeof(unsigned), c->stream));
    LBM_CUDA(c, c->ops->init(c->opt.precision, 0, drho, du, dT, c->f[0], c->dmax, c->opt.force_order, c->p, c->stream));
    unsigned bits = 0;
    LBM_CUDA(c, cudaMemcpyAsync(&bits, c->dmax, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    float mx;
    std::memcpy(&mx, &bits, sizeof mx);
    if (!std::isfinite(mx)) return fail(c, LBM_EINVAL, "initial state is not finite");
    // scale s = 2^k with max |d/w| * s in [2^12, 2^13): headroom of 8x below the
    // half-precision maximum for the state to grow into
    int k = 0;
    if (mx > 0.f) k = 12 - (int)std::floor(std::log2((double)mx));
    if (k > 60) k = 60;
    if (k < -60) k = -60;
    const float scale = std::ldexp(1.0f, k);
    if (scale != c->p.h_scale) drop_graphs(c);  // captured launches hold the old scale
    c->p.h_scale = scale;
    c->p.h_inv_scale = std::ldexp(1.0f, -k);
    fp16_factors(c);
  }
  LBM_CUDA(c, c->ops->init(c->opt.precision, 1, drho, du, dT, c->f[0], nullptr, c->opt.force_order, c->p, c->stream));
  // host arrays (staged or read in place) may be freed after return
  if (!is_device_ptr(rho) || !is_device_ptr(u) || !is_device_ptr(T))
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->initialised = true;
  c->steps = 0;
  lbm::batch_mark_dirty(c->batch);  // buffer parity and FP16 scale may have changed
  return LBM_OK;
}

int lbm_set_solid(lbm_ctx* c, const unsigned char* solid, const double* T_wall) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (!solid || !T_wall) return fail(c, LBM_EINVAL, "solid and T_wall are required");
  if (c->initialised) return fail(c, LBM_ESTATE, "lbm_set_solid must precede lbm_init");
  if (c->batch) return fail(c, LBM_ESTATE, "ctx is in a batch");
  if (c->p.wall != lbm::W_NONE) return fail(c, LBM_EINVAL, "solid sites need all axes periodic");
  if (c->slab) return fail(c, LBM_EINVAL, "solid sites are not supported on slabs");
  if (c->opt.fp64_arith != LBM_ARITH_DOUBLE)
    return fail(c, LBM_EINVAL, "solid sites run with IEEE double arithmetic (fp64_arith 0)");
  if (c->opt.precision == LBM_FP16_SCALED)
    return fail(c, LBM_EINVAL, "solid sites run with FP64 or FP32-shifted storage");
  if (c->use_tma || c->use_async || c->use_wave)
    return fail(c, LBM_EINVAL, "solid sites run in the plain step kernel");
  LBM_CUDA(c, cudaSetDevice(c->device));
  const size_t N = (size_t)c->N;
  std::vector<unsigned char> s(N);
  std::vector<double> th(N, 0.0);
  std::vector<float> thf(N, 0.f);
  for (size_t k = 0; k < N; ++k) {
    s[k] = solid[k] ? 1 : 0;
    if (s[k]) {
      if (!(T_wall[k] > 0.0) || !std::isfinite(T_wall[k]))
        return fail(c, LBM_EINVAL, "wall temperature at site %zu must be positive", k);
      th[k] = T_wall[k] - 1.0;
      thf[k] = (float)th[k];
    }
  }
  if (!c->solid) {
    if (cudaMalloc(&c->solid, N) != cudaSuccess || cudaMalloc(&c->wall_th, N * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->wall_th_f, N * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, LBM_ENOMEM, "device allocation of the solid-site tables failed");
    }
    c->bytes += N * (1 + sizeof(double) + sizeof(float));
  }
  LBM_CUDA(c, cudaMemcpy(c->solid, s.data(), N, cudaMemcpyHostToDevice));
  LBM_CUDA(c, cudaMemcpy(c->wall_th, th.data(), N * sizeof(double), cudaMemcpyHostToDevice));
  LBM_CUDA(c, cudaMemcpy(c->wall_th_f, thf.data(), N * sizeof(float), cudaMemcpyHostToDevice));
  c->p.solid = c->solid;
  c->p.wall_th = c->wall_th;
  c->p.wall_th_f = c->wall_th_f;
  drop_graphs(c);
  return LBM_OK;
}

int lbm_step(lbm_ctx* c, int n) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0 (got %d)", n);
  if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_step before lbm_init");
  if (c->batch) return fail(c, LBM_ESTATE, "ctx is stepped by its batch (lbm_batch_step)");
  LBM_CUDA(c, cudaSetDevice(c->device));
  int left = n;
  const int G = c->opt.graph_steps;
  while (G > 0 && left >= G) {
    if (!c->graph[c->cur]) {
      int rc = build_graph(c, c->cur);
      if (rc) return rc;
    }
    LBM_CUDA(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
    left -= G;
  }
  if (c->use_wave && left > 0) {
    int rc = launch_wave_steps(c, left);
    if (rc) return rc;
    left = 0;
  }
  for (; left > 0; --left) {
    int rc = launch_one_step(c);
    if (rc) return rc;
  }
  c->steps += n;
  return LBM_OK;
}

int lbm_moments(lbm_ctx* c, double* rho, double* u, double* T, double* q) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_moments before lbm_init");
  LBM_CUDA(c, cudaSetDevice(c->device));
  int rc = ensure_tmp(c);
  if (rc) return rc;
  const size_t N = (size_t)c->N;
  double* outs[4] = {rho, u, T, q};
  const size_t cnt[4] = {N, c->D * N, N, c->D * N};
  double* dst[4];
  bool staged[4];
  double* t = c->tmp;
  for (int k = 0; k < 4; ++k) {
    dst[k] = outs[k] && !c->slab ? device_view(outs[k]) : nullptr;
    staged[k] = outs[k] && !dst[k];
    if (staged[k]) dst[k] = t;
    t += cnt[k];
  }
  LBM_CUDA(c, c->ops->moments(c->opt.precision, c->f[c->cur], dst[0], dst[1], dst[2], dst[3],
                              c->fo, c->p, c->stream));
  const int rows[4] = {1, c->D, 1, c->D};
  for (int k = 0; k < 4; ++k)
    if (staged[k]) {
      if (c->slab) LBM_CUDA(c, copy_rows(c, outs[k], dst[k], rows[k], true));
      else LBM_CUDA(c, cudaMemcpyAsync(outs[k], dst[k], cnt[k] * sizeof(double), cudaMemcpyDefault, c->stream));
    }
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_moments_async(lbm_ctx* c, double* rho, double* u, double* T, double* q) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_moments_async before lbm_init");
  double* outs[4] = {rho, u, T, q};
  double* dst[4];
  for (int k = 0; k < 4; ++k) {
    dst[k] = outs[k] ? device_view(outs[k]) : nullptr;
    if (outs[k] && !dst[k])
      return fail(c, LBM_EINVAL, "lbm_moments_async needs device or page-locked outputs");
  }
  LBM_CUDA(c, cudaSetDevice(c->device));
  if (c->slab) {  // through the buffer layout, then the slab's own layers
    int rc = ensure_tmp(c);
    if (rc) return rc;
    const size_t N = (size_t)c->N;
    double* t[4] = {c->tmp, c->tmp + N, c->tmp + (1 + c->D) * N, c->tmp + (2 + c->D) * N};
    LBM_CUDA(c, c->ops->moments(c->opt.precision, c->f[c->cur], rho ? t[0] : nullptr, u ? t[1] : nullptr,
                                T ? t[2] : nullptr, q ? t[3] : nullptr, c->fo, c->p, c->stream));
    const int rows[4] = {1, c->D, 1, c->D};
    for (int k = 0; k < 4; ++k)
      if (outs[k]) LBM_CUDA(c, copy_rows(c, dst[k], t[k], rows[k], true));
    return LBM_OK;
  }
  LBM_CUDA(c, c->ops->moments(c->opt.precision, c->f[c->cur], dst[0], dst[1], dst[2], dst[3], c->fo, c->p,
                              c->stream));
  return LBM_OK;
}

int lbm_set_params(lbm_ctx* c, double tau, const lbm_gfield* g) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(c, LBM_EINVAL, "tau-hat must be > 1/2 (got %g)", tau);
  if (c->p.gkind != lbm::G_UNIFORM)
    return fail(c, LBM_EINVAL, "lbm_set_params serves contexts created with a uniform (or no) force");
  if (g && g->kind != LBM_G_UNIFORM) return fail(c, LBM_EINVAL, "lbm_set_params takes a uniform force");
  c->tau = tau;
  c->p.omega = 1.0 / tau;
  c->p.omega_f = (float)c->p.omega;
  for (int a = 0; a < 3; ++a) {
    c->p.g0[a] = (g && a < c->D) ? g->g0[a] : 0.0;
    c->p.g0_f[a] = (float)c->p.g0[a];
  }
  drop_graphs(c);
  lbm::batch_mark_dirty(c->batch);
  return LBM_OK;
}

int lbm_conserved(lbm_ctx* c, double* mass, double* mom, double* energy) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_conserved before lbm_init");
  LBM_CUDA(c, cudaSetDevice(c->device));
  // one launch: block partials, then the last block's fixed-order final
  // reduction written straight into the page-locked result when it is mapped
  double* hview = device_view(c->hres);
  LBM_CUDA(c, c->ops->conserved(c->opt.precision, c->f[c->cur], c->part, c->bad, c->ticket,
                                hview ? hview : c->dres, c->derr, c->p, c->nblk_cons, c->stream));
  if (!hview)
    LBM_CUDA(c, cudaMemcpyAsync(c->hres, c->dres, sizeof(double) * (2 * lbm::NCONS + 2),
                                cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (c->hres[2 * lbm::NCONS + 1] != 0.0) {
    LBM_CUDA(c, cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream));
    return fail(c, LBM_ETIMEOUT, "a bounded device wait ran out in an earlier step; its results are void");
  }
  const double* r = c->hres;
  if (mass) *mass = r[0] + r[1];
  if (mom)
    for (int a = 0; a < c->D; ++a) mom[a] = r[2 * (1 + a)] + r[2 * (1 + a) + 1];
  if (energy) *energy = r[8] + r[9];
  if (r[2 * lbm::NCONS] > 0.0)
    return fail(c, LBM_EUNSTABLE, "%.0f sites have a non-finite moment, rho <= 0 or T <= 0",
                r[2 * lbm::NCONS]);
  return LBM_OK;
}

int lbm_get_populations(lbm_ctx* c, double* out) {
  if (!c || !out) return fail(c, LBM_EINVAL, "ctx and out are required");
  if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_get_populations before lbm_init");
  LBM_CUDA(c, cudaSetDevice(c->device));
  const size_t n = (size_t)c->Q * c->N;
  const bool dev = is_device_ptr(out) && !c->slab;
  double* dst = out;
  if (!dev) {
    LBM_CUDA(c, cudaMallocAsync(&dst, n * sizeof(double), c->stream));
  }
  cudaError_t e = c->ops->pulled(c->opt.precision, c->f[c->cur], dst, c->p, c->stream);
  if (e == cudaSuccess && !dev)
    e = c->slab ? copy_rows(c, out, dst, c->Q, true)
                : cudaMemcpyAsync(out, dst, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (!dev) cudaFreeAsync(dst, c->stream);
  if (e != cudaSuccess) return fail(c, LBM_ECUDA, "get_populations failed: %s", cudaGetErrorString(e));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

static int state_io(lbm_ctx* c, double* io, int dir) {
  LBM_CUDA(c, cudaSetDevice(c->device));
  const size_t n = (size_t)c->Q * c->N;
  const bool dev = is_device_ptr(io) && !c->slab;
  double* d = io;
  if (!dev) {
    LBM_CUDA(c, cudaMallocAsync(&d, n * sizeof(double), c->stream));
    if (dir == 1) {
      if (c->slab) LBM_CUDA(c, copy_rows(c, d, io, c->Q, false));
      else LBM_CUDA(c, cudaMemcpyAsync(d, io, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }
  }
  cudaError_t e = c->ops->state(c->opt.precision, dir, c->f[c->cur], d, c->p, c->stream);
  if (e == cudaSuccess && !dev && dir == 0)
    e = c->slab ? copy_rows(c, io, d, c->Q, true)
                : cudaMemcpyAsync(io, d, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (!dev) cudaFreeAsync(d, c->stream);
  if (e != cudaSuccess) return fail(c, LBM_ECUDA, "state transfer failed: %s", cudaGetErrorString(e));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_get_state(lbm_ctx* c, double* out) {
  if (!c || !out) return fail(c, LBM_EINVAL, "ctx and out are required");
  if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_get_state before lbm_init");
  return state_io(c, out, 0);
}

int lbm_set_state(lbm_ctx* c, const double* in) {
  if (!c || !in) return fail(c, LBM_EINVAL, "ctx and in are required");
  if (c->opt.precision == LBM_FP16_SCALED && !c->initialised)
    return fail(c, LBM_ESTATE, "the FP16 scale is fixed by lbm_init; call it first");
  drop_graphs(c);
  int rc = state_io(c, const_cast<double*>(in), 1);
  if (rc == LBM_OK) c->initialised = true;
  lbm::batch_mark_dirty(c->batch);
  return rc;
}

long long lbm_step_count(const lbm_ctx* c) { return c ? c->steps : 0; }

int lbm_step_kernel(const lbm_ctx* c) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (c->use_wave) return LBM_KERNEL_WAVE;
  return c->use_tma ? LBM_KERNEL_TMA : (c->use_async ? LBM_KERNEL_PREFETCH : LBM_KERNEL_PLAIN);
}

double lbm_fp16_scale(const lbm_ctx* c) {
  return (c && c->opt.precision == LBM_FP16_SCALED) ? (double)c->p.h_scale : 0.0;
}

size_t lbm_device_bytes(const lbm_ctx* c) { return c ? c->bytes : 0; }

namespace {
struct CkptHeader {
  char magic[8];
  int version, lat, nx, ny, nz, precision;
  float h_scale, h_inv_scale;
  long long steps;
  double tau;
};
}  // namespace

int lbm_save(lbm_ctx* c, const char* path) {
  if (!c || !path) return fail(c, LBM_EINVAL, "ctx and path are required");
  if (!c->initialised) return fail(c, LBM_ESTATE, "nothing to save before lbm_init");
  LBM_CUDA(c, cudaSetDevice(c->device));
  const size_t nb = (size_t)c->Q * c->N * c->elem;
  void* h = std::malloc(nb);
  if (!h) return fail(c, LBM_ENOMEM, "out of host memory");
  cudaError_t e = cudaMemcpyAsync(h, c->f[c->cur], nb, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    std::free(h);
    return fail(c, LBM_ECUDA, "checkpoint copy failed: %s", cudaGetErrorString(e));
  }
  CkptHeader hd{};
  std::memcpy(hd.magic, "LBMGB300", 8);
  hd.version = 1; hd.lat = c->lat; hd.nx = c->nx; hd.ny = c->ny; hd.nz = c->nz;
  hd.precision = c->opt.precision; hd.h_scale = c->p.h_scale; hd.h_inv_scale = c->p.h_inv_scale;
  hd.steps = c->steps; hd.tau = c->tau;
  FILE* fp = std::fopen(path, "wb");
  bool ok = fp && std::fwrite(&hd, sizeof hd, 1, fp) == 1 && std::fwrite(h, 1, nb, fp) == nb;
  if (fp) ok = (std::fclose(fp) == 0) && ok;
  std::free(h);
  if (!ok) return fail(c, LBM_EIO, "cannot write checkpoint %s", path);
  return LBM_OK;
}

int lbm_load(lbm_ctx* c, const char* path) {
  if (!c || !path) return fail(c, LBM_EINVAL, "ctx and path are required");
  LBM_CUDA(c, cudaSetDevice(c->device));
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(c, LBM_EIO, "cannot open checkpoint %s", path);
  CkptHeader hd{};
  if (std::fread(&hd, sizeof hd, 1, fp) != 1 || std::memcmp(hd.magic, "LBMGB300", 8) || hd.version != 1) {
    std::fclose(fp);
    return fail(c, LBM_EIO, "%s is not a checkpoint of this library", path);
  }
  if (hd.lat != c->lat || hd.nx != c->nx || hd.ny != c->ny || hd.nz != c->nz || hd.precision != c->opt.precision) {
    std::fclose(fp);
    return fail(c, LBM_EINVAL, "checkpoint grid/lattice/precision differ from the context");
  }
  const size_t nb = (size_t)c->Q * c->N * c->elem;
  void* h = std::malloc(nb);
  if (!h) {
    std::fclose(fp);
    return fail(c, LBM_ENOMEM, "out of host memory");
  }
  const bool ok = std::fread(h, 1, nb, fp) == nb;
  std::fclose(fp);
  if (!ok) {
    std::free(h);
    return fail(c, LBM_EIO, "checkpoint %s is truncated", path);
  }
  drop_graphs(c);
  c->cur = 0;
  cudaError_t e = cudaMemcpyAsync(c->f[0], h, nb, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  std::free(h);
  if (e != cudaSuccess) return fail(c, LBM_ECUDA, "checkpoint upload failed: %s", cudaGetErrorString(e));
  c->p.h_scale = hd.h_scale;
  c->p.h_inv_scale = hd.h_inv_scale;
  fp16_factors(c);
  c->steps = hd.steps;
  c->initialised = true;
  lbm::batch_mark_dirty(c->batch);
  return LBM_OK;
}

size_t lbm_slab_halo_bytes(const lbm_ctx* c) {
  if (!c || !c->slab) return 0;
  int layer[kMaxHaloPlanes * 2], pop[kMaxHaloPlanes * 2];
  return (size_t)halo_list(c, 1, layer, pop) * layer_sites(c) * c->elem;
}

int lbm_slab_halo_pack(lbm_ctx* c, int side, void* dst) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (!c->slab) return fail(c, LBM_EINVAL, "ctx is not a slab");
  if (side != 0 && side != 1) return fail(c, LBM_EINVAL, "side must be 0 (below) or 1 (above)");
  if ((side == 0 ? c->gb : c->ga) == 0) return fail(c, LBM_EINVAL, "no neighbour on that side (a wall)");
  if (!dst || !is_device_ptr(dst)) return fail(c, LBM_EINVAL, "dst must be device memory");
  if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_slab_halo_pack before lbm_init");
  LBM_CUDA(c, cudaSetDevice(c->device));
  const HaloPlanes hp = halo_planes(c, side, c, nullptr);
  LBM_CUDA(c, launch_halo(c->f[c->cur], dst, hp, layer_sites(c), c->elem, c->stream));
  return LBM_OK;
}

int lbm_slab_halo_unpack(lbm_ctx* c, int side, const void* src) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (!c->slab) return fail(c, LBM_EINVAL, "ctx is not a slab");
  if (side != 0 && side != 1) return fail(c, LBM_EINVAL, "side must be 0 (below) or 1 (above)");
  if ((side == 0 ? c->gb : c->ga) == 0) return fail(c, LBM_EINVAL, "no neighbour on that side (a wall)");
  if (!src || !is_device_ptr(src)) return fail(c, LBM_EINVAL, "src must be device memory");
  if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_slab_halo_unpack before lbm_init");
  LBM_CUDA(c, cudaSetDevice(c->device));
  // the message from below is the lower neighbour's upward message (dir 1)
  const HaloPlanes hp = halo_planes(c, side == 0 ? 1 : 0, nullptr, c);
  LBM_CUDA(c, launch_halo(src, c->f[c->cur], hp, layer_sites(c), c->elem, c->stream));
  return LBM_OK;
}

int lbm_slab_exchange(lbm_ctx* lo, lbm_ctx* hi) {
  if (!lo || !hi) return fail(nullptr, LBM_EINVAL, "both slabs are required");
  if (!lo->slab || !hi->slab) return fail(lo, LBM_EINVAL, "both contexts must be slabs");
  if (lo->lat != hi->lat || lo->opt.precision != hi->opt.precision || lo->nx != hi->nx ||
      (lo->D == 3 && lo->ny != hi->ny) || lo->n_axis != hi->n_axis)
    return fail(lo, LBM_EINVAL, "slabs of different grids");
  const bool adjacent = lo->a_end == hi->a_begin || (lo->a_end == lo->n_axis && hi->a_begin == 0);
  if (!adjacent || lo->ga == 0 || hi->gb == 0)
    return fail(lo, LBM_EINVAL, "hi must follow lo along the last axis (periodic wrap included)");
  if (!lo->initialised || !hi->initialised) return fail(lo, LBM_ESTATE, "lbm_slab_exchange before lbm_init");
  if (lo->device != hi->device) return fail(lo, LBM_EINVAL, "slabs on different devices: use pack / unpack");
  if (lo->opt.precision == LBM_FP16_SCALED && lo->p.h_scale != hi->p.h_scale)
    return fail(lo, LBM_EINVAL, "FP16 slabs need one scale (lbm_set_fp16_scale)");
  LBM_CUDA(lo, cudaSetDevice(lo->device));
  const size_t S = layer_sites(lo);
  HaloPlanes up = halo_planes(lo, 1, lo, hi), down = halo_planes(lo, 0, hi, lo);
  LBM_CUDA(lo, launch_halo(lo->f[lo->cur], hi->f[hi->cur], up, S, lo->elem, lo->stream));
  LBM_CUDA(lo, launch_halo(hi->f[hi->cur], lo->f[lo->cur], down, S, lo->elem, lo->stream));
  return LBM_OK;
}

int lbm_slab_info(const lbm_ctx* c, int* a_begin, int* a_end, int* ghosts_below, int* ghosts_above) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (a_begin) *a_begin = c->slab ? c->a_begin : 0;
  if (a_end) *a_end = c->slab ? c->a_end : (c->D == 2 ? c->ny : c->nz);
  if (ghosts_below) *ghosts_below = c->gb;
  if (ghosts_above) *ghosts_above = c->ga;
  return LBM_OK;
}

int lbm_set_fp16_scale(lbm_ctx* c, double scale) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (c->opt.precision != LBM_FP16_SCALED) return fail(c, LBM_EINVAL, "ctx does not store FP16");
  int ex = 0;
  if (!(scale > 0.0) || !std::isfinite(scale) || std::frexp(scale, &ex) != 0.5 || ex < -60 || ex > 62)
    return fail(c, LBM_EINVAL, "scale must be a power of two in [2^-60, 2^60]");
  if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_set_fp16_scale before lbm_init");
  LBM_CUDA(c, cudaSetDevice(c->device));
  const float factor = (float)(scale / (double)c->p.h_scale);
  if (factor != 1.0f) {
    const size_t n = (size_t)c->Q * c->N;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
    k_rescale_half<<<blocks, 256, 0, c->stream>>>((unsigned short*)c->f[c->cur], n, factor);
    LBM_CUDA(c, cudaGetLastError());
    drop_graphs(c);
  }
  c->p.h_scale = (float)scale;
  c->p.h_inv_scale = (float)(1.0 / scale);
  fp16_factors(c);
  lbm::batch_mark_dirty(c->batch);
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.empty() ? "no error" : c->err.c_str();
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  if (c->batch) lbm::batch_detach(c->batch, c);
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  cudaFree(c->f[0]);
  cudaFree(c->f[1]);
  cudaFree(c->gtab);
  cudaFree(c->gtab_f);
  cudaFree(c->solid);
  cudaFree(c->wall_th);
  cudaFree(c->wall_th_f);
  cudaFree(c->part);
  cudaFree(c->bad);
  cudaFree(c->dres);
  cudaFree(c->dmax);
  cudaFree(c->tmp);
  cudaFree(c->derr);
  cudaFree(c->ticket);
  cudaFree(c->wave_sync);
  if (c->hres) cudaFreeHost(c->hres);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
}

}  // extern "C"

namespace lbm {
// Context-free calls report their message through lbm_last_error(NULL).
void set_global_error(const char* msg) { g_create_error = msg; }

int ctx_fail(lbm_ctx* c, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  int rc = vfail(c, code, fmt, ap);
  va_end(ap);
  return rc;
}
}  // namespace lbm

