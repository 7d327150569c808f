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

// Equilibrium deviation f0_i(1, 0, T) - w_i = w_i A0(|xi_i|^2) of a wall at
// rest (u = 0), the rest-frame value of the Hermite-expanded equilibrium.
template <class L>
void wall_equilibrium(double T, double* fwd, double* fw) {
  const double th = T - 1.0;
  const int D = L::D;
  for (int i = 0; i < L::Q; ++i) {
    const double e2 = L::e[i][0] * L::e[i][0] + L::e[i][1] * L::e[i][1] + L::e[i][2] * L::e[i][2];
    const double X2 = L::c2 * e2;
    double a0 = 0.5 * th * (X2 - D);
    if (L::NEQ >= 4) a0 += (3.0 * th * th * (X2 * X2 - 2.0 * (D + 2) * X2 + D * (D + 2))) / 24.0;
    fwd[i] = L::w[i] * a0;
    fw[i] = L::w[i] + fwd[i];
  }
}

// The FP16 codec factors of the context's lattice for its current scale.
void fp16_factors(lbm_ctx* c) {
  if (c->lat == LBM_D2Q37) lbm::set_fp16_factors<lbm::D2Q37>(c->p);
  else lbm::set_fp16_factors<lbm::D3Q39>(c->p);
}

template <class L>
void wall_tables(StepParams& p, double T_lo, double T_hi) {
  const int A = L::D - 1;
  for (int side = 0; side < 2; ++side) {
    wall_equilibrium<L>(side == 0 ? T_lo : T_hi, p.fwd[side], p.fw[side]);
    double sfwd = 0.0, sfw = 0.0;
    for (int i = 0; i < L::Q; ++i) {
      const int eA = L::e[i][A];
      const int cnt = side == 0 ? (eA > 0 ? eA : 0) : (eA < 0 ? -eA : 0);  // slots per column
      sfwd += cnt * p.fwd[side][i];
      sfw += cnt * p.fw[side][i];
    }
    p.wallA[side] = -sfwd;
    p.wall_inv_den[side] = 1.0 / sfw;
  }
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
    e = c->ops->step(c->opt.precision, c->fo, c->f[c->cur], c->f[c->cur ^ 1], c->p,
                     c->opt.block_x, c->overlap, c->stream);
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

int lbm_create(lbm_lattice lat, int nx, int ny, int nz, double tau, const lbm_gfield* g,
               const lbm_options* opt, lbm_ctx** out) {
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
  if (o.tma_stages != 0 && (o.tma_stages < 2 || o.tma_stages > 8))
    return fail(nullptr, LBM_EINVAL, "tma_stages must be 0 or 2..8 (got %d)", o.tma_stages);
  lbm_gfield gf{};
  gf.kind = LBM_G_UNIFORM;
  if (g) gf = *g;
  if (gf.kind < LBM_G_UNIFORM || gf.kind > LBM_G_FIELD) return fail(nullptr, LBM_EINVAL, "bad force kind %d", gf.kind);
  if (gf.kind == LBM_G_SINE && (gf.wave_axis < 0 || gf.wave_axis >= D))
    return fail(nullptr, LBM_EINVAL, "bad wave_axis %d", gf.wave_axis);
  if (gf.kind == LBM_G_FIELD && !gf.field) return fail(nullptr, LBM_EINVAL, "force field is NULL");

  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return fail(nullptr, LBM_ENOMEM, "out of host memory");
  c->lat = lat; c->D = D; c->Q = ops->Q; c->nx = nx; c->ny = ny; c->nz = nz; c->N = (int)N;
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
  const size_t fbytes = (size_t)c->Q * N * c->elem;
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
  p.nx = nx; p.ny = ny; p.nz = nz; p.N = (int)N; p.wall = wall;
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
  if (wall != lbm::W_NONE) {
    if (lat == LBM_D2Q37) wall_tables<lbm::D2Q37>(p, o.T_lo[D - 1], o.T_hi[D - 1]);
    else wall_tables<lbm::D3Q39>(p, o.T_lo[D - 1], o.T_hi[D - 1]);
  }
  if (gf.kind == LBM_G_SINE) {
    const int na = n[gf.wave_axis];
    double* h = (double*)std::malloc(sizeof(double) * na);
    if (!h) { fail(c, LBM_ENOMEM, "out of host memory"); return bail(LBM_ENOMEM); }
    for (int k = 0; k < na; ++k) h[k] = std::sin(2.0 * M_PI * k / na);
    cudaError_t e = cudaMalloc(&c->gtab, sizeof(double) * na);
    if (e == cudaSuccess) e = cudaMemcpy(c->gtab, h, sizeof(double) * na, cudaMemcpyHostToDevice);
    std::free(h);
    if (e != cudaSuccess) { cudaGetLastError(); fail(c, LBM_ECUDA, "force table upload failed"); return bail(LBM_ECUDA); }
    c->bytes += sizeof(double) * na;
  } else if (gf.kind == LBM_G_FIELD) {
    const size_t gb = sizeof(double) * D * N;
    cudaError_t e = cudaMalloc(&c->gtab, gb);
    if (e == cudaSuccess) e = cudaMemcpy(c->gtab, gf.field, gb, cudaMemcpyDefault);
    if (e != cudaSuccess) { cudaGetLastError(); fail(c, LBM_ECUDA, "force field upload failed"); return bail(LBM_ECUDA); }
    c->bytes += gb;
  }
  p.gtab = c->gtab;
  if (c->gtab) {  // float copy of the force table for the float kernels
    const size_t cnt = gf.kind == LBM_G_SINE ? (size_t)n[gf.wave_axis] : (size_t)D * N;
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
    const long long tiles = (long long)((nx + 127) / 128) * ny * nz;
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

int lbm_init(lbm_ctx* c, const double* rho, const double* u, const double* T) {
  if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
  if (!rho || !u || !T) return fail(c, LBM_EINVAL, "rho, u and T are required");
  LBM_CUDA(c, cudaSetDevice(c->device));
  const size_t N = (size_t)c->N;
  const double *drho = device_view(rho), *du = device_view(u), *dT = device_view(T);
  const bool dev = drho && du && dT;
  if (!dev) {
    int rc = ensure_tmp(c);
    if (rc) return rc;
    double* t = c->tmp;
    LBM_CUDA(c, cudaMemcpyAsync(t, rho, N * sizeof(double), cudaMemcpyDefault, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync(t + N, u, c->D * N * sizeof(double), cudaMemcpyDefault, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync(t + (1 + c->D) * N, T, N * sizeof(double), cudaMemcpyDefault, c->stream));
    drho = t; du = t + N; dT = t + (1 + c->D) * N;
  }
  c->cur = 0;
  if (c->opt.precision == LBM_FP16_SCALED) {
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
    dst[k] = outs[k] ? device_view(outs[k]) : nullptr;
    staged[k] = outs[k] && !dst[k];
    if (staged[k]) dst[k] = t;
    t += cnt[k];
  }
  LBM_CUDA(c, c->ops->moments(c->opt.precision, c->f[c->cur], dst[0], dst[1], dst[2], dst[3],
                              c->fo, c->p, c->stream));
  for (int k = 0; k < 4; ++k)
    if (staged[k])
      LBM_CUDA(c, cudaMemcpyAsync(outs[k], dst[k], cnt[k] * sizeof(double), cudaMemcpyDefault, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
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
  const bool dev = is_device_ptr(out);
  double* dst = out;
  if (!dev) {
    LBM_CUDA(c, cudaMallocAsync(&dst, n * sizeof(double), c->stream));
  }
  cudaError_t e = c->ops->pulled(c->opt.precision, c->f[c->cur], dst, c->p, c->stream);
  if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(out, dst, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (!dev) cudaFreeAsync(dst, c->stream);
  if (e != cudaSuccess) return fail(c, LBM_ECUDA, "get_populations failed: %s", cudaGetErrorString(e));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

static int state_io(lbm_ctx* c, double* io, int dir) {
  LBM_CUDA(c, cudaSetDevice(c->device));
  const size_t n = (size_t)c->Q * c->N;
  const bool dev = is_device_ptr(io);
  double* d = io;
  if (!dev) {
    LBM_CUDA(c, cudaMallocAsync(&d, n * sizeof(double), c->stream));
    if (dir == 1) LBM_CUDA(c, cudaMemcpyAsync(d, io, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  }
  cudaError_t e = c->ops->state(c->opt.precision, dir, c->f[c->cur], d, c->p, c->stream);
  if (e == cudaSuccess && !dev && dir == 0)
    e = cudaMemcpyAsync(io, d, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
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

