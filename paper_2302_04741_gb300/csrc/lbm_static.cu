// lbm_static.cu -- lbm_conserved_static: the conservation sums of a caller's
// population buffer without any device allocation.
//
// Who needs it: code that may not allocate device memory at all -- a plugin
// inside a host application that owns every device byte through its own
// pool, a runtime whose memory budget is fully reserved up front, or a
// latency-sensitive loop that cannot afford cudaMalloc / cudaFree, which
// synchronise the whole device and stall every other stream.  Such a caller
// cannot create an lbm_ctx (lbm_create allocates), so this entry point takes
// the raw state and writes the sums to memory the caller already owns.
//
// Its per-block partial sums live in the file-scope static device arrays
// below, a fixed 3.0 MB on every GPU that loads the library, held until the
// process exits.  Host code cannot use the array names as addresses (they
// name host-side shadows), so the address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_launch.cuh"

namespace {

constexpr int kMaxTiles = LBM_STATIC_MAX_TILES;  // row tiles of 128 sites along x
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double s_part[kMaxTiles * lbm::CONS_SLOT];
static __device__ __align__(256) unsigned s_bad[kMaxTiles];
static __device__ __align__(256) double s_res[2 * lbm::NCONS + 1];

struct StaticScratch {
  double* part = nullptr;
  unsigned* bad = nullptr;
  double* res = nullptr;
  bool ready = false;
};

std::mutex s_mutex;
StaticScratch s_scratch[kMaxDevices];

// The message is readable through lbm_last_error(NULL).
int set_error(int code, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[512];
  if (e != cudaSuccess)
    std::snprintf(buf, sizeof buf, "lbm_conserved_static: %s: %s", msg, cudaGetErrorString(e));
  else
    std::snprintf(buf, sizeof buf, "lbm_conserved_static: %s", msg);
  lbm::set_global_error(buf);
  return code;
}

// Device addresses of the static arrays for the current device (first call
// on a device looks them up).
int scratch_for_current_device(StaticScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(LBM_ECUDA, "cudaGetDevice failed", e);
  if (dev < 0 || dev >= kMaxDevices) return set_error(LBM_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(s_mutex);
  StaticScratch& s = s_scratch[dev];
  if (!s.ready) {
    e = cudaGetSymbolAddress((void**)&s.part, s_part);
    if (e != cudaSuccess) return set_error(LBM_ECUDA, "cudaGetSymbolAddress(partials) failed", e);
    e = cudaGetSymbolAddress((void**)&s.bad, s_bad);
    if (e != cudaSuccess) return set_error(LBM_ECUDA, "cudaGetSymbolAddress(counts) failed", e);
    e = cudaGetSymbolAddress((void**)&s.res, s_res);
    if (e != cudaSuccess) return set_error(LBM_ECUDA, "cudaGetSymbolAddress(result) failed", e);
    s.ready = true;
  }
  *out = &s;
  return LBM_OK;
}

// out[0] mass, out[1..3] momentum, out[4] energy, out[5] number of bad sites.
__global__ void k_static_combine(const double* __restrict__ res, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < lbm::NCONS; ++k) out[k] = res[2 * k] + res[2 * k + 1];
    out[lbm::NCONS] = res[2 * lbm::NCONS];
  }
}

// True when ptr is device (or managed) memory that kernels on device `dev`
// can read: a host address, pageable or page-locked, or memory of another GPU
// is refused before any launch.
bool on_device(const void* ptr, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int lbm_conserved_static(lbm_lattice lat, int nx, int ny, int nz,
                                    const lbm_options* opt, const lbm_gfield* g,
                                    double fp16_scale, const void* f, double* out) {
  const lbm::LatticeOps* ops = lat == LBM_D2Q37 ? &lbm::ops_d2q37()
                                                : (lat == LBM_D3Q39 ? &lbm::ops_d3q39() : nullptr);
  if (!ops) return set_error(LBM_EINVAL, "unknown lattice");
  if (!f || !out) return set_error(LBM_EINVAL, "f and out are required");
  lbm_options o;
  if (opt) o = *opt;
  else lbm_default_options(&o);
  const int D = ops->D;
  if (D == 2 && nz != 1) return set_error(LBM_EINVAL, "D2Q37 needs nz == 1");
  if (nx < 3 || ny < 3 || nz < 1) return set_error(LBM_EINVAL, "grid too small");
  if (D == 3 && nz < 3) return set_error(LBM_EINVAL, "grid too small");
  const long long tiles = (long long)((nx + 127) / 128) * ny * nz;
  if (tiles > kMaxTiles) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "grid needs %lld row tiles of 128 sites; the static scratch holds at most %d "
                  "(use lbm_conserved on a context for larger grids)", tiles, kMaxTiles);
    return set_error(LBM_EINVAL, msg);
  }
  if (o.precision < LBM_FP64 || o.precision > LBM_FP16_SCALED) return set_error(LBM_EINVAL, "unknown precision");
  lbm::StepParams p;
  std::memset(&p, 0, sizeof p);
  p.nx = nx; p.ny = ny; p.nz = nz; p.N = nx * ny * nz;
  p.a0 = 0;
  p.na = D == 2 ? ny : nz;
  p.omega = 1.0;
  p.wall = lbm::W_NONE;
  for (int a = 0; a < D; ++a) {
    if (o.bc[a] == LBM_PERIODIC) continue;
    if (a != D - 1 || o.bc[a] < 0 || o.bc[a] > LBM_THERMAL_WALL)
      return set_error(LBM_EINVAL, "walls are supported on the last axis only");
    if ((a == 1 ? ny : nz) < 6) return set_error(LBM_EINVAL, "a walled axis needs >= 6 sites");
    p.wall = o.bc[a] == LBM_BOUNCE_BACK ? lbm::W_BOUNCE : lbm::W_THERMAL;
  }
  if (p.wall != lbm::W_NONE) {
    if (lat == LBM_D2Q37) lbm::wall_tables<lbm::D2Q37>(p, o.T_lo[D - 1], o.T_hi[D - 1]);
    else lbm::wall_tables<lbm::D3Q39>(p, o.T_lo[D - 1], o.T_hi[D - 1]);
  }
  p.gkind = lbm::G_UNIFORM;
  if (g) {
    if (g->kind == LBM_G_UNIFORM) {
      for (int a = 0; a < D; ++a) p.g0[a] = g->g0[a];
    } else if (g->kind == LBM_G_FIELD) {
      if (!g->field) return set_error(LBM_EINVAL, "force field is NULL");
      p.gkind = lbm::G_FIELD;
      // device pointer, D*N doubles; p.gtab_f stays NULL: the conservation
      // pass of the float codecs then reads this double field and rounds it
      // to float, as a context's float copy of the field is rounded
      p.gtab = g->field;
    } else {
      return set_error(LBM_EINVAL, "force kind must be UNIFORM or FIELD (a device array)");
    }
  }
  p.omega_f = 1.0f;
  for (int a = 0; a < 3; ++a) p.g0_f[a] = (float)p.g0[a];
  if (o.precision == LBM_FP16_SCALED) {
    if (!(fp16_scale > 0.0)) return set_error(LBM_EINVAL, "fp16_scale must be > 0");
    p.h_scale = (float)fp16_scale;
    p.h_inv_scale = (float)(1.0 / fp16_scale);
  } else {
    p.h_scale = p.h_inv_scale = 1.0f;
  }
  if (lat == LBM_D2Q37) lbm::set_fp16_factors<lbm::D2Q37>(p);
  else lbm::set_fp16_factors<lbm::D3Q39>(p);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(LBM_EINVAL, "f and out must be device memory of the current device "
                                 "(no CUDA device is usable)", e);
  }
  if (!on_device(f, dev)) return set_error(LBM_EINVAL, "f must be device memory of the current device");
  if (!on_device(out, dev))
    return set_error(LBM_EINVAL, "out must be device memory of the current device");
  if (p.gkind == lbm::G_FIELD && !on_device(p.gtab, dev))
    return set_error(LBM_EINVAL, "the force field must be device memory of the current device");
  StaticScratch* s = nullptr;
  int rc = scratch_for_current_device(&s);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)o.stream;
  // the grid-stride pass writes one partial per block: at most one per tile;
  // the same block count as a context's pass (lbm_create)
  int nsm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(LBM_ECUDA, "cudaDeviceGetAttribute failed", e);
  if (nsm < 1) nsm = 1;
  const long long cap = (long long)LBM_CONSERVED_BLOCKS * nsm;
  const int nblocks = (int)(tiles < cap ? tiles : cap);
  e = ops->conserved(o.precision, f, s->part, s->bad, nullptr, nullptr, nullptr, p,
                                 nblocks, st);
  if (e != cudaSuccess) return set_error(LBM_ECUDA, "conservation kernel launch failed", e);
  e = ops->conserved_final(o.precision, s->part, s->bad, nblocks, s->res, p, st);
  if (e != cudaSuccess) return set_error(LBM_ECUDA, "final reduction launch failed", e);
  k_static_combine<<<1, 32, 0, st>>>(s->res, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(LBM_ECUDA, "combine launch failed", e);
  return LBM_OK;
}

