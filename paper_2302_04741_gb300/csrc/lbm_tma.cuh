// lbm_tma.cuh -- TMA-staged persistent variant of the step kernel.
//
// Each CTA has 4 consumer warps (one row tile of 128 sites, one site per
// thread) and one producer warp.  The producer streams, for every tile, the
// Q shifted row segments the pull needs into a ring of shared-memory stages
// with cp.async.bulk.tensor (one 2-D box of (128 + 2H) x 1 per direction:
// plane i, row y - e_iy, columns [x0 - H, x0 + 128 + H)), signalling a "full"
// mbarrier with the transaction bytes; consumers read f*_i(x - e_i) from
// shared memory at a compile-time offset, release the stage on an "empty"
// mbarrier and collide exactly as the plain kernel does (same device code),
// so both kernels give bit-identical results.
//
// H is 16 bytes of elements (>= 3 columns) so every box starts on a 16-byte
// boundary; boxes that start before x = 0 or end after x = nx are zero-filled
// by the TMA unit, and the few threads whose pull wraps around x read those
// values from global memory instead.  Rows beyond a wall are not loaded: the
// wall rule supplies those slots from global memory as in the plain kernel.
//
// Every wait is bounded: after TMA_WAIT_LIMIT polls a thread sets *p.err and
// stops; the producer always waits (bounded) for its last loads before it
// exits so that no copy writes shared memory of a finished CTA.
#pragma once

#include <cuda.h>

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int TMA_W = 128;                  // sites per row tile = consumer threads
constexpr int TMA_CWARPS = TMA_W / 32;      // consumer warps
constexpr int TMA_THREADS = TMA_W + 32;     // + one producer warp
constexpr long long TMA_WAIT_LIMIT = 1LL << 25;

template <int P>
struct TmaGeom {
  using T = typename Codec<P>::T;
  static constexpr int ES = (int)sizeof(T);
  static constexpr int H = (16 / ES) < 4 ? 4 : (16 / ES);  // halo: >= 3 columns, 16-B aligned
  static constexpr int RW = TMA_W + 2 * H;                 // elements per box
  static constexpr int BOX_BYTES = RW * ES;
  static constexpr int ROW_BYTES = (BOX_BYTES + 127) / 128 * 128;  // 128-B aligned smem rows
  static constexpr int ROW_ELEMS = ROW_BYTES / ES;
};

template <class L, int P>
__host__ __device__ constexpr int tma_stage_bytes() {
  return L::Q * TmaGeom<P>::ROW_BYTES;
}

// ------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false (and *err set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  for (long long it = 0; it < TMA_WAIT_LIMIT; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) atomicExch(err, 1);
  return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// ----------------------------------------------------- staged pull of one site
// stage: the tile's shared-memory stage; x0: first site of the tile.
template <class L, int P, class R, bool SC>
__device__ __forceinline__ void pull_staged(const unsigned char* stage,
                                            const typename Codec<P>::T* __restrict__ fin,
                                            const StepParams& p, int x0, int x, int y, int z,
                                            bool warp_edge, R (&d)[L::Q]) {
  using C = Codec<P>;
  using T = typename C::T;
  using G = TmaGeom<P>;
  constexpr int D = L::D, Q = L::Q;
  const T* sb = reinterpret_cast<const T*>(stage) + (x - x0) + G::H;
  const int a = D == 2 ? y : z;
  const int nA = D == 2 ? p.ny : p.nz;
  const bool near = p.wall != W_NONE && (a < 3 || a >= nA - 3);
  if (!near && !warp_edge) {
    static_for<0, Q>([&](auto I) {
      constexpr int i = I;
      constexpr int ex = L::E(i, 0);
      d[i] = R(step_in<L, P, i, SC>(sb[i * G::ROW_ELEMS - ex], p));
    });
    return;
  }
  // general path: x wrap-around columns and wall slots from global memory
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const size_t N = (size_t)p.N;
  const int side = a < 3 ? 0 : 1;
  const int colbase = D == 2 ? x : (y * nx + x);
  const int lineA = D == 2 ? nx : nx * ny;
  R rm1 = R(0);
  if (near && p.wall == W_THERMAL) {
    R sum = R(0);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int row = side == 0 ? r : nA - 1 - r;
      static_for<0, Q>([&](auto J) {
        constexpr int j = J;
        constexpr int eA = L::E(j, D - 1);
        if constexpr (eA != 0) {
          const bool leaves = side == 0 ? (eA < 0 && r + eA < 0) : (eA > 0 && r - eA < 0);
          if (leaves)
            sum += R(C::template decode<L, j>(C::load(fin + j * N + colbase + row * lineA, p), p));
        }
      });
    }
    rm1 = (R(p.wallA[side]) + sum) * R(p.wall_inv_den[side]);
  }
  static_for<0, Q>([&](auto I) {
    constexpr int i = I;
    constexpr int ex = L::E(i, 0), ey = L::E(i, 1), ez = L::E(i, 2);
    constexpr int eA = L::E(i, D - 1);
    const int sA = a - eA;
    if (!near || (sA >= 0 && sA < nA)) {
      const int xs = x - ex;
      if (xs >= 0 && xs < nx) {
        d[i] = R(step_in<L, P, i, SC>(sb[i * G::ROW_ELEMS - ex], p));
      } else {
        const int sx = wrap3(xs, nx);
        const int sy = wrap3(y - ey, ny);
        const int sz = D == 3 ? wrap3(z - ez, nz) : 0;
        d[i] = R(step_in<L, P, i, SC>(C::load(fin + i * N + (sz * ny + sy) * nx + sx, p), p));
      }
    } else if (p.wall == W_BOUNCE) {
      constexpr int io = opposite<i>();
      const int mA = side == 0 ? eA - 1 - a : 2 * nA - 1 - sA;
      d[i] = R(step_in<L, P, io, SC>(C::load(fin + io * N + colbase + mA * lineA, p), p));
    } else {
      d[i] = step_from_dev<i, SC>(fma(rm1, R(p.fw[side][i]), R(p.fwd[side][i])), p);
    }
  });
}

// ------------------------------------------------------------- the kernel
template <class L, int P, int FO>
__global__ void __launch_bounds__(TMA_THREADS, 3) k_step_tma(const __grid_constant__ CUtensorMap tin,
                                                          const typename Codec<P>::T* __restrict__ fin,
                                                          typename Codec<P>::T* __restrict__ fout,
                                                          const StepParams p, int stages) {
  using C = Codec<P>;
  using R = typename C::R;
  using G = TmaGeom<P>;
  constexpr int Q = L::Q, D = L::D;
  constexpr int SB = tma_stage_bytes<L, P>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // stage rows must start on 128-byte boundaries: align the base explicitly
  // (the allocation carries 128 spare bytes for this)
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int S = stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * SB);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntx = (p.nx + TMA_W - 1) / TMA_W;
  const int ntiles = ntx * p.ny * p.nz;
  const int nA = D == 2 ? p.ny : p.nz;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, TMA_CWARPS);
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == TMA_CWARPS) {
    // ------------------------------------------------ producer (one lane)
    if (lane != 0) return;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int s = k % S;
      if (k >= S && !mbar_wait(empty0 + 8 * s, ((k / S) - 1) & 1, p.err)) break;
      const int xt = t % ntx, row = t / ntx;
      const int y = row % p.ny, z = row / p.ny;
      const int a = D == 2 ? y : z;
      const int xb = xt * TMA_W - G::H;
      uint32_t bytes = 0;
      static_for<0, Q>([&](auto I) {
        constexpr int eA = L::E(I, D - 1);
        const int sA = a - eA;
        if (p.wall == W_NONE || (sA >= 0 && sA < nA)) bytes += G::BOX_BYTES;
      });
      const uint32_t bar = full0 + 8 * s;
      mbar_arrive_expect_tx(bar, bytes);
      const uint32_t dst = smem_u32(smem + (size_t)s * SB);
      static_for<0, Q>([&](auto I) {
        constexpr int i = I;
        constexpr int ey = L::E(i, 1), ez = L::E(i, 2), eA = L::E(i, D - 1);
        const int sA = a - eA;
        if (p.wall == W_NONE || (sA >= 0 && sA < nA)) {
          const int ys = wrap3(y - ey, p.ny);
          if constexpr (D == 2) {
            tma_load_3d(dst + i * G::ROW_BYTES, &tin, xb, ys, i, bar);
          } else {
            const int zs = wrap3(z - ez, p.nz);
            tma_load_4d(dst + i * G::ROW_BYTES, &tin, xb, ys, zs, i, bar);
          }
        }
      });
    }
    // drain: the last load issued into each stage must land before exit
    const int issued = k;
    for (int s = 0; s < S && s < issued; ++s) {
      const int last = s + ((issued - 1 - s) / S) * S;  // last k with k % S == s
      mbar_wait(full0 + 8 * s, (last / S) & 1, p.err);
    }
    return;
  }

  // -------------------------------------------------- consumers
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const int s = k % S;
    const bool ok = mbar_wait(full0 + 8 * s, (k / S) & 1, p.err);
    if (!__all_sync(0xffffffffu, ok)) break;  // leave the loop as a whole warp
    const int xt = t % ntx, row = t / ntx;
    const int y = row % p.ny, z = row / p.ny;
    const int x0 = xt * TMA_W;
    const int x = x0 + tid;
    const int wx0 = x0 + 32 * warp;
    const bool warp_edge = wx0 < 3 || wx0 + 31 >= p.nx - 3;
    const bool active = x < p.nx;
    R d[Q];
    constexpr bool SC = scaled_step<P, FO>();
    if (active) pull_staged<L, P, R, SC>(smem + (size_t)s * SB, fin, p, x0, x, y, z, warp_edge, d);
    __syncwarp();
    if (lane == 0) mbar_arrive(empty0 + 8 * s);
    if (active) {
      const int site = (z * p.ny + y) * p.nx + x;
      R g[3];
      site_force_r<D, R>(p, x, y, z, site, g);
      collide_store<L, P, FO, SC>(d, g, site, fout, p);
    }
  }
}

}  // namespace lbm
