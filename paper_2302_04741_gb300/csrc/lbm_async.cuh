// lbm_async.cuh -- persistent step kernel that prefetches the next tile.
//
// Blocks stride over the grid's row tiles (blockDim.x sites of one row).
// While a thread collides its site of tile k, the 37 (39) populations its
// site of tile k+1 pulls are already being copied, with cp.async, into the
// thread's own column of a two-stage shared-memory buffer, so the loads of
// the next tile overlap the arithmetic of the current one.  A thread reads
// only the shared-memory slots it filled itself, so the only synchronisation
// is cp.async.wait_group on the thread's own copies.  Tiles next to a wall,
// and warps whose pulls wrap around x, use the plain pull (direct loads).
// The collision is the device code of k_step: results are bit-identical.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 4-byte async copies of the populations the plain fast path would load.
template <class L, int P>
__device__ __forceinline__ void prefetch_interior(const typename Codec<P>::T* __restrict__ fsite,
                                                  const StepParams& p, int y, int z,
                                                  uint32_t col, int stride_bytes) {
  constexpr int D = L::D, Q = L::Q;
  static_assert(sizeof(typename Codec<P>::T) == 4, "4-byte elements only");
  const long long N = p.N;
  long long dy[7], dz[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    dy[k] = (long long)(wrap3(y - (k - 3), p.ny) - y) * p.nx;
    dz[k] = D == 3 ? (long long)(wrap3(z - (k - 3), p.nz) - z) * p.nx * p.ny : 0;
  }
  static_for<0, Q>([&](auto I) {
    constexpr int i = I;
    constexpr int ex = L::E(i, 0), ey = L::E(i, 1), ez = L::E(i, 2);
    const long long off = i * N + dz[ez + 3] + dy[ey + 3] - ex;
    cp_async4(col + i * stride_bytes, fsite + off);
  });
}

template <class L, int P, int FO>
__global__ void __launch_bounds__(256, min_blocks<L, P>())
    k_step_async(const typename Codec<P>::T* __restrict__ fin, typename Codec<P>::T* __restrict__ fout,
                 const StepParams p) {
  using C = Codec<P>;
  using T = typename C::T;
  using R = typename C::R;
  constexpr int Q = L::Q, D = L::D;
  extern __shared__ __align__(16) unsigned char sbuf[];  // [2][Q][blockDim.x] of T
  const int bx = blockDim.x, tid = threadIdx.x;
  const int ntx = (p.nx + bx - 1) / bx;
  const int ntiles = ntx * p.ny * p.nz;
  const int nA = D == 2 ? p.ny : p.nz;
  const int stride = bx * (int)sizeof(T);               // bytes between directions
  const uint32_t col0 = (uint32_t)__cvta_generic_to_shared(sbuf) + tid * (int)sizeof(T);
  const uint32_t stage_bytes = (uint32_t)Q * stride;

  // tile geometry and whether its pulls can be prefetched (block-uniform
  // except for the per-warp x-wrap test)
  auto tile_of = [&](int t, int& x, int& y, int& z, bool& fast) {
    const int xt = t % ntx, row = t / ntx;
    y = row % p.ny;
    z = row / p.ny;
    x = xt * bx + tid;
    const int a = D == 2 ? y : z;
    const bool near = p.wall != W_NONE && (a < 3 || a >= nA - 3);
    const int wx0 = xt * bx + (tid & ~31);
    fast = !near && wx0 >= 3 && wx0 + 31 <= p.nx - 4;
  };

  int t = blockIdx.x;
  if (t >= ntiles) return;
  int x, y, z;
  bool fast;
  tile_of(t, x, y, z, fast);
  if (fast) prefetch_interior<L, P>(fin + ((z * p.ny + y) * p.nx + x), p, y, z, col0, stride);
  cp_async_commit();
  for (int k = 0; t < ntiles; t += gridDim.x, ++k) {
    // issue the next tile's copies before working on this one
    const int tn = t + gridDim.x;
    int xn = 0, yn = 0, zn = 0;
    bool fastn = false;
    if (tn < ntiles) {
      tile_of(tn, xn, yn, zn, fastn);
      if (fastn)
        prefetch_interior<L, P>(fin + ((zn * p.ny + yn) * p.nx + xn), p, yn, zn,
                                col0 + ((k + 1) & 1) * stage_bytes, stride);
    }
    cp_async_commit();
    cp_async_wait<1>();  // this thread's copies of tile t have landed
    if (x < p.nx) {
      const int site = (z * p.ny + y) * p.nx + x;
      R d[Q];
      if (fast) {
        const T* sc = reinterpret_cast<const T*>(sbuf + (k & 1) * stage_bytes) + tid;
        static_for<0, Q>([&](auto I) {
          constexpr int i = I;
          d[i] = R(C::template decode<L, i>(sc[i * bx], p));
        });
      } else {
        pull<L, P, R>(fin, p, x, y, z, d);
      }
      R g[3];
      site_force_r<D, R>(p, x, y, z, site, g);
      collide_store<L, P, FO>(d, g, site, fout, p);
    }
    x = xn;
    y = yn;
    z = zn;
    fast = fastn;
  }
  cp_async_wait<0>();
}

}  // namespace lbm
