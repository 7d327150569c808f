// lbm_batch.cuh -- one launch per step for a ragged set of grids.
//
// Every member grid keeps its own buffers and parameters; a device table
// holds, per grid, its StepParams, both buffer pointers and the parity of the
// buffer that holds its state before launch 0 of a sequence.  Launch k of a
// sequence reads buffer (cur + k) & 1 and writes the other one.  A tile is a
// run of blockDim.x * SPT consecutive sites of one grid's flattened index
// (x fastest), so grids whose rows are shorter than a block keep every
// thread busy; prefix[g] is the first global tile of grid g (prefix[ngrids]
// = all tiles).  CTAs (several waves of the resident capacity) stride over
// the global tiles, so grids of any mix of sizes share one launch, and every
// site goes through exactly the device code of k_step (bit-identical
// results to stepping each grid alone).
#pragma once

#include "lbm_async.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

struct __align__(16) BatchGrid {
  StepParams p;
  void* f[2];
  int cur;
  int pad[3];
};
static_assert(sizeof(BatchGrid) % 16 == 0, "BatchGrid is copied as int4");

// header[0] = number of grids, header[1] = number of tiles
template <class L, int P, int FO, int SPT>
__global__ void __launch_bounds__(256, min_blocks<L, P>())
    k_step_batch(const BatchGrid* __restrict__ grids, const int* __restrict__ prefix,
                 const int* __restrict__ header, int k) {
  using C = Codec<P>;
  using T = typename C::T;
  using R = typename C::R;
  // the parameters of the tile's grid, staged in shared memory once per tile
  __shared__ __align__(16) BatchGrid sg;
  const int ngrids = __ldg(header), ntiles = __ldg(header + 1);
  const int bx = blockDim.x, TW = bx * SPT;
  int gcur = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int lo = 0, hi = ngrids;  // prefix[lo] <= t < prefix[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(prefix + mid) <= t) lo = mid;
      else hi = mid;
    }
    if (lo != gcur) {  // block-uniform
      __syncthreads();
      const int4* src = reinterpret_cast<const int4*>(grids + lo);
      int4* dst = reinterpret_cast<int4*>(&sg);
      for (int w = threadIdx.x; w < (int)(sizeof(BatchGrid) / sizeof(int4)); w += bx) dst[w] = src[w];
      __syncthreads();
      gcur = lo;
    }
    const StepParams& p = sg.p;
    const int lt = t - __ldg(prefix + lo);
    const int par = (sg.cur + k) & 1;
    const T* __restrict__ fin = static_cast<const T*>(sg.f[par]);
    T* __restrict__ fout = static_cast<T*>(sg.f[par ^ 1]);
    const int nA = L::D == 2 ? p.ny : p.nz;
#pragma unroll 1
    for (int s = 0; s < SPT; ++s) {
      const int wbase = lt * TW + s * bx;          // first site of this block pass
      const int site = wbase + threadIdx.x;
      const int site0 = wbase + (threadIdx.x & ~31);  // lane 0 of this warp
      if (site0 >= p.N) break;                     // warp-uniform
      // warp-uniform fast-path test from lane 0: the warp's 32 sites lie in
      // one row, wrap around no axis in x and touch no wall
      const int x0 = site0 % p.nx, r0 = site0 / p.nx;
      const int a0 = L::D == 2 ? r0 % p.ny : r0 / p.ny;
      const bool near0 = p.wall != W_NONE && (a0 < 3 || a0 >= nA - 3);
      const bool interior = !near0 && x0 >= 3 && x0 + 31 <= p.nx - 4;
      if (site >= p.N) continue;
      const int x = site % p.nx, row = site / p.nx;
      const int y = row % p.ny, z = row / p.ny;
      constexpr bool SC = scaled_step<P, FO>();
      R d[L::Q];
      if (interior) pull_interior<L, P, R, LD_RO, SC>(fin + site, p, y, z, d);
      else pull<L, P, R, LD_RO, SC>(fin, p, x, y, z, d);
      R g[3];
      site_force_r<L::D, R>(p, x, y, z, site, g);
      collide_store<L, P, FO, SC>(d, g, site, fout, p);
    }
  }
}

// Halo-staged variant (FP32-shifted storage, one site per thread): while a
// block collides tile t, the populations its sites pull for its next tile
// t + gridDim.x are already being copied with cp.async into the other stage
// of a shared-memory buffer [2][Q][blockDim.x] (each thread fills and reads
// its own column, so cp.async.wait_group orders its reads); warps whose pulls
// wrap around x or touch a wall load directly.  The parameters of the two
// tiles in flight occupy two shared-memory slots.  Same device code per site
// as k_step: results are bit-identical.  The autotuner times it against the
// plain batch kernel.
template <class L, int P, int FO>
__global__ void __launch_bounds__(256, min_blocks<L, P>())
    k_step_batch_staged(const BatchGrid* __restrict__ grids, const int* __restrict__ prefix,
                        const int* __restrict__ header, int k) {
  static_assert(P == P_FP32S, "4-byte populations (cp.async of 4 bytes)");
  using C = Codec<P>;
  using T = typename C::T;
  using R = typename C::R;
  constexpr int Q = L::Q, D = L::D;
  extern __shared__ __align__(16) unsigned char sbuf[];  // [2][Q][blockDim.x] of T
  __shared__ __align__(16) BatchGrid sg[2];
  const int ngrids = __ldg(header), ntiles = __ldg(header + 1);
  const int bx = blockDim.x, tid = threadIdx.x;
  const int stride = bx * (int)sizeof(T);
  const uint32_t col0 = (uint32_t)__cvta_generic_to_shared(sbuf) + tid * (int)sizeof(T);
  const uint32_t stage_bytes = (uint32_t)Q * stride;

  auto grid_of = [&](int t) {
    int lo = 0, hi = ngrids;  // prefix[lo] <= t < prefix[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(prefix + mid) <= t) lo = mid;
      else hi = mid;
    }
    return lo;
  };
  auto load_params = [&](int g, int slot) {
    const int4* src = reinterpret_cast<const int4*>(grids + g);
    int4* dst = reinterpret_cast<int4*>(&sg[slot]);
    for (int w = tid; w < (int)(sizeof(BatchGrid) / sizeof(int4)); w += bx) dst[w] = src[w];
  };
  // site of this thread in tile t of grid g, and whether its warp can be
  // prefetched (32 sites in one row, no x wrap, no wall)
  auto geometry = [&](int t, int g, const StepParams& p, int& site, int& x, int& y, int& z, bool& fast) {
    const int lt = t - __ldg(prefix + g);
    site = lt * bx + tid;
    const int site0 = lt * bx + (tid & ~31);
    const int nA = D == 2 ? p.ny : p.nz;
    const int x0 = site0 % p.nx, r0 = site0 / p.nx;
    const int a0 = D == 2 ? r0 % p.ny : r0 / p.ny;
    const bool near0 = p.wall != W_NONE && (a0 < 3 || a0 >= nA - 3);
    fast = site0 < p.N && !near0 && x0 >= 3 && x0 + 31 <= p.nx - 4;
    x = site % p.nx;
    const int row = site / p.nx;
    y = row % p.ny;
    z = row / p.ny;
  };

  int t = blockIdx.x;
  if (t >= ntiles) return;
  int g = grid_of(t);
  load_params(g, 0);
  __syncthreads();
  int site, x, y, z;
  bool fast;
  geometry(t, g, sg[0].p, site, x, y, z, fast);
  {
    const StepParams& p = sg[0].p;
    const T* fin = static_cast<const T*>(sg[0].f[(sg[0].cur + k) & 1]);
    if (fast) prefetch_interior<L, P>(fin + site, p, y, z, col0, stride);
  }
  cp_async_commit();
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int cs = it & 1, ns = cs ^ 1;
    const int tn = t + gridDim.x;
    int gn = 0, siten = 0, xn = 0, yn = 0, zn = 0;
    bool fastn = false;
    __syncthreads();  // every thread is done with the slot and stage of tile it - 1
    if (tn < ntiles) {
      gn = grid_of(tn);
      load_params(gn, ns);
    }
    __syncthreads();
    if (tn < ntiles) {
      const StepParams& pn = sg[ns].p;
      geometry(tn, gn, pn, siten, xn, yn, zn, fastn);
      const T* finn = static_cast<const T*>(sg[ns].f[(sg[ns].cur + k) & 1]);
      if (fastn) prefetch_interior<L, P>(finn + siten, pn, yn, zn, col0 + ns * stage_bytes, stride);
    }
    cp_async_commit();
    cp_async_wait<1>();  // this thread's copies of tile t have landed
    const StepParams& p = sg[cs].p;
    if (site < p.N) {
      const int par = (sg[cs].cur + k) & 1;
      const T* __restrict__ fin = static_cast<const T*>(sg[cs].f[par]);
      T* __restrict__ fout = static_cast<T*>(sg[cs].f[par ^ 1]);
      R d[Q];
      if (fast) {
        const T* sc = reinterpret_cast<const T*>(sbuf + cs * stage_bytes) + tid;
        static_for<0, Q>([&](auto I) {
          constexpr int i = I;
          d[i] = R(C::template decode<L, i>(sc[i * bx], p));
        });
      } else {
        pull<L, P, R, LD_RO>(fin, p, x, y, z, d);
      }
      R gv[3];
      site_force_r<D, R>(p, x, y, z, site, gv);
      collide_store<L, P, FO>(d, gv, site, fout, p);
    }
    site = siten;
    x = xn;
    y = yn;
    z = zn;
    fast = fastn;
  }
  cp_async_wait<0>();
}

}  // namespace lbm
