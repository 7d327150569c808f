// lbm_wave.cuh -- several steps in one persistent launch (wavefront order).
//
// A launch of the plain step kernel ends with a drain (the last blocks run
// while SMs empty out) and the next starts with a ramp; on the 1024 x 512
// cell that is a noticeable share of a 32 us step.  Here one launch runs K
// steps: blocks take work items (step s, line a of the last axis, tile k of
// that line) from an atomic counter in step-major order, so the GPU moves on
// to step s + 1 while step s finishes its last lines.
//
// Dependencies.  A site pulls from at most 3 lines away along the last axis
// (|e| <= 3), so line a of step s may run once lines a - 3 .. a + 3 (wrapped
// when that axis is periodic) have finished step s - 1.  That also covers
// the ping-pong hazard: step s writes the buffer step s - 1 read, and the
// reads of line a's old values all belong to lines a - 3 .. a + 3 of step
// s - 1.  done[a] counts the tiles of line a finished over all steps, so
// "line a finished step s - 1" is done[a] >= s * tiles_per_line (a tile of
// line a at step s needs done[a] >= s * tiles_per_line itself, so the count
// cannot include a later step's tiles before an earlier step's are all in).
//
// Progress: a block waits only on items dispensed before its own, and a
// dispensed item belongs to a block that is running, so the waits end.  They
// are still bounded: after WAVE_SPIN_LIMIT polls a block sets the context's
// error flag and carries on (the results are then void and lbm_conserved
// reports LBM_ETIMEOUT).
//
// Memory order: a finished tile's stores are fenced by every thread, the
// block synchronises, and one thread publishes with a release add; a waiting
// thread polls with acquire loads and the block synchronises before it pulls
// with L2-only loads (the read-only and L1 paths could return lines of this
// buffer from two steps earlier).  The collision is the device code of
// k_step: results are bit-identical to K launches of the plain kernel.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int WAVE_BX = 128;                       // sites per tile (one row segment)
constexpr unsigned WAVE_SPIN_LIMIT = 1u << 22;     // polls (~0.5 s) before giving up

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Resident 128-thread blocks per SM the register cap is sized for (the same
// per-thread budgets as the plain kernel: 85 registers for float D2Q37, 128
// for float D3Q39, no cap in FP64).
#ifndef LBM_WAVE_D2Q37_BLOCKS  // tuning hook
#define LBM_WAVE_D2Q37_BLOCKS 6
#endif
template <class L, int P>
constexpr int wave_min_blocks() {
  return P == P_FP64 ? 2 : (L::Q > 37 ? 4 : LBM_WAVE_D2Q37_BLOCKS);
}

// sync: [0] the item counter, [1 + a] done count of line a; zero at launch.
template <class L, int P, int FO>
__global__ void __launch_bounds__(WAVE_BX, wave_min_blocks<L, P>())
    k_step_wave(typename Codec<P>::T* f0, typename Codec<P>::T* f1, const StepParams p, int nsteps,
                unsigned* sync) {
  using C = Codec<P>;
  using T = typename C::T;
  using R = typename C::R;
  constexpr int D = L::D;
  const int nA = D == 2 ? p.ny : p.nz;
  const int ntx = (p.nx + WAVE_BX - 1) / WAVE_BX;
  const int tpl = ntx * (D == 2 ? 1 : p.ny);  // tiles per line
  const unsigned per_step = (unsigned)nA * (unsigned)tpl;
  const unsigned total = per_step * (unsigned)nsteps;
  unsigned* done = sync + 1;
  __shared__ unsigned s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(sync, 1u);
    __syncthreads();
    const unsigned item = s_item;
    if (item >= total) return;
    const int s = (int)(item / per_step);
    const unsigned r = item - (unsigned)s * per_step;
    const int a = (int)(r / (unsigned)tpl), k = (int)(r % (unsigned)tpl);
    const int y = D == 2 ? a : k / ntx;
    const int z = D == 2 ? 0 : a;
    const int xt = D == 2 ? k : k % ntx;
    if (s > 0 && threadIdx.x == 0) {
      const unsigned target = (unsigned)s * (unsigned)tpl;
      // once any block has given up, nobody waits any more (results void)
      bool gave_up = *(volatile const int*)p.err != 0;
      for (int da = -3; da <= 3 && !gave_up; ++da) {
        int a2 = a + da;
        if (a2 < 0 || a2 >= nA) {
          if (p.wall != W_NONE) continue;
          a2 = a2 < 0 ? a2 + nA : a2 - nA;
        }
        unsigned polls = 0;
        while (ld_acquire_gpu(done + a2) < target) {
          if (++polls > WAVE_SPIN_LIMIT) {
            atomicExch(p.err, 1);
            gave_up = true;
            break;
          }
          __nanosleep(64);
        }
      }
    }
    __syncthreads();
    const T* fin = (s & 1) ? f1 : f0;
    T* fout = (s & 1) ? f0 : f1;
    const int x = xt * WAVE_BX + threadIdx.x;
    if (x < p.nx) {
      const int site = (z * p.ny + y) * p.nx + x;
      const int aw = D == 2 ? y : z;
      const bool near = p.wall != W_NONE && (aw < 3 || aw >= nA - 3);
      const int wx0 = xt * WAVE_BX + (threadIdx.x & ~31);
      const bool interior = !near && wx0 >= 3 && wx0 + 31 <= p.nx - 4;
      R g[3];
      site_force_r<D, R>(p, x, y, z, site, g);
      constexpr bool SC = scaled_step<P, FO>();
      R d[L::Q];
      if (interior) pull_interior<L, P, R, LD_CG, SC>(fin + site, p, y, z, d);
      else pull<L, P, R, LD_CG, SC>(fin, p, x, y, z, d);
      collide_store<L, P, FO, SC>(d, g, site, fout, p);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) red_release_gpu(done + a, 1u);
  }
}

}  // namespace lbm
