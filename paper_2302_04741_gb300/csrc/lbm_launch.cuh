// lbm_launch.cuh -- host-side launchers of one lattice's kernels (runtime
// precision / force-order dispatch to the template instantiations).
#pragma once

#include <cuda_runtime.h>

#include "lbm_async.cuh"
#include "lbm_batch.cuh"
#include "lbm_tma.cuh"
#include "lbm_wave.cuh"

namespace lbm {

// Function table of one lattice, filled by lattice_ops<L>().
struct LatticeOps {
  int Q, D;
  cudaError_t (*step)(int P, int FO, const void* fin, void* fout, const StepParams& p, int bx,
                      bool overlap, cudaStream_t s);  // p.solid set: FP64 / FP32 only
  cudaError_t (*init)(int P, int mode, const double* rho, const double* u, const double* T,
                      void* fout, unsigned* maxbits, int FO, const StepParams& p, cudaStream_t s);
  cudaError_t (*moments)(int P, const void* fin, double* rho, double* u, double* T, double* q,
                         int FO, const StepParams& p, cudaStream_t s);
  // ticket != nullptr: the last block also reduces into out (see k_conserved)
  cudaError_t (*conserved)(int P, const void* fin, double* part, unsigned* bad,
                           unsigned* ticket, double* out, const int* err,
                           const StepParams& p, int nblocks, cudaStream_t s);
  // two-kernel form: merge the partials of a ticketless conserved() into out
  cudaError_t (*conserved_final)(int P, const double* part, const unsigned* bad, int nblocks,
                                 double* out, const StepParams& p, cudaStream_t s);
  cudaError_t (*pulled)(int P, const void* fin, double* out, const StepParams& p, cudaStream_t s);
  cudaError_t (*state)(int P, int dir, void* f, double* io, const StepParams& p, cudaStream_t s);
  // TMA-staged step (FP32-shifted and FP16-scaled storage only)
  size_t (*tma_smem)(int P, int stages);
  cudaError_t (*tma_prepare)(int P, int stages, int* blocks_per_sm);
  cudaError_t (*step_tma)(int P, int FO, const CUtensorMap* map, const void* fin, void* fout,
                          const StepParams& p, int grid, int stages, cudaStream_t s);
  // prefetching persistent step (FP32-shifted storage)
  cudaError_t (*async_occupancy)(int FO, int bx, int* blocks_per_sm);
  cudaError_t (*step_async)(int FO, const void* fin, void* fout, const StepParams& p, int grid,
                            int bx, cudaStream_t s);
  // batch step (FP32-shifted and FP16-scaled storage; SPT 1 or 2)
  cudaError_t (*batch_occupancy)(int P, int FO, int spt, int bx, int* blocks_per_sm);
  cudaError_t (*batch_step)(int P, int FO, int spt, const BatchGrid* grids, const int* prefix,
                            const int* header, int k, int grid, int bx, cudaStream_t s);
  // halo-staged batch step (FP32-shifted storage, one site per thread)
  cudaError_t (*batch_staged_occupancy)(int FO, int bx, int* blocks_per_sm);
  cudaError_t (*batch_step_staged)(int FO, const BatchGrid* grids, const int* prefix, const int* header,
                                   int k, int grid, int bx, cudaStream_t s);
  // several steps in one persistent launch (FP32-shifted and FP16-scaled
  // storage; force orders 0..2); sync: 1 + n_lines zeroed words
  cudaError_t (*wave_occupancy)(int P, int FO, int* blocks_per_sm);
  cudaError_t (*step_wave)(int P, int FO, void* f0, void* f1, const StepParams& p, int nsteps,
                           unsigned* sync, int grid, cudaStream_t s);
};

// ---- wall tables (host side; shared by lbm_create and lbm_conserved_static)
// Equilibrium deviation f0_i(1, 0, T) - w_i = w_i A0(|xi_i|^2) of a wall at
// rest (u = 0), the rest-frame value of the Hermite-expanded equilibrium.
template <class L>
inline void wall_equilibrium(double T, double* fwd, double* fw) {
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

// The thermal-wall constants of StepParams for wall temperatures T_lo (at
// x_a = -1/2) and T_hi (at x_a = n_a - 1/2) on the last axis: the wall
// Maxwellian per side and the per-column mass balance of the diffuse wall.
template <class L>
inline void wall_tables(StepParams& p, double T_lo, double T_hi) {
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

// Per-site launch: blocks of bx sites along x, one row per block, over the
// layers a0 .. a0 + na - 1 of the last axis (StepParams::a0, na).
template <int D>
inline dim3 row_grid(const StepParams& p, int bx) {
  return dim3((unsigned)((p.nx + bx - 1) / bx), (unsigned)(D == 2 ? p.na : p.ny),
              (unsigned)(D == 2 ? 1 : p.na));
}

template <class L>
struct Ops {
  template <int P>
  using T = typename Codec<P>::T;

  // overlap: launch as a programmatic dependent of the stream's previous
  // kernel (the step kernel waits with griddepcontrol.wait before its loads)
  static cudaError_t step(int P, int FO, const void* fin, void* fout, const StepParams& p, int bx,
                          bool overlap, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = row_grid<L::D>(p, bx);
    cfg.blockDim = dim3(bx);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 1 : 0;
    cudaError_t e = cudaSuccess;
    if (p.solid) {
#define LBM_SOLID_CASE(PP, FF)                                                                 \
  case PP * 4 + FF:                                                                            \
    e = cudaLaunchKernelEx(&cfg, k_step<L, PP, FF, true>, (const T<PP>*)fin, (T<PP>*)fout, p); \
    break;
      switch (P * 4 + FO) {
        LBM_SOLID_CASE(0, 0) LBM_SOLID_CASE(0, 1) LBM_SOLID_CASE(0, 2) LBM_SOLID_CASE(0, 3)
        LBM_SOLID_CASE(1, 0) LBM_SOLID_CASE(1, 1) LBM_SOLID_CASE(1, 2) LBM_SOLID_CASE(1, 3)
        default: return cudaErrorInvalidValue;
      }
#undef LBM_SOLID_CASE
      return e != cudaSuccess ? e : cudaGetLastError();
    }
#define LBM_STEP_CASE(PP, FF)                                                            \
  case PP * 4 + FF:                                                                      \
    e = cudaLaunchKernelEx(&cfg, k_step<L, PP, FF>, (const T<PP>*)fin, (T<PP>*)fout, p); \
    break;
    // FO 3: force order 2 with the sigma-bar terms (plain kernel only);
    // P 3: FP64 storage with float-float arithmetic
    switch (P * 4 + FO) {
      LBM_STEP_CASE(0, 0) LBM_STEP_CASE(0, 1) LBM_STEP_CASE(0, 2) LBM_STEP_CASE(0, 3)
      LBM_STEP_CASE(1, 0) LBM_STEP_CASE(1, 1) LBM_STEP_CASE(1, 2) LBM_STEP_CASE(1, 3)
      LBM_STEP_CASE(2, 0) LBM_STEP_CASE(2, 1) LBM_STEP_CASE(2, 2) LBM_STEP_CASE(2, 3)
      LBM_STEP_CASE(3, 0) LBM_STEP_CASE(3, 1) LBM_STEP_CASE(3, 2) LBM_STEP_CASE(3, 3)
      default: return cudaErrorInvalidValue;
    }
#undef LBM_STEP_CASE
    return e != cudaSuccess ? e : cudaGetLastError();
  }

  static cudaError_t init(int P, int mode, const double* rho, const double* u, const double* T_,
                          void* fout, unsigned* maxbits, int FO, const StepParams& p,
                          cudaStream_t s) {
    const dim3 g = row_grid<L::D>(p, 128), b(128);
    if (mode == 0) {
      k_init<L, P_FP16S, 0><<<g, b, 0, s>>>(rho, u, T_, (T<P_FP16S>*)fout, maxbits, FO, p);
    } else if (P == P_FP64) {
      k_init<L, P_FP64, 1><<<g, b, 0, s>>>(rho, u, T_, (T<P_FP64>*)fout, maxbits, FO, p);
    } else if (P == P_FP32S) {
      k_init<L, P_FP32S, 1><<<g, b, 0, s>>>(rho, u, T_, (T<P_FP32S>*)fout, maxbits, FO, p);
    } else {
      k_init<L, P_FP16S, 1><<<g, b, 0, s>>>(rho, u, T_, (T<P_FP16S>*)fout, maxbits, FO, p);
    }
    return cudaGetLastError();
  }

  static cudaError_t moments(int P, const void* fin, double* rho, double* u, double* T_,
                             double* q, int FO, const StepParams& p, cudaStream_t s) {
    const dim3 g = row_grid<L::D>(p, 128), b(128);
    if (P == P_FP64) k_moments<L, P_FP64><<<g, b, 0, s>>>((const T<P_FP64>*)fin, rho, u, T_, q, FO, p);
    else if (P == P_FP32S) k_moments<L, P_FP32S><<<g, b, 0, s>>>((const T<P_FP32S>*)fin, rho, u, T_, q, FO, p);
    else k_moments<L, P_FP16S><<<g, b, 0, s>>>((const T<P_FP16S>*)fin, rho, u, T_, q, FO, p);
    return cudaGetLastError();
  }

  // nblocks: blocks of the grid-stride conservation pass (partials written)
  static cudaError_t conserved(int P, const void* fin, double* part, unsigned* bad,
                               unsigned* ticket, double* out, const int* err,
                               const StepParams& p, int nblocks, cudaStream_t s) {
    const dim3 g(nblocks), b(128);
    if (P == P_FP64)
      k_conserved<L, P_FP64><<<g, b, 0, s>>>((const T<P_FP64>*)fin, part, bad, ticket, out, err, p);
    else if (P == P_FP32S)
      k_conserved<L, P_FP32S><<<g, b, 0, s>>>((const T<P_FP32S>*)fin, part, bad, ticket, out, err, p);
    else
      k_conserved<L, P_FP16S><<<g, b, 0, s>>>((const T<P_FP16S>*)fin, part, bad, ticket, out, err, p);
    return cudaGetLastError();
  }

  static cudaError_t conserved_final(int P, const double* part, const unsigned* bad, int nblocks,
                                     double* out, const StepParams& p, cudaStream_t s) {
    if (P == P_FP64) k_conserved_final<L, P_FP64><<<1, 128, 0, s>>>(part, bad, nblocks, out, p);
    else if (P == P_FP32S) k_conserved_final<L, P_FP32S><<<1, 128, 0, s>>>(part, bad, nblocks, out, p);
    else k_conserved_final<L, P_FP16S><<<1, 128, 0, s>>>(part, bad, nblocks, out, p);
    return cudaGetLastError();
  }

  static cudaError_t pulled(int P, const void* fin, double* out, const StepParams& p,
                            cudaStream_t s) {
    const dim3 g = row_grid<L::D>(p, 128), b(128);
    if (P == P_FP64) k_get_pulled<L, P_FP64><<<g, b, 0, s>>>((const T<P_FP64>*)fin, out, p);
    else if (P == P_FP32S) k_get_pulled<L, P_FP32S><<<g, b, 0, s>>>((const T<P_FP32S>*)fin, out, p);
    else k_get_pulled<L, P_FP16S><<<g, b, 0, s>>>((const T<P_FP16S>*)fin, out, p);
    return cudaGetLastError();
  }

  static cudaError_t state(int P, int dir, void* f, double* io, const StepParams& p,
                           cudaStream_t s) {
    const dim3 g = row_grid<L::D>(p, 128), b(128);
#define LBM_STATE_CASE(PP)                                                                 \
  if (P == PP) {                                                                           \
    if (dir == 0) k_state<L, PP, 0><<<g, b, 0, s>>>((T<PP>*)f, io, p);                     \
    else k_state<L, PP, 1><<<g, b, 0, s>>>((T<PP>*)f, io, p);                              \
  }
    LBM_STATE_CASE(P_FP64) LBM_STATE_CASE(P_FP32S) LBM_STATE_CASE(P_FP16S)
#undef LBM_STATE_CASE
    return cudaGetLastError();
  }

  static size_t tma_smem(int P, int S) {
    const size_t sb = P == P_FP16S ? tma_stage_bytes<L, P_FP16S>() : tma_stage_bytes<L, P_FP32S>();
    return (size_t)S * sb + 2 * (size_t)S * sizeof(uint64_t) + 128;  // + alignment slack
  }

  // Opts every instantiation of precision P into `stages` stages of dynamic
  // shared memory and returns the resident blocks per SM.
  static cudaError_t tma_prepare(int P, int S, int* bps) {
    const int smem = (int)tma_smem(P, S);
    cudaError_t e = cudaSuccess;
    int occ = 0;
#define LBM_TMA_PREP(PP, FF)                                                                  \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step_tma<L, PP, FF>,                       \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
  if (e == cudaSuccess && FF == 2)                                                            \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_tma<L, PP, FF>, TMA_THREADS, smem);
    if (P == P_FP32S) { LBM_TMA_PREP(P_FP32S, 0) LBM_TMA_PREP(P_FP32S, 1) LBM_TMA_PREP(P_FP32S, 2) }
    else if (P == P_FP16S) { LBM_TMA_PREP(P_FP16S, 0) LBM_TMA_PREP(P_FP16S, 1) LBM_TMA_PREP(P_FP16S, 2) }
    else return cudaErrorInvalidValue;
#undef LBM_TMA_PREP
    *bps = occ;
    return e;
  }

  static cudaError_t step_tma(int P, int FO, const CUtensorMap* map, const void* fin, void* fout,
                              const StepParams& p, int grid, int S, cudaStream_t s) {
    const size_t smem = tma_smem(P, S);
#define LBM_TMA_CASE(PP, FF)                                                               \
  case PP * 3 + FF:                                                                        \
    k_step_tma<L, PP, FF><<<grid, TMA_THREADS, smem, s>>>(*map, (const T<PP>*)fin,         \
                                                           (T<PP>*)fout, p, S);            \
    break;
    switch (P * 3 + FO) {
      LBM_TMA_CASE(1, 0) LBM_TMA_CASE(1, 1) LBM_TMA_CASE(1, 2)
      LBM_TMA_CASE(2, 0) LBM_TMA_CASE(2, 1) LBM_TMA_CASE(2, 2)
      default: return cudaErrorInvalidValue;
    }
#undef LBM_TMA_CASE
    return cudaGetLastError();
  }

  template <int PP, int FF, int SS>
  static cudaError_t batch_occ_one(int bx, int* bps) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_step_batch<L, PP, FF, SS>, bx, 0);
  }

  static cudaError_t batch_occupancy(int P, int FO, int spt, int bx, int* bps) {
#define LBM_BOCC(PP, FF, SS) \
  if (P == PP && FO == FF && spt == SS) return batch_occ_one<PP, FF, SS>(bx, bps);
    LBM_BOCC(1, 0, 1) LBM_BOCC(1, 1, 1) LBM_BOCC(1, 2, 1) LBM_BOCC(1, 0, 2) LBM_BOCC(1, 1, 2) LBM_BOCC(1, 2, 2)
    LBM_BOCC(2, 0, 1) LBM_BOCC(2, 1, 1) LBM_BOCC(2, 2, 1) LBM_BOCC(2, 0, 2) LBM_BOCC(2, 1, 2) LBM_BOCC(2, 2, 2)
#undef LBM_BOCC
    return cudaErrorInvalidValue;
  }

  static cudaError_t batch_step(int P, int FO, int spt, const BatchGrid* grids, const int* prefix,
                                const int* header, int k, int grid, int bx, cudaStream_t s) {
#define LBM_BSTEP(PP, FF, SS)                                                               \
  if (P == PP && FO == FF && spt == SS) {                                                    \
    k_step_batch<L, PP, FF, SS><<<grid, bx, 0, s>>>(grids, prefix, header, k);                \
    return cudaGetLastError();                                                              \
  }
    LBM_BSTEP(1, 0, 1) LBM_BSTEP(1, 1, 1) LBM_BSTEP(1, 2, 1) LBM_BSTEP(1, 0, 2) LBM_BSTEP(1, 1, 2) LBM_BSTEP(1, 2, 2)
    LBM_BSTEP(2, 0, 1) LBM_BSTEP(2, 1, 1) LBM_BSTEP(2, 2, 1) LBM_BSTEP(2, 0, 2) LBM_BSTEP(2, 1, 2) LBM_BSTEP(2, 2, 2)
#undef LBM_BSTEP
    return cudaErrorInvalidValue;
  }

  // same shared-memory stages as the prefetching step: [2][Q][bx] floats
  static cudaError_t batch_staged_occupancy(int FO, int bx, int* bps) {
    const int smem = (int)async_smem(bx);
    cudaError_t e = cudaSuccess;
#define LBM_SBOCC(FF)                                                                            \
  if (FO == FF) {                                                                                \
    e = cudaFuncSetAttribute(k_step_batch_staged<L, P_FP32S, FF>,                                \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);                 \
    if (e == cudaSuccess)                                                                        \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_step_batch_staged<L, P_FP32S, FF>, \
                                                        bx, smem);                               \
    return e;                                                                                    \
  }
    LBM_SBOCC(0) LBM_SBOCC(1) LBM_SBOCC(2)
#undef LBM_SBOCC
    return cudaErrorInvalidValue;
  }

  static cudaError_t batch_step_staged(int FO, const BatchGrid* grids, const int* prefix, const int* header,
                                       int k, int grid, int bx, cudaStream_t s) {
    const size_t smem = async_smem(bx);
    if (FO == 0) k_step_batch_staged<L, P_FP32S, 0><<<grid, bx, smem, s>>>(grids, prefix, header, k);
    else if (FO == 1) k_step_batch_staged<L, P_FP32S, 1><<<grid, bx, smem, s>>>(grids, prefix, header, k);
    else if (FO == 2) k_step_batch_staged<L, P_FP32S, 2><<<grid, bx, smem, s>>>(grids, prefix, header, k);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
  }

  static cudaError_t wave_occupancy(int P, int FO, int* bps) {
#define LBM_WOCC(PP, FF)                                                                         \
  if (P == PP && FO == FF)                                                                       \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_step_wave<L, PP, FF>, WAVE_BX, 0);
    LBM_WOCC(1, 0) LBM_WOCC(1, 1) LBM_WOCC(1, 2) LBM_WOCC(2, 0) LBM_WOCC(2, 1) LBM_WOCC(2, 2)
#undef LBM_WOCC
    return cudaErrorInvalidValue;
  }

  static cudaError_t step_wave(int P, int FO, void* f0, void* f1, const StepParams& p, int nsteps,
                               unsigned* sync, int grid, cudaStream_t s) {
#define LBM_WSTEP(PP, FF)                                                                      \
  if (P == PP && FO == FF) {                                                                   \
    k_step_wave<L, PP, FF><<<grid, WAVE_BX, 0, s>>>((T<PP>*)f0, (T<PP>*)f1, p, nsteps, sync);  \
    return cudaGetLastError();                                                                 \
  }
    LBM_WSTEP(1, 0) LBM_WSTEP(1, 1) LBM_WSTEP(1, 2) LBM_WSTEP(2, 0) LBM_WSTEP(2, 1) LBM_WSTEP(2, 2)
#undef LBM_WSTEP
    return cudaErrorInvalidValue;
  }

  static size_t async_smem(int bx) { return 2 * (size_t)L::Q * bx * sizeof(float); }

  static cudaError_t async_occupancy(int FO, int bx, int* bps) {
    const int smem = (int)async_smem(bx);
    cudaError_t e = cudaSuccess;
#define LBM_AOCC(FF)                                                                            \
  if (FO == FF) {                                                                               \
    e = cudaFuncSetAttribute(k_step_async<L, P_FP32S, FF>,                                      \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);                \
    if (e == cudaSuccess)                                                                       \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_step_async<L, P_FP32S, FF>, bx,  \
                                                        smem);                                  \
    return e;                                                                                   \
  }
    LBM_AOCC(0) LBM_AOCC(1) LBM_AOCC(2)
#undef LBM_AOCC
    return cudaErrorInvalidValue;
  }

  static cudaError_t step_async(int FO, const void* fin, void* fout, const StepParams& p, int grid,
                                int bx, cudaStream_t s) {
    const size_t smem = async_smem(bx);
    if (FO == 0) k_step_async<L, P_FP32S, 0><<<grid, bx, smem, s>>>((const float*)fin, (float*)fout, p);
    else if (FO == 1) k_step_async<L, P_FP32S, 1><<<grid, bx, smem, s>>>((const float*)fin, (float*)fout, p);
    else k_step_async<L, P_FP32S, 2><<<grid, bx, smem, s>>>((const float*)fin, (float*)fout, p);
    return cudaGetLastError();
  }

  static LatticeOps table() {
    return LatticeOps{L::Q, L::D, &step, &init, &moments, &conserved, &conserved_final, &pulled, &state,
                      &tma_smem, &tma_prepare, &step_tma, &async_occupancy, &step_async,
                      &batch_occupancy, &batch_step, &batch_staged_occupancy, &batch_step_staged,
                      &wave_occupancy, &step_wave};
  }
};

const LatticeOps& ops_d2q37();
const LatticeOps& ops_d3q39();
void set_global_error(const char* msg);

}  // namespace lbm
