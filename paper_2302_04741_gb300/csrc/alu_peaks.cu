// alu_peaks.cu -- issue-rate probes of the arithmetic the FP64 step uses.
//
// On GB300 the FP64 units run at a small fraction of the FP32 rate, so the
// FP64 step is bound by arithmetic, not by bytes; the roofline of that step
// needs the measured rates of its operations.  Each probe kernel runs a
// long chain of the probed instruction in 8 independent accumulators per
// thread (enough to cover the pipeline latency) over a grid of 8 blocks of
// 256 threads per SM, and returns operations per second (an FMA counts as
// one operation here; flop rates are twice that for FMAs).
//
// kinds: 0 DFMA, 1 DADD, 2 FFMA, 3 double -> float conversion,
//        4 float -> double conversion, 5 integer add (32-bit),
//        6 packed FFMA (fma.rn.f32x2: two FMAs per instruction, counted as
//        two operations), 7 float -> half -> float round trips (two
//        conversions per step)
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdio>

namespace {

constexpr int kAcc = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_dfma(double* out, double a, double b) {
  double x[kAcc];
  for (int k = 0; k < kAcc; ++k) x[k] = threadIdx.x * 1e-9 + k;
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int k = 0; k < kAcc; ++k) x[k] = fma(x[k], a, b);
  double s = 0.0;
  for (int k = 0; k < kAcc; ++k) s += x[k];
  if (s == 12345.678) out[0] = s;  // keeps the chain; never true
}

__global__ void __launch_bounds__(256) k_dadd(double* out, double a) {
  double x[kAcc];
  for (int k = 0; k < kAcc; ++k) x[k] = threadIdx.x * 1e-9 + k;
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int k = 0; k < kAcc; ++k) x[k] = x[k] + a;
  double s = 0.0;
  for (int k = 0; k < kAcc; ++k) s += x[k];
  if (s == 12345.678) out[0] = s;
}

__global__ void __launch_bounds__(256) k_ffma(double* out, float a, float b) {
  float x[kAcc];
  for (int k = 0; k < kAcc; ++k) x[k] = threadIdx.x * 1e-6f + k;
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int k = 0; k < kAcc; ++k) x[k] = fmaf(x[k], a, b);
  float s = 0.f;
  for (int k = 0; k < kAcc; ++k) s += x[k];
  if (s == 12345.678f) out[0] = s;
}

// double -> float -> double round trips: two conversions per step of each
// chain (counted as two operations)
__global__ void __launch_bounds__(256) k_cvt(double* out, double a) {
  double x[kAcc];
  for (int k = 0; k < kAcc; ++k) x[k] = threadIdx.x * 1e-9 + k + a;
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int k = 0; k < kAcc; ++k) x[k] = (double)(__double2float_rn(x[k]));
  double s = 0.0;
  for (int k = 0; k < kAcc; ++k) s += x[k];
  if (s == 12345.678) out[0] = s;
}

__global__ void __launch_bounds__(256) k_iadd(double* out, int a) {
  int x[kAcc];
  for (int k = 0; k < kAcc; ++k) x[k] = threadIdx.x + k;
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int k = 0; k < kAcc; ++k) x[k] = (x[k] ^ a) + a;  // two integer operations
  int s = 0;
  for (int k = 0; k < kAcc; ++k) s += x[k];
  if (s == 12345678) out[0] = s;
}

__global__ void __launch_bounds__(256) k_ffma2(double* out, float a, float b) {
  unsigned long long x[kAcc], av, bv;
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
  for (int k = 0; k < kAcc; ++k) {
    const float lo = threadIdx.x * 1e-6f + k, hi = lo + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(lo), "f"(hi));
  }
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int k = 0; k < kAcc; ++k) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(av), "l"(bv));
  float s = 0.f;
  for (int k = 0; k < kAcc; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
    s += lo + hi;
  }
  if (s == 12345.678f) out[0] = s;
}

__global__ void __launch_bounds__(256) k_half(double* out, float a) {
  float x[kAcc];
  for (int k = 0; k < kAcc; ++k) x[k] = threadIdx.x * 1e-6f + k + a;
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int k = 0; k < kAcc; ++k) x[k] = __half2float(__float2half_rn(x[k])) + a;
  float s = 0.f;
  for (int k = 0; k < kAcc; ++k) s += x[k];
  if (s == 12345.678f) out[0] = s;
}

}  // namespace

// Operations per second of probe `kind` on the current device (reps timed
// launches after one warm-up); returns 0 on a CUDA error.
extern "C" double alu_probe(int kind, int reps) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0.0;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return 0.0;
  const dim3 grid(nsm * 8), block(256);
  auto launch = [&]() {
    switch (kind) {
      case 0: k_dfma<<<grid, block>>>(out, 0.999999, 1e-7); break;
      case 1: k_dadd<<<grid, block>>>(out, 1e-7); break;
      case 2: k_ffma<<<grid, block>>>(out, 0.9999f, 1e-4f); break;
      case 3: case 4: k_cvt<<<grid, block>>>(out, 0.25); break;
      case 6: k_ffma2<<<grid, block>>>(out, 0.9999f, 1e-4f); break;
      case 7: k_half<<<grid, block>>>(out, 0.25f); break;
      default: k_iadd<<<grid, block>>>(out, 12345); break;
    }
  };
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();
  cudaEventRecord(e0);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const bool ok = cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (!ok || ms <= 0.f) return 0.0;
  const double per_launch = (double)grid.x * block.x * kAcc * kIters * (kind >= 3 ? 2.0 : 1.0);
  // (kind 7 also adds one FADD per step, which is not counted)
  return per_launch * reps / (ms * 1e-3);
}
