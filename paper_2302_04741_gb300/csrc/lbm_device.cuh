// lbm_device.cuh -- device-side building blocks of the fused step.
//
// Notation follows Li & Shan (arXiv 2302.04741), Sec. 2: xi_i = c e_i are the
// abscissae, w_i the weights, f~ the pulled (pre-collision) distribution, the
// mid-point state is rho, u = u~ + g/2, theta.  All arithmetic works on the
// deviations d_i = f~_i - w_i (rho_0 = 1), which keeps float arithmetic
// accurate: the moments of the uniform state (sum w = 1, sum w xi = 0,
// sum w xi^2 = D) are carried exactly and only the deviations are rounded.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lattice_tables.cuh"
#include "lbm_df.cuh"

namespace lbm {

constexpr int QMAX = 39;

// P_FP64DF: FP64 storage with float-float arithmetic in the step kernel
// (the other kernels of such a context run P_FP64 on the same buffers).
enum Precision { P_FP64 = 0, P_FP32S = 1, P_FP16S = 2, P_FP64DF = 3 };
enum Wall { W_NONE = 0, W_BOUNCE = 1, W_THERMAL = 2 };
enum GKind { G_UNIFORM = 0, G_SINE = 1, G_FIELD = 2 };

// Everything a step kernel needs, passed by value (constant bank).
struct StepParams {
  int nx, ny, nz;    // nz = 1 on D2Q37
  int N;             // sites (< 2^31)
  int wall;          // Wall, on the last axis (y for D = 2, z for D = 3)
  double omega;      // 1 / tau-hat
  int gkind;         // GKind
  int gaxis;         // G_SINE: axis of the wave
  double g0[3];      // G_UNIFORM / G_SINE amplitude
  const double* gtab;  // G_SINE: sin(2 pi k / n_axis), k < n_axis; G_FIELD: D*N field
  // thermal wall, side s = 0 (low) / 1 (high): fw = f0_i(1, 0, T_s), fwd = fw - w,
  // wallA = -sum over one column's incoming slots of fwd, wall_inv_den = 1 / sum of fw
  double fw[2][QMAX];
  double fwd[2][QMAX];
  double wallA[2];
  double wall_inv_den[2];
  float h_scale;      // FP16 codec scale s and 1/s
  float h_inv_scale;
  // FP16 codec factors per direction, float(w_i) / s and float(1 / w_i) s
  // (set_fp16_factors): a decode or encode is then one multiply by a kernel
  // parameter instead of two
  float h_dec[QMAX];
  float h_enc[QMAX];
  int* err;           // set to 1 by a kernel whose bounded wait ran out
  double mu;          // > 0: constant dynamic viscosity, 1/omega = mu/(rho theta) + 1/2 per site
  // float copies for the float kernels (no FP64 conversion on their path)
  float omega_f;
  float mu_f;
  float g0_f[3];
  const float* gtab_f;  // float copy of gtab (same layout)
  // solid sites (staircase walls, fully periodic grids): flag per site and
  // wall temperature minus 1 per site (read at solid sites only); nullptr
  // when the grid has none
  const unsigned char* solid;
  const double* wall_th;
  const float* wall_th_f;
  int l2_evict_first;  // 1: population loads are evict-first in L2 (see ld_pop_policy)
  int storage_probe;   // FP64 codec: round stored deviations to P_FP32S / P_FP16S format (0 off)
  // layers of the last axis the per-site kernels visit: a0 .. a0 + na - 1
  // (the whole axis, a0 = 0 and na = n_axis, except on a slab context, whose
  // buffer also holds the ghost layers of its neighbours)
  int a0, na;
};

// The parameters a kernel of arithmetic type R reads.
template <class R>
struct ParamsOf;
template <>
struct ParamsOf<double> {
  __device__ __forceinline__ static double wall_th(const StepParams& p, int k) { return __ldg(p.wall_th + k); }
  __device__ __forceinline__ static double omega(const StepParams& p) { return p.omega; }
  __device__ __forceinline__ static double mu(const StepParams& p) { return p.mu; }
  __device__ __forceinline__ static double g0(const StepParams& p, int a) { return p.g0[a]; }
  __device__ __forceinline__ static double gtab(const StepParams& p, size_t k) { return __ldg(p.gtab + k); }
};
template <>
struct ParamsOf<float> {
  __device__ __forceinline__ static float wall_th(const StepParams& p, int k) { return __ldg(p.wall_th_f + k); }
  __device__ __forceinline__ static float omega(const StepParams& p) { return p.omega_f; }
  __device__ __forceinline__ static float mu(const StepParams& p) { return p.mu_f; }
  __device__ __forceinline__ static float g0(const StepParams& p, int a) { return p.g0_f[a]; }
  __device__ __forceinline__ static float gtab(const StepParams& p, size_t k) { return __ldg(p.gtab_f + k); }
};

template <>
struct ParamsOf<DF> {
  __device__ __forceinline__ static DF wall_th(const StepParams& p, int k) { return df_split(__ldg(p.wall_th + k)); }
  __device__ __forceinline__ static DF omega(const StepParams& p) { return df_split(p.omega); }
  __device__ __forceinline__ static DF mu(const StepParams& p) { return df_split(p.mu); }
  __device__ __forceinline__ static DF g0(const StepParams& p, int a) { return df_split(p.g0[a]); }
  __device__ __forceinline__ static DF gtab(const StepParams& p, size_t k) { return df_split(__ldg(p.gtab + k)); }
};

// ---------------------------------------------------------------- helpers
// Compile-time index usable in device code (std::integral_constant's
// conversion operator is host-only).
template <int V>
struct ic {
  static constexpr int value = V;
  __host__ __device__ constexpr operator int() const { return V; }
};

template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(ic<B>{});
    static_for<B + 1, E>(f);
  }
}

// acc + K * v for a compile-time integer K, without a multiply for K in {0, +-1}.
template <int K, class R>
__device__ __forceinline__ R mac(R v, R acc) {
  if constexpr (K == 0) return acc;
  else if constexpr (K == 1) return acc + v;
  else if constexpr (K == -1) return acc - v;
  else return fma(R(K), v, acc);
}

// K * v for a compile-time integer K.
template <int K, class R>
__device__ __forceinline__ R imul(R v) {
  if constexpr (K == 0) return R(0);
  else if constexpr (K == 1) return v;
  else if constexpr (K == -1) return -v;
  else return R(K) * v;
}

// Relaxation rate 1/tau-hat at a site: the grid's constant, or with constant
// dynamic viscosity mu (the paper's validation runs set tau = mu/(rho theta))
// 1 / (mu / (rho theta) + 1/2) from the mid-point rho and theta.
template <class R>
struct ParamsOf;
template <class R>
__device__ __forceinline__ R site_omega(const StepParams& p, R rho, R theta) {
  const R mu = ParamsOf<R>::mu(p);
  if (mu > R(0)) return R(1) / (mu / (rho * theta) + R(0.5));
  return ParamsOf<R>::omega(p);
}

// Products by the quadrature constants (w_i, c, c^2, |xi|^2).  In float the
// constant is carried as hi + lo (both floats, ~48 bits): a float-rounded
// constant would break the identities sum w = 1, c^2 sum w e e = delta by
// ~1e-7 and the collision would then create momentum and energy at that
// relative rate every step.  In double the constant is used as is.
struct F2 {
  float hi, lo;
};
__host__ __device__ constexpr F2 f2_of(double k) {
  return F2{float(k), float(k - double(float(k)))};
}
// EX = false (FP16 storage, whose rounding of ~5e-4 dwarfs the ~1e-8 a
// float-rounded constant costs): one float multiply instead of two.
template <class R, bool EX = true>
__device__ __forceinline__ R kmul(double k, F2 k2, R x) {
  if constexpr (std::is_same<R, DF>::value) return DF(k2.hi, k2.lo) * x;  // the constant's float-float split
  else if constexpr (sizeof(R) == sizeof(double)) return R(k) * x;
  else if constexpr (EX) return fmaf(k2.hi, x, k2.lo * x);
  else return k2.hi * x;
}
template <class L, int I, class R, bool EX = true>
__device__ __forceinline__ R mul_w(R x) {
  constexpr double k = L::W(I);
  constexpr F2 k2 = f2_of(k);
  return kmul<R, EX>(k, k2, x);
}
template <class L, class R, bool EX = true>
__device__ __forceinline__ R mul_c(R x) {
  constexpr F2 k2 = f2_of(L::c);
  return kmul<R, EX>(L::c, k2, x);
}
template <class L, class R, bool EX = true>
__device__ __forceinline__ R mul_c2(R x) {
  constexpr F2 k2 = f2_of(L::c2);
  return kmul<R, EX>(L::c2, k2, x);
}

// e_i . v for compile-time e_i.
template <class L, int I, class R>
__device__ __forceinline__ R edot(const R (&v)[3]) {
  constexpr int ex = L::E(I, 0), ey = L::E(I, 1), ez = L::E(I, 2);
  R acc = imul<ex>(v[0]);
  acc = mac<ey>(v[1], acc);
  if constexpr (L::D == 3) acc = mac<ez>(v[2], acc);
  return acc;
}

// ------------------------------------------- population cache policies
// A step reads each stored population once and the next step reads what
// this one writes.  With loads marked evict-first in L2
// (StepParams::l2_evict_first) the lines just read leave L2 before the lines
// just written.  In one A/B on one GB300 the 1024 x 512 D2Q37 step
// (2 x 77.6 MB in FP32, L2 129 MB) went from 25.2 to 22.5 us in FP32 and
// from 20.3 to 19.5 us in FP16 when launched back to back; serialised
// launches under a profiler showed no gain (the same DRAM reads, fewer
// writes inside the launch), so the benefit comes from how consecutive steps
// share L2 and DRAM.  On working sets of twice L2 and more the hint cost
// 4-8 %, so the host sets the flag only below 1.5 times the L2 size.  The
// results are bit-identical either way.
template <class T>
__device__ __forceinline__ T ld_pop_policy(const T* ptr, bool evict_first) {
  unsigned long long first, normal;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(first));
  asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(normal));
  const unsigned long long pol = evict_first ? first : normal;
  // volatile, like the read-only-path intrinsics: the load stays after the
  // griddepcontrol.wait of a programmatic dependent launch
  if constexpr (sizeof(T) == 4) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(ptr), "l"(pol));
    return v;
  } else {
    static_assert(sizeof(T) == 2, "16- or 32-bit populations");
    unsigned short v;
    asm volatile("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(v) : "l"(ptr), "l"(pol));
    return __ushort_as_half(v);
  }
}

// ------------------------------------------------------- storage codecs
// decode(stored, i) -> deviation d_i = f_i - w_i ; encode(d_i, i) -> stored
template <int P> struct Codec;

template <> struct Codec<P_FP64> {
  using T = double;
  using R = double;
  template <class L, int I>
  __device__ __forceinline__ static R decode(T v, const StepParams&) { return v - L::W(I); }
  template <class L, int I>
  __device__ __forceinline__ static T encode(R d, const StepParams&) { return d + L::W(I); }
  __device__ __forceinline__ static T load(const T* ptr, const StepParams&) { return __ldg(ptr); }
  __device__ __forceinline__ static T load_cg(const T* p) { return __ldcg(p); }
};

// Storage probe of the FP64 codec (StepParams::storage_probe): the deviation
// d rounded as the float codecs store it -- to float (P_FP32S), or to half of
// d / w_i times the grid scale and back through the same float factors as
// Codec<P_FP16S> (P_FP16S).  Exact arithmetic around it.
template <int I>
__device__ __forceinline__ double probe_round(double d, const StepParams& p) {
  if (p.storage_probe == P_FP32S) return double(float(d));
  if (p.storage_probe == P_FP16S)
    return double(__half2float(__float2half_rn(float(d) * p.h_enc[I])) * p.h_dec[I]);
  return d;
}

// FP64 storage, float-float arithmetic: the double is split with integer
// operations and the deviation from w_i taken in float-float; the store adds
// w_i back and rounds to the nearest double (lbm_df.cuh).
template <> struct Codec<P_FP64DF> {
  using T = double;
  using R = DF;
  template <class L, int I>
  __device__ __forceinline__ static R decode(T v, const StepParams&) {
    constexpr DF w = DF(L::W(I));
    return df_split(v) - w;
  }
  template <class L, int I>
  __device__ __forceinline__ static T encode(R d, const StepParams&) {
    constexpr DF w = DF(L::W(I));
    return df_to_double(d + w);
  }
  __device__ __forceinline__ static T load(const T* ptr, const StepParams&) { return __ldg(ptr); }
  __device__ __forceinline__ static T load_cg(const T* p) { return __ldcg(p); }
};

template <> struct Codec<P_FP32S> {
  using T = float;
  using R = float;
  template <class L, int I>
  __device__ __forceinline__ static R decode(T v, const StepParams&) { return v; }
  template <class L, int I>
  __device__ __forceinline__ static T encode(R d, const StepParams&) { return d; }
  __device__ __forceinline__ static T load(const T* ptr, const StepParams& p) {
    return ld_pop_policy(ptr, p.l2_evict_first != 0);
  }
  __device__ __forceinline__ static T load_cg(const T* p) { return __ldcg(p); }
};

template <> struct Codec<P_FP16S> {
  using T = __half;
  using R = float;
  template <class L, int I>
  __device__ __forceinline__ static R decode(T v, const StepParams& p) {
    return __half2float(v) * p.h_dec[I];
  }
  template <class L, int I>
  __device__ __forceinline__ static T encode(R d, const StepParams& p) {
    return __float2half_rn(d * p.h_enc[I]);
  }
  __device__ __forceinline__ static T load(const T* ptr, const StepParams& p) {
    return ld_pop_policy(ptr, p.l2_evict_first != 0);
  }
  __device__ __forceinline__ static T load_cg(const T* p) { return __ldcg(p); }
};

// Working representation of the step kernels.  An FP16-scaled step collides
// the stored value itself, h_i = s (f_i - w_i) / w_i, instead of the deviation
// d_i = w_i h_i / s: Eq. lbm divided by w_i / s reads
//   h*_i = (1 - om) h_i + s [om drho + rho (om p_i + (1 - om/2) F'_i)],
// since the pair weights cancel, so the decode multiply, the weight multiply
// of the equilibrium and the encode multiply of every population drop out;
// s, a power of two, scales the handful of per-site coefficients exactly.
// The sigma-bar force order (FO 3) keeps deviations (its stress tensor is a
// sum over them).
template <int P, int FO>
__host__ __device__ constexpr bool scaled_step() {
  return P == P_FP16S && FO != 3;
}
template <class L, int P, int I, bool SC>
__device__ __forceinline__ typename Codec<P>::R step_in(typename Codec<P>::T v, const StepParams& p) {
  if constexpr (SC) return __half2float(v);
  else return Codec<P>::template decode<L, I>(v, p);
}
// a deviation formed in the kernel (a wall slot) in the working representation
template <int I, bool SC, class R>
__device__ __forceinline__ R step_from_dev(R d, const StepParams& p) {
  if constexpr (SC) return d * R(p.h_enc[I]);
  else return d;
}
template <class L, int P, int I, bool SC>
__device__ __forceinline__ typename Codec<P>::T step_out(typename Codec<P>::R x, const StepParams& p) {
  if constexpr (SC) return __float2half_rn(x);
  else return Codec<P>::template encode<L, I>(x, p);
}

// The FP16 factors of a lattice for the scale in p (host side).  Both are
// products of two floats, as the device formed them before they became
// parameters, so the stored values are unchanged.
template <class L>
inline void set_fp16_factors(StepParams& p) {
  for (int i = 0; i < QMAX; ++i) p.h_dec[i] = p.h_enc[i] = 0.0f;
  for (int i = 0; i < L::Q; ++i) {
    p.h_dec[i] = float(L::w[i]) * p.h_inv_scale;
    p.h_enc[i] = float(1.0 / L::w[i]) * p.h_scale;
  }
}

// Load modes of a population pull: LD_HINT the codec's load (float codecs:
// the L2 policy of StepParams::l2_evict_first), LD_RO the plain read-only
// path (for kernels at their register cap: the policy costs two registers),
// LD_CG from L2 only (for a kernel that reads what other blocks of the same
// launch wrote: the read-only and L1 paths may hold stale lines).
enum { LD_HINT = 0, LD_RO = 1, LD_CG = 2 };
template <class C, int LD>
__device__ __forceinline__ typename C::T ldpop(const typename C::T* ptr, const StepParams& p) {
  if constexpr (LD == LD_CG) return C::load_cg(ptr);
  else if constexpr (LD == LD_RO) return __ldg(ptr);
  else return C::load(ptr, p);
}

// ------------------------------------------------------------ body force
template <class R>
__device__ __forceinline__ void body_force(const StepParams& p, int x, int y, int z, int site,
                                           R (&g)[3]) {
  if (p.gkind == G_UNIFORM) {
    g[0] = R(p.g0[0]); g[1] = R(p.g0[1]); g[2] = R(p.g0[2]);
  } else if (p.gkind == G_SINE) {
    const int k = p.gaxis == 0 ? x : (p.gaxis == 1 ? y : z);
    const double s = __ldg(p.gtab + k);
    g[0] = R(p.g0[0] * s); g[1] = R(p.g0[1] * s); g[2] = R(p.g0[2] * s);
  } else {
    g[0] = R(__ldg(p.gtab + site));
    g[1] = R(__ldg(p.gtab + (size_t)p.N + site));
    g[2] = p.nz > 1 ? R(__ldg(p.gtab + 2 * (size_t)p.N + site)) : R(0);
  }
}

// --------------------------------------------------------- mid-point state
// Moments of the pulled f~ (Eq. rut1) and the mid-point state of Eq. lbm:
// rho, u = u~ + g/2 and the physical temperature
// theta = (sum f~ xi^2 / rho - |u~|^2) / D + |g|^2 / (4 D).
// Per shell (|xi|^2 = X2) it also prepares the coefficients of the
// equilibrium polynomial p(t) = f0_i/(w_i rho) - 1 in t = xi_i . u:
//   p = A0 + A1 t + A2 t^2 + t^3/6 + [NEQ = 4] t^4/24, with
//   A0 = -u^2/2 + Th (X2 - D)/2
//        + [NEQ=4] (3 u^4 - 6 Th u^2 (X2-D-2) + 3 Th^2 (X2^2 - 2(D+2) X2 + D(D+2)))/24
//   A1 = 1 - u^2/2 + Th (X2 - D - 2)/2
//   A2 = 1/2 + [NEQ=4] (-u^2 + Th (X2 - D - 4))/4,        Th = theta - 1,
// i.e. sum_n a^(n)_0 : H^(n)(xi) / n! of Eq. fN with the Maxwellian
// coefficients (Eq. f2 and its higher-order analogues) written out in t.
// The force polynomial F_i/(w_i rho) (Eq. fi without sigma terms) is, with
// s = xi_i . g and Z = -u^2 + Th (X2 - D - 2):
//   order 0: s;  order 1: s (1 + t) - g.u;
//   order 2: s (1 + t + (t^2 + Z)/2) - g.u (1 + t)     (A1 = 1 + Z/2)
template <class L, class R>
struct MidState {
  static constexpr int NS = L::NSHELL;
  R drho, rho, u[3], theta_m1, u2, gu, cu[3], cg[3];
  R A0[NS], A1[NS], A2[NS];
};

template <class L, class R>
__device__ __forceinline__ void prepare_shells(MidState<L, R>& m) {
  constexpr int D = L::D;
  const R Th = m.theta_m1, u2 = m.u2;
  static_for<0, L::NSHELL>([&](auto S) {
    constexpr int s = S;
    constexpr double X2d = L::c2 * double(L::E2(s));
    constexpr F2 X2f = f2_of(X2d);
    const R ThX2 = kmul<R>(X2d, X2f, Th);  // Th * |xi|^2, constant carried as hi + lo
    R a0 = R(-0.5) * u2 + R(0.5) * (ThX2 - R(D) * Th);
    R a1 = R(1) - R(0.5) * u2 + R(0.5) * (ThX2 - R(D + 2) * Th);
    R a2 = R(0.5);
    if constexpr (L::NEQ >= 4) {
      constexpr double q2 = X2d * X2d - 2.0 * (D + 2) * X2d + double(D * (D + 2));
      constexpr F2 q2f = f2_of(q2);
      a0 += R(1.0 / 24.0) * (R(3) * u2 * u2 - R(6) * u2 * (ThX2 - R(D + 2) * Th) +
                             R(3) * Th * kmul<R>(q2, q2f, Th));
      a2 += R(0.25) * ((ThX2 - R(D + 4) * Th) - u2);
    }
    m.A0[s] = a0;
    m.A1[s] = a1;
    m.A2[s] = a2;
  });
}

// Raw moments of the deviations: drho = sum d, j = sum e d, k2 = sum |e|^2 d
// (so rho = 1 + drho, sum f xi = c j, sum f xi^2 = D + c^2 k2), summed per
// opposite pair.
template <class L, class R>
struct RawMoments {
  R drho, j[3], k2;
};

template <class L, class R>
__device__ __forceinline__ RawMoments<L, R> raw_moments(const R (&d)[L::Q]) {
  constexpr int Q = L::Q, D = L::D, NP = (Q - 1) / 2;
  RawMoments<L, R> r;
  R drho = d[0], j0 = R(0), j1 = R(0), j2 = R(0), k2 = R(0);
  static_for<0, NP>([&](auto K) {
    constexpr int ip = 2 * K + 1, im = ip + 1;
    constexpr int ex = L::E(ip, 0), ey = L::E(ip, 1), ez = L::E(ip, 2);
    constexpr int e2 = ex * ex + ey * ey + ez * ez;
    const R s = d[ip] + d[im];
    const R a = d[ip] - d[im];
    drho += s;
    j0 = mac<ex>(a, j0);
    j1 = mac<ey>(a, j1);
    if constexpr (D == 3) j2 = mac<ez>(a, j2);
    k2 = mac<e2>(s, k2);
  });
  r.drho = drho;
  r.j[0] = j0; r.j[1] = j1; r.j[2] = j2;
  r.k2 = k2;
  return r;
}

// The same sums from the scaled values h_i = s d_i / w_i of an FP16-scaled
// step: each pair is weighted by its common w_i, and 1/s (a power of two)
// applied once to each sum.
template <class L, class R>
__device__ __forceinline__ RawMoments<L, R> raw_moments_scaled(const R (&h)[L::Q], R inv_s) {
  constexpr int Q = L::Q, D = L::D, NP = (Q - 1) / 2;
  RawMoments<L, R> r;
  R drho = h[0] * R(float(L::W(0))), j0 = R(0), j1 = R(0), j2 = R(0), k2 = R(0);
  static_for<0, NP>([&](auto K) {
    constexpr int ip = 2 * K + 1, im = ip + 1;
    constexpr int ex = L::E(ip, 0), ey = L::E(ip, 1), ez = L::E(ip, 2);
    constexpr int e2 = ex * ex + ey * ey + ez * ez;
    constexpr double w = L::W(ip);
    const R s = h[ip] + h[im];
    const R a = h[ip] - h[im];
    drho = fma(s, R(float(w)), drho);
    if constexpr (ex != 0) j0 = fma(a, R(float(ex * w)), j0);
    if constexpr (ey != 0) j1 = fma(a, R(float(ey * w)), j1);
    if constexpr (D == 3 && ez != 0) j2 = fma(a, R(float(ez * w)), j2);
    k2 = fma(s, R(float(e2 * w)), k2);
  });
  r.drho = drho * inv_s;
  r.j[0] = j0 * inv_s; r.j[1] = j1 * inv_s; r.j[2] = j2 * inv_s;
  r.k2 = k2 * inv_s;
  return r;
}

// From the deviations of the pulled distribution.
template <class L, class R>
__device__ __forceinline__ void midpoint_state(const R (&d)[L::Q], const R (&g)[3], MidState<L, R>& m) {
  constexpr int D = L::D;
  const RawMoments<L, R> r = raw_moments<L, R>(d);
  const R drho = r.drho;
  const R rho = R(1) + drho;
  const R irho = R(1) / rho;
  const R ut0 = mul_c<L, R>(r.j[0] * irho), ut1 = mul_c<L, R>(r.j[1] * irho),
          ut2 = mul_c<L, R>(r.j[2] * irho);
  const R ut_sq = ut0 * ut0 + ut1 * ut1 + ut2 * ut2;
  const R g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  m.drho = drho;
  m.rho = rho;
  m.u[0] = ut0 + R(0.5) * g[0];
  m.u[1] = ut1 + R(0.5) * g[1];
  m.u[2] = ut2 + R(0.5) * g[2];
  m.theta_m1 = ((mul_c2<L, R>(r.k2) - R(D) * drho) * irho - ut_sq) * R(1.0 / D) + g2 * R(0.25 / D);
  m.u2 = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
  m.gu = g[0] * m.u[0] + g[1] * m.u[1] + g[2] * m.u[2];
  for (int a = 0; a < 3; ++a) {
    m.cu[a] = mul_c<L, R>(m.u[a]);
    m.cg[a] = mul_c<L, R>(g[a]);
  }
  prepare_shells<L, R>(m);
}

// From given physical fields (initialisation): drho = rho - 1 and
// theta_m1 = T - 1 are formed in double by the caller, so that the small
// deviations keep their precision when R is float.
template <class L, class R>
__device__ __forceinline__ void given_state(R drho, const R (&u)[3], R theta_m1, const R (&g)[3],
                                            MidState<L, R>& m) {
  m.drho = drho;
  m.rho = R(1) + drho;
  m.theta_m1 = theta_m1;
  for (int a = 0; a < 3; ++a) {
    m.u[a] = u[a];
    m.cu[a] = mul_c<L, R>(u[a]);
    m.cg[a] = mul_c<L, R>(g[a]);
  }
  m.u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  m.gu = g[0] * u[0] + g[1] * u[1] + g[2] * u[2];
  prepare_shells<L, R>(m);
}

// Equilibrium and force polynomials for the pair (e, -e) of direction IP:
// p(+-) = E +- O, F'(+-) = Fe +- Fo  (F' = F/(w rho)).
template <class L, int FO, int IP, class R>
__device__ __forceinline__ void pair_terms(const MidState<L, R>& m, R& E, R& O, R& Fe, R& Fo) {
  constexpr int s = L::SH(IP);
  const R t = edot<L, IP>(m.cu);
  const R tg = edot<L, IP>(m.cg);
  const R t2 = t * t;
  if constexpr (L::NEQ >= 4) {
    E = fma(t2, fma(t2, R(1.0 / 24.0), m.A2[s]), m.A0[s]);
  } else {
    E = fma(t2, m.A2[s], m.A0[s]);
  }
  O = t * fma(t2, R(1.0 / 6.0), m.A1[s]);
  if constexpr (FO == 0) {
    Fe = R(0);
    Fo = tg;
  } else if constexpr (FO == 1) {
    Fe = fma(tg, t, -m.gu);
    Fo = tg;
  } else {
    Fe = fma(tg, t, -m.gu);
    Fo = fma(tg, fma(R(0.5), t2, m.A1[s]), -m.gu * t);
  }
}

// Rest particle: t = s = 0.
template <class L, int FO, class R>
__device__ __forceinline__ void rest_terms(const MidState<L, R>& m, R& E, R& Fe) {
  E = m.A0[0];
  Fe = FO >= 1 ? -m.gu : R(0);
}

// ------------------------------------------- sigma-bar terms (force order 2)
// Keeping the deviatoric stress in the second Hermite coefficient of the
// force, a^(2) = a^(2)_0 - sigma-bar (Eq. f2), adds to the n = 3 term of
// Eq. F (w_i / 2 times g a^(2) : H^(3)) the odd part
//   -(w_i / 2) [(g.xi)(xi.sigma.xi - tr sigma) - 2 g.sigma.xi],
// sigma-bar = -(1 - om/2) S (the reading of Eq. sigma used throughout) with
//   S = sum_i f~_i (xi_i - u)(xi_i - u) - rho theta delta
//     = c^2 P - (drho + rho Th) delta - rho u u + rho (u g + g u) / 2,
// P_ab = sum_i d_i e_ia e_ib over the deviations (sum_i w_i xi xi = delta),
// u the mid-point velocity, u~ = u - g/2.  tr S vanishes identically because
// theta is taken from the same f~, so the trace term is dropped.
// S is stored as (xx, yy, zz, xy, xz, yz); in 2-D the z entries are zero.
template <class L, class R>
__device__ __forceinline__ void stress_tensor(const R (&d)[L::Q], R drho, R rho, R Th,
                                              const R (&u)[3], const R (&g)[3], R (&S)[6]) {
  constexpr int NP = (L::Q - 1) / 2;
  R P0 = R(0), P1 = R(0), P2 = R(0), P3 = R(0), P4 = R(0), P5 = R(0);
  static_for<0, NP>([&](auto K) {
    constexpr int ip = 2 * K + 1, im = ip + 1;
    constexpr int ex = L::E(ip, 0), ey = L::E(ip, 1), ez = L::E(ip, 2);
    const R s = d[ip] + d[im];
    P0 = mac<ex * ex>(s, P0);
    P1 = mac<ey * ey>(s, P1);
    P3 = mac<ex * ey>(s, P3);
    if constexpr (L::D == 3) {
      P2 = mac<ez * ez>(s, P2);
      P4 = mac<ex * ez>(s, P4);
      P5 = mac<ey * ez>(s, P5);
    }
  });
  const R iso = fma(rho, Th, drho);
  const R hr = R(0.5) * rho;
  // -rho u_a u_b + rho (u_a g_b + g_a u_b) / 2
  auto conv = [&](int a, int b) { return hr * (u[a] * (g[b] - u[b]) + u[b] * (g[a] - u[a])); };
  S[0] = mul_c2<L, R>(P0) - iso + conv(0, 0);
  S[1] = mul_c2<L, R>(P1) - iso + conv(1, 1);
  S[3] = mul_c2<L, R>(P3) + conv(0, 1);
  if constexpr (L::D == 3) {
    S[2] = mul_c2<L, R>(P2) - iso + conv(2, 2);
    S[4] = mul_c2<L, R>(P4) + conv(0, 2);
    S[5] = mul_c2<L, R>(P5) + conv(1, 2);
  } else {
    S[2] = S[4] = S[5] = R(0);
  }
}

// Per-site factors of the odd term k [(g.xi)(xi.S.xi) - 2 (S g).xi] in
// lattice vectors: gs = k c^3 g, hs = 2 k c S g.
template <class R>
struct StressTerms {
  R gs[3], S[6], hs[3];
};

template <class L, class R>
__device__ __forceinline__ StressTerms<R> stress_terms(const R (&S)[6], const R (&g)[3], R k) {
  StressTerms<R> st;
  const R kc3 = k * R(L::c * L::c2), kc2 = R(2) * k * R(L::c);
  const R Sg0 = S[0] * g[0] + S[3] * g[1] + S[4] * g[2];
  const R Sg1 = S[3] * g[0] + S[1] * g[1] + S[5] * g[2];
  const R Sg2 = S[4] * g[0] + S[5] * g[1] + S[2] * g[2];
  st.gs[0] = kc3 * g[0]; st.gs[1] = kc3 * g[1]; st.gs[2] = kc3 * g[2];
  st.hs[0] = kc2 * Sg0; st.hs[1] = kc2 * Sg1; st.hs[2] = kc2 * Sg2;
  for (int a = 0; a < 6; ++a) st.S[a] = S[a];
  return st;
}

// The odd stress term of the pair (e, -e) of direction IP (value for +e).
template <class L, int IP, class R>
__device__ __forceinline__ R stress_pair(const StressTerms<R>& st) {
  constexpr int ex = L::E(IP, 0), ey = L::E(IP, 1), ez = L::E(IP, 2);
  R eSe = imul<ex * ex>(st.S[0]);
  eSe = mac<ey * ey>(st.S[1], eSe);
  eSe = mac<2 * ex * ey>(st.S[3], eSe);
  if constexpr (L::D == 3) {
    eSe = mac<ez * ez>(st.S[2], eSe);
    eSe = mac<2 * ex * ez>(st.S[4], eSe);
    eSe = mac<2 * ey * ez>(st.S[5], eSe);
  }
  return fma(edot<L, IP>(st.gs), eSe, -edot<L, IP>(st.hs));
}

}  // namespace lbm
