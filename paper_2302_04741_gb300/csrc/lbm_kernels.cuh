// lbm_kernels.cuh -- the kernels of one lattice, included by one .cu per lattice.
//
// Storage: structure of arrays, population i of site s at f[i*N + s], sites
// row-major [nz][ny][nx] with x fastest; two buffers (ping-pong).  The stored
// buffer holds the post-collision distribution f*; a step pulls
// f~_i(x) = f*_i(x - e_i), collides (Eq. lbm) and stores f*_i(x) coalesced.
//
// Launch shape of the per-site kernels: blockDim = (bx, 1, 1) along x,
// grid = (ceil(nx / bx), ny, nz): every block works on one row, so the
// near-wall branch is uniform across a block.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

template <int I>
__host__ __device__ constexpr int opposite() {
  return I == 0 ? 0 : ((I & 1) ? I + 1 : I - 1);
}

__device__ __forceinline__ int wrap3(int v, int n) {
  v += v < 0 ? n : 0;
  v -= v >= n ? n : 0;
  return v;
}

template <int D>
__device__ __forceinline__ void site_force(const StepParams& p, int x, int y, int z, int site,
                                           double (&g)[3]) {
  if (p.gkind == G_UNIFORM) {
    g[0] = p.g0[0]; g[1] = p.g0[1]; g[2] = p.g0[2];
  } else if (p.gkind == G_SINE) {
    const int k = p.gaxis == 0 ? x : (p.gaxis == 1 ? y : z);
    const double s = __ldg(p.gtab + k);
    g[0] = p.g0[0] * s; g[1] = p.g0[1] * s; g[2] = p.g0[2] * s;
  } else {
    g[0] = __ldg(p.gtab + site);
    g[1] = __ldg(p.gtab + (size_t)p.N + site);
    g[2] = D == 3 ? __ldg(p.gtab + 2 * (size_t)p.N + site) : 0.0;
  }
  if (D == 2) g[2] = 0.0;
}

// g(x) in the arithmetic type of the kernel (float kernels read float copies).
template <int D, class R>
__device__ __forceinline__ void site_force_r(const StepParams& p, int x, int y, int z, int site,
                                             R (&g)[3]) {
  using PP = ParamsOf<R>;
  if (p.gkind == G_UNIFORM) {
    g[0] = PP::g0(p, 0); g[1] = PP::g0(p, 1); g[2] = PP::g0(p, 2);
  } else if (p.gkind == G_SINE) {
    const int k = p.gaxis == 0 ? x : (p.gaxis == 1 ? y : z);
    const R s = PP::gtab(p, k);
    g[0] = PP::g0(p, 0) * s; g[1] = PP::g0(p, 1) * s; g[2] = PP::g0(p, 2) * s;
  } else {
    g[0] = PP::gtab(p, site);
    g[1] = PP::gtab(p, (size_t)p.N + site);
    g[2] = D == 3 ? PP::gtab(p, 2 * (size_t)p.N + site) : R(0);
  }
  if (D == 2) g[2] = R(0);
}

// Pull of all Q populations of site (x, y, z) with the boundary rules, decoded
// to deviations in type RR (SC: the scaled values of an FP16-scaled step, see
// scaled_step).  The wall axis is the last axis (y in 2-D, z in 3-D).
template <class L, int P, class RR, int LD = LD_HINT, bool SC = false>
__device__ __forceinline__ void pull(const typename Codec<P>::T* __restrict__ fin,
                                     const StepParams& p, int x, int y, int z, RR (&d)[L::Q]) {
  using C = Codec<P>;
  constexpr int D = L::D, Q = L::Q;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const size_t N = (size_t)p.N;
  const int a = D == 2 ? y : z;          // coordinate along the wall axis
  const int nA = D == 2 ? ny : nz;
  int xs[7], ys[7], zs[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    xs[k] = wrap3(x - (k - 3), nx);
    ys[k] = wrap3(y - (k - 3), ny) * nx;
    zs[k] = D == 3 ? wrap3(z - (k - 3), nz) * nx * ny : 0;
  }
  const bool near = p.wall != W_NONE && (a < 3 || a >= nA - 3);
  if (!near) {
    static_for<0, Q>([&](auto I) {
      constexpr int i = I;
      constexpr int ex = L::E(i, 0), ey = L::E(i, 1), ez = L::E(i, 2);
      const int off = zs[ez + 3] + ys[ey + 3] + xs[ex + 3];
      d[i] = RR(step_in<L, P, i, SC>(ldpop<C, LD>(fin + i * N + off, p), p));
    });
    return;
  }
  // ---- a row next to a wall: slots whose source lies beyond the wall
  const int side = a < 3 ? 0 : 1;
  const int colbase = D == 2 ? x : (y * nx + x);     // site of the column at wall coord 0
  const int lineA = D == 2 ? nx : nx * ny;           // stride along the wall axis
  RR rm1 = RR(0);                                    // rho_w - 1 of the thermal wall
  if (p.wall == W_THERMAL) {
    RR sum = RR(0);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int row = side == 0 ? r : nA - 1 - r;
      static_for<0, Q>([&](auto J) {
        constexpr int j = J;
        constexpr int eA = L::E(j, D - 1);
        if constexpr (eA != 0) {
          const bool leaves = side == 0 ? (eA < 0 && r + eA < 0) : (eA > 0 && r - eA < 0);
          if (leaves)
            sum += RR(C::template decode<L, j>(ldpop<C, LD>(fin + j * N + colbase + row * lineA, p), p));
        }
      });
    }
    rm1 = (RR(p.wallA[side]) + sum) * RR(p.wall_inv_den[side]);
  }
  static_for<0, Q>([&](auto I) {
    constexpr int i = I;
    constexpr int ex = L::E(i, 0), ey = L::E(i, 1), ez = L::E(i, 2);
    constexpr int eA = L::E(i, D - 1);
    const int sA = a - eA;
    if (sA >= 0 && sA < nA) {
      const int off = zs[ez + 3] + ys[ey + 3] + xs[ex + 3];
      d[i] = RR(step_in<L, P, i, SC>(ldpop<C, LD>(fin + i * N + off, p), p));
    } else if (p.wall == W_BOUNCE) {
      // d_i = d_io and w_i = w_io: the scaled values agree as well
      constexpr int io = opposite<i>();
      const int mA = side == 0 ? eA - 1 - a : 2 * nA - 1 - sA;
      d[i] = RR(step_in<L, P, io, SC>(ldpop<C, LD>(fin + io * N + colbase + mA * lineA, p), p));
    } else {
      d[i] = step_from_dev<i, SC>(fma(rm1, RR(p.fw[side][i]), RR(p.fwd[side][i])), p);
    }
  });
}

// ------------------------------------------------------- solid sites
// A solid site y emits into a fluid neighbour x = y + e_i the wall
// Maxwellian rho_w(x) f0_i(1, 0, T_y) (diffuse thermal wall on a staircase):
// f0_i(1, 0, T) / w_i = 1 + A0 with, for |xi_i|^2 = X2 and Th = T - 1,
//   A0 = Th (X2 - D) / 2 + [NEQ 4] Th^2 (X2^2 - 2 (D + 2) X2 + D (D + 2)) / 8.
// rho_w(x) equals the mass x sends into solid sites (its post-collision slots
// -e_i of the solid-sourced directions) over sum_i f0_i(1, 0, T_y), so every
// fluid site keeps its mass.  In deviations:
//   rho_w - 1 = sum (d*_-i - w_i A0_i) / sum w_i (1 + A0_i),
//   d_i = w_i ((rho_w - 1)(1 + A0_i) + A0_i).
template <class L, int I, class R>
__device__ __forceinline__ R wall_a0(R th) {
  constexpr int D = L::D;
  constexpr double X2 = L::c2 * double(L::E2(L::SH(I)));
  R a0 = R(0.5 * (X2 - D)) * th;
  if constexpr (L::NEQ >= 4) {
    constexpr double q2 = (X2 * X2 - 2.0 * (D + 2) * X2 + double(D * (D + 2))) / 8.0;
    a0 = fma(R(q2) * th, th, a0);
  }
  return a0;
}

// Pull of a fluid site of a grid with solid sites (all axes periodic).
template <class L, int P, class RR>
__device__ __forceinline__ void pull_solid(const typename Codec<P>::T* __restrict__ fin,
                                           const StepParams& p, int x, int y, int z, int site,
                                           RR (&d)[L::Q]) {
  using C = Codec<P>;
  constexpr int D = L::D, Q = L::Q;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const size_t N = (size_t)p.N;
  int xs[7], ys[7], zs[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    xs[k] = wrap3(x - (k - 3), nx);
    ys[k] = wrap3(y - (k - 3), ny) * nx;
    zs[k] = D == 3 ? wrap3(z - (k - 3), nz) * nx * ny : 0;
  }
  RR num = RR(0), den = RR(0);
  unsigned long long walls = 0;
  static_for<0, Q>([&](auto I) {
    constexpr int i = I;
    constexpr int ex = L::E(i, 0), ey = L::E(i, 1), ez = L::E(i, 2);
    const int src = zs[ez + 3] + ys[ey + 3] + xs[ex + 3];
    if (__ldg(p.solid + src)) {
      constexpr int io = opposite<i>();
      constexpr RR w = RR(L::W(i));
      const RR a0 = wall_a0<L, i, RR>(ParamsOf<RR>::wall_th(p, src));
      num += RR(C::template decode<L, io>(C::load(fin + io * N + site, p), p)) - w * a0;
      den = fma(w, RR(1) + a0, den);
      walls |= 1ull << i;
      d[i] = a0;  // kept for the second pass
    } else {
      d[i] = RR(C::template decode<L, i>(C::load(fin + i * N + src, p), p));
    }
  });
  if (!walls) return;
  const RR rm1 = num / den;
  static_for<0, Q>([&](auto I) {
    constexpr int i = I;
    if (walls >> i & 1ull) d[i] = RR(L::W(i)) * fma(rm1, RR(1) + d[i], d[i]);
  });
}

// Pull for a warp whose 32 sites neither wrap around x nor touch a wall: every
// source offset relative to the thread's own site, i*N + (row / plane shift)
// - e_ix, is the same for the whole block (rows wrap only through the block's
// y, z), so addresses are a per-thread base plus block-uniform offsets.
template <class L, int P, class RR, int LD = LD_HINT, bool SC = false>
__device__ __forceinline__ void pull_interior(const typename Codec<P>::T* __restrict__ fsite,
                                              const StepParams& p, int y, int z,
                                              RR (&d)[L::Q]) {
  using C = Codec<P>;
  constexpr int D = L::D, Q = L::Q;
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
    d[i] = RR(step_in<L, P, i, SC>(ldpop<C, LD>(fsite + off, p), p));
  });
}

// ------------------------------------------ float-float step: pair body
// The float-float FP64 step executes ~9,700 instructions per site, almost
// all of it straight-line code: unrolled over the direction pairs it
// exceeds the instruction cache many times over, and instruction fetch
// became its top stall.  Its pair body therefore runs out of line, one
// copy for all pairs, with the pair's directions passed at run time and
// the site's values in one struct (the arithmetic is the inlined body's,
// operation for operation, so the results are the same bits): 1.3x faster
// on GB300.
struct DFSite {
  DF cu[3], cs[3], hom1, P4, Q3;
};
struct DFPair {
  DF p, m;
};
// k * v and acc + k * v for a small run-time integer k, as imul / mac do
// for a compile-time one
__device__ __forceinline__ DF df_imul(int k, DF v) {
  return k == 0 ? DF() : (k == 1 ? v : (k == -1 ? -v : DF(k) * v));
}
__device__ __forceinline__ DF df_mac(int k, DF v, DF acc) {
  return k == 0 ? acc : (k == 1 ? acc + v : (k == -1 ? acc - v : fma(DF(k), v, acc)));
}
template <int D, int FO, bool NEQ4>
__device__ __noinline__ DFPair df_pair(DF dp, DF dm, int ex, int ey, int ez, DF P0, DF P2, DF Q1, DF A1, DF w,
                                       const DFSite& S) {
  DF t = df_imul(ex, S.cu[0]);
  t = df_mac(ey, S.cu[1], t);
  if (D == 3) t = df_mac(ez, S.cu[2], t);
  DF sp = df_imul(ex, S.cs[0]);
  sp = df_mac(ey, S.cs[1], sp);
  if (D == 3) sp = df_mac(ez, S.cs[2], sp);
  const DF t2 = t * t;
  DF ev_in = fma(t2, NEQ4 ? fma(t2, S.P4, P2) : P2, P0);
  DF od_in = t * fma(t2, S.Q3, Q1);
  if (FO >= 1) {
    ev_in = fma(sp, t, ev_in);
    od_in = FO >= 2 ? fma(sp, fma(DF(0.5), t2, A1), od_in) : od_in + sp;
  } else {
    od_in = od_in + sp;
  }
  const DF ev = fma(dp + dm, S.hom1, w * ev_in);
  const DF od = fma(dp - dm, S.hom1, w * od_in);
  return DFPair{ev + od, ev - od};
}

// ------------------------------------------------------------ the step
// Collision of one site from its pulled deviations d (Eq. lbm) and store of
// f*(x) at `site`; shared by the plain and the TMA-staged step kernels.
//
// f*_i - w_i = d_i (1 - om) + w_i [om drho + rho (om p_i + (1 - om/2) F'_i)],
// with p_i = E +- O the equilibrium polynomial and F'_i = Fe +- Fo the force
// polynomial of the pair (e, -e) (see MidState).  rho om and rho (1 - om/2)
// are folded into per-shell coefficients:
//   even: P0 + t^2 (P2 + t^2 rho om / 24) + s' t,   P0 = rho om A0 + om drho - rho k g.u,
//   odd:  t (Q1 + t^2 rho om / 6) + s' (A1 + t^2 / 2),  Q1 = rho om A1 - rho k g.u
//   (order 1: odd force part is s' alone and Q1 = rho om A1; order 0 also drops
//   the even force part s' t - g.u),
// with t = xi.u, s' = rho k xi.g, k = 1 - om/2 (force order 2; lower orders
// drop terms).  Each pair is stored as even +- odd: the even part (density,
// temperature) is shared by e and -e, so its rounding cancels in the odd part
// that carries the momentum; only the final rounding of each member remains.
// SC (scaled_step): d holds h_i = s d_i / w_i, and every coefficient that
// multiplies w_i above is carried times s instead (exact: s is a power of two).
template <class L, int P, int FO, bool SC = false>
__device__ __forceinline__ void collide_store(typename Codec<P>::R (&d)[L::Q],
                                              const typename Codec<P>::R (&g)[3], int site,
                                              typename Codec<P>::T* __restrict__ fout,
                                              const StepParams& p) {
  using C = Codec<P>;
  using R = typename C::R;
  constexpr int NP = (L::Q - 1) / 2, NS = L::NSHELL, D = L::D;
  constexpr bool EX = P != P_FP16S;  // quadrature constants as hi + lo pairs
  static_assert(!SC || scaled_step<P, FO>(), "scaled values: FP16-scaled storage, FO 0..2");
  const size_t N = (size_t)p.N;
  const RawMoments<L, R> r = SC ? raw_moments_scaled<L, R>(d, R(p.h_inv_scale)) : raw_moments<L, R>(d);
  // times s: the coefficients of w_i in the scaled representation
  auto scl = [&](R v) {
    if constexpr (SC) return v * R(p.h_scale);
    else return v;
  };
  // mid-point state (R1): rho, u = u~ + g/2, theta
  const R rho = R(1) + r.drho;
  const R irho = R(1) / rho;
  R u[3];
  for (int a = 0; a < 3; ++a) u[a] = mul_c<L, R, EX>(r.j[a] * irho) + R(0.5) * g[a];
  const R ut0 = u[0] - R(0.5) * g[0], ut1 = u[1] - R(0.5) * g[1], ut2 = u[2] - R(0.5) * g[2];
  const R g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  const R Th = ((mul_c2<L, R, EX>(r.k2) - R(D) * r.drho) * irho - (ut0 * ut0 + ut1 * ut1 + ut2 * ut2)) *
                   R(1.0 / D) + g2 * R(0.25 / D);
  const R u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const R gu = g[0] * u[0] + g[1] * u[1] + g[2] * u[2];
  const R om = site_omega<R>(p, rho, R(1) + Th);
  const R om1 = R(1) - om;
  const R hom1 = R(0.5) * om1;
  const R kf = R(1) - R(0.5) * om;
  const R rom0 = rho * om;
  const R rom = scl(rom0);
  const R rkgu = scl(FO >= 1 ? rho * kf * gu : R(0));
  const R rkf = scl(rho * kf);
  R cu[3], cs[3];
  for (int a = 0; a < 3; ++a) {
    cu[a] = mul_c<L, R, EX>(u[a]);
    cs[a] = mul_c<L, R, EX>(rkf * g[a]);
  }
  // per-shell coefficients as polynomials in tx = Th |xi|^2 (constant hi + lo)
  //   A0 = a00 + tx (c1 + tx / 8 [NEQ 4]),  A1 = b0 + tx / 2,  A2 = g0 + tx / 4 [NEQ 4]
  R a00 = R(-0.5) * u2 - R(0.5 * D) * Th;
  R c1 = R(0.5);
  R g0c = R(0.5);
  if constexpr (L::NEQ >= 4) {
    a00 += R(0.125) * u2 * u2 + R(0.25 * (D + 2)) * Th * u2 + R(0.125 * D * (D + 2)) * Th * Th;
    c1 += R(-0.25) * u2 - R(0.25 * (D + 2)) * Th;
    g0c += R(-0.25) * u2 - R(0.25 * (D + 4)) * Th;
  }
  c1 *= Th;  // A0 = a00 + c1 X2 + Th^2 X2^2 / 8 = a00 + (c1 / Th) tx + tx^2 / 8
  const R b0 = R(1) - R(0.5) * u2 - R(0.5 * (D + 2)) * Th;
  R P0[NS], P2[NS], Q1[NS], A1[NS];
  const R base = scl(om * r.drho) - rkgu;
  // rho om multiplies every direction's equilibrium part at this site, so its
  // rounding would act as a common factor (a coherent momentum / energy error
  // per step): carry it as rom + rom_lo, with the exact FMA residual (in
  // double the product's rounding is far below the tolerances: rom_lo = 0).
  const R rom_lo = sizeof(R) == sizeof(double) ? R(0) : scl(fma(rho, om, -rom0));
  static_for<0, NS>([&](auto S) {
    constexpr int sh = S;
    constexpr double X2d = L::c2 * double(L::E2(sh));
    constexpr F2 X2f = f2_of(X2d);
    const R tx = kmul<R, EX>(X2d, X2f, Th);
    R A0, A2;
    if constexpr (L::NEQ >= 4) {
      A0 = fma(R(0.125) * tx, tx, kmul<R, EX>(X2d, X2f, c1) + a00);
      A2 = fma(R(0.25), tx, g0c);
    } else {
      A0 = fma(R(0.5), tx, a00);
      A2 = g0c;
    }
    A1[sh] = fma(R(0.5), tx, b0);
    P0[sh] = fma(rom, A0, fma(rom_lo, A0, base));
    P2[sh] = fma(rom, A2, rom_lo * A2);
    Q1[sh] = fma(rom, A1[sh], fma(rom_lo, A1[sh], FO >= 2 ? -rkgu : R(0)));
  });
  const R P4 = L::NEQ >= 4 ? rom * R(1.0 / 24.0) : R(0);
  const R Q3 = rom * R(1.0 / 6.0);
  // sigma-bar terms (FO 3 = force order 2 with sigma-bar): the odd part gains
  // rho k dF'_i = (k^2 / 2) [(g.xi)(xi.S.xi) - 2 (S g).xi]
  StressTerms<R> st;
  if constexpr (FO == 3) {
    R S[6];
    stress_tensor<L, R>(d, r.drho, rho, Th, u, g, S);
    st = stress_terms<L, R>(S, g, R(0.5) * kf * kf);
  }
  // rest particle: t = s' = 0
  typename C::T* __restrict__ fo = fout + site;
  // FP64 storage probe: the stored deviation rounded as a float codec stores it
  const bool probe = P == P_FP64 && p.storage_probe != 0;
  {
    R d0 = fma(d[0], om1, SC ? P0[0] : mul_w<L, 0, R, EX>(P0[0]));
    if constexpr (P == P_FP64)
      if (probe) d0 = probe_round<0>(d0, p);
    fo[0] = step_out<L, P, 0, SC>(d0, p);
  }
  constexpr bool DF_OUT_OF_LINE = std::is_same<R, DF>::value && FO <= 2;
  DFSite dfs;
  if constexpr (DF_OUT_OF_LINE) {
    for (int a = 0; a < 3; ++a) {
      dfs.cu[a] = cu[a];
      dfs.cs[a] = cs[a];
    }
    dfs.hom1 = hom1;
    dfs.P4 = P4;
    dfs.Q3 = Q3;
  }
  static_for<0, NP>([&](auto K) {
    constexpr int ip = 2 * K + 1, im = ip + 1;
    constexpr int sh = L::SH(ip);
    if constexpr (DF_OUT_OF_LINE) {
      constexpr F2 wk = f2_of(L::W(ip));
      const DFPair o = df_pair<D, FO, (L::NEQ >= 4)>(d[ip], d[im], L::E(ip, 0), L::E(ip, 1), L::E(ip, 2), P0[sh],
                                                     P2[sh], Q1[sh], A1[sh], DF(wk.hi, wk.lo), dfs);
      fo[ip * N] = step_out<L, P, ip, SC>(o.p, p);
      fo[im * N] = step_out<L, P, im, SC>(o.m, p);
      return;
    }
    const R t = edot<L, ip>(cu);
    const R t2 = t * t;
    R ev_in = fma(t2, L::NEQ >= 4 ? fma(t2, P4, P2[sh]) : P2[sh], P0[sh]);
    R od_in = t * fma(t2, Q3, Q1[sh]);
    if constexpr (FO >= 1) {
      const R sp = edot<L, ip>(cs);
      ev_in = fma(sp, t, ev_in);
      od_in = FO >= 2 ? fma(sp, fma(R(0.5), t2, A1[sh]), od_in) : od_in + sp;
    } else {
      od_in = od_in + edot<L, ip>(cs);
    }
    if constexpr (FO == 3) od_in += stress_pair<L, ip, R>(st);
    const R ev = fma(d[ip] + d[im], hom1, SC ? ev_in : mul_w<L, ip, R, EX>(ev_in));
    const R od = fma(d[ip] - d[im], hom1, SC ? od_in : mul_w<L, ip, R, EX>(od_in));
    R dp = ev + od, dm = ev - od;
    if constexpr (P == P_FP64) {
      if (probe) {
        dp = probe_round<ip>(dp, p);
        dm = probe_round<im>(dm, p);
      }
    }
    fo[ip * N] = step_out<L, P, ip, SC>(dp, p);
    fo[im * N] = step_out<L, P, im, SC>(dm, p);
  });
}

// Resident 256-thread blocks per SM the register cap is sized for: float
// kernels fit 85 registers (3 blocks) -- D2Q37 without spilling, D3Q39 with
// at most 24 B of spill per thread, which measured 7-10 % faster than its
// 128-register, 2-block variant (the batch kernel's two-sites-per-thread
// variants spill more; its tuner measures both); FP64 kernels keep their
// registers.
// LBM_FLOAT_D2Q37_BLOCKS and LBM_FLOAT_D3Q39_BLOCKS override the float values
// at build time (tuning hooks).
#ifndef LBM_FLOAT_D2Q37_BLOCKS
#define LBM_FLOAT_D2Q37_BLOCKS 3
#endif
#ifndef LBM_FLOAT_D3Q39_BLOCKS
#define LBM_FLOAT_D3Q39_BLOCKS 3
#endif
// LBM_DF_BLOCKS: the same for the float-float FP64 step; 2 (128 registers,
// ~240 B of spill) measured 1.45x faster than 1 (255 registers) on GB300:
// the wider kernel hides the instruction-fetch stalls of its long code.
#ifndef LBM_DF_BLOCKS
#define LBM_DF_BLOCKS 2
#endif
// LBM_HALF_D2Q37_BLOCKS, LBM_HALF_D3Q39_BLOCKS: the same for FP16-scaled
// storage (whose 2-byte loads bring half the bytes per load instruction).
#ifndef LBM_HALF_D2Q37_BLOCKS
#define LBM_HALF_D2Q37_BLOCKS LBM_FLOAT_D2Q37_BLOCKS
#endif
#ifndef LBM_HALF_D3Q39_BLOCKS
#define LBM_HALF_D3Q39_BLOCKS LBM_FLOAT_D3Q39_BLOCKS
#endif
template <class L, int P>
constexpr int min_blocks() {
  return P == P_FP64     ? 1
         : P == P_FP64DF ? LBM_DF_BLOCKS
         : P == P_FP16S  ? (L::Q > 37 ? LBM_HALF_D3Q39_BLOCKS : LBM_HALF_D2Q37_BLOCKS)
                         : (L::Q > 37 ? LBM_FLOAT_D3Q39_BLOCKS : LBM_FLOAT_D2Q37_BLOCKS);
}

// Line of the wall axis a block works on.  With walls, the six wall rows
// (whose pull gathers the wall sums and is slower) take the first six block
// indices along that axis, so they start with the first wave instead of
// forming the last blocks of the launch; the bulk rows follow in order.
__device__ __forceinline__ int wall_rows_first(int b, int n, bool walls) {
  if (!walls || n < 6) return b;
  return b < 3 ? b : (b < 6 ? n - 6 + b : b - 3);
}

// SOLID: the grid has solid sites (they are skipped; their fluid neighbours
// take the diffuse-wall pull).
template <class L, int P, int FO, bool SOLID = false>
__global__ void __launch_bounds__(256, min_blocks<L, P>())
    k_step(const typename Codec<P>::T* __restrict__ fin, typename Codec<P>::T* __restrict__ fout,
           const StepParams p) {
  using R = typename Codec<P>::R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const bool walls = p.wall != W_NONE;
  const int y = L::D == 2 ? p.a0 + wall_rows_first(blockIdx.y, p.na, walls) : (int)blockIdx.y;
  const int z = L::D == 3 ? p.a0 + wall_rows_first(blockIdx.z, p.na, walls) : (int)blockIdx.z;
  const int site = (z * p.ny + y) * p.nx + x;
  if constexpr (SOLID) {
    if (__ldg(p.solid + site)) return;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    R g[3];
    site_force_r<L::D, R>(p, x, y, z, site, g);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    R d[L::Q];
    pull_solid<L, P, R>(fin, p, x, y, z, site, d);
    collide_store<L, P, FO>(d, g, site, fout, p);
    return;
  }
  const int a = L::D == 2 ? y : z;
  const int nA = L::D == 2 ? p.ny : p.nz;
  const bool near = p.wall != W_NONE && (a < 3 || a >= nA - 3);
  const int wx0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  const bool interior = !near && wx0 >= 3 && wx0 + 31 <= p.nx - 4;
  // Programmatic dependent launch: let the next step's blocks be scheduled
  // now, and wait for the previous kernel (and its memory) before pulling.
  // Both are no-ops when the launch has no programmatic dependency.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  R g[3];
  site_force_r<L::D, R>(p, x, y, z, site, g);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  constexpr bool SC = scaled_step<P, FO>();
  R d[L::Q];
  if (interior) pull_interior<L, P, R, LD_HINT, SC>(fin + site, p, y, z, d);
  else pull<L, P, R, LD_HINT, SC>(fin, p, x, y, z, d);
  collide_store<L, P, FO, SC>(d, g, site, fout, p);
}

// ------------------------------------------------------------ init
// f~_i = f0_i(rho, u, T) - F_i(rho, u, T)/2 as deviations
// d_i = w_i [drho + rho (p_i - F'_i/2)], placed at the slot the next pull of
// (x, i) reads: x - e_i (periodic), or the mirrored slot of the opposite
// direction beyond a wall.  MODE 0 only records max |d_i / w_i| (FP16 scale).
template <class L, int FO, class R>
__device__ __forceinline__ void init_site(const MidState<L, R>& m, R (&d)[L::Q]) {
  constexpr int NP = (L::Q - 1) / 2;
  {
    R E, Fe;
    rest_terms<L, FO, R>(m, E, Fe);
    d[0] = mul_w<L, 0>(fma(m.rho, E - R(0.5) * Fe, m.drho));
  }
  static_for<0, NP>([&](auto K) {
    constexpr int ip = 2 * K + 1, im = ip + 1;
    R E, O, Fe, Fo;
    pair_terms<L, FO, ip, R>(m, E, O, Fe, Fo);
    const R ev = mul_w<L, ip>(fma(m.rho, E - R(0.5) * Fe, m.drho));
    const R od = mul_w<L, ip>(m.rho * (O - R(0.5) * Fo));
    d[ip] = ev + od;
    d[im] = ev - od;
  });
}

template <class L, int P, int MODE>
__global__ void __launch_bounds__(128) k_init(const double* __restrict__ rho,
                                              const double* __restrict__ u,
                                              const double* __restrict__ T,
                                              typename Codec<P>::T* __restrict__ fout,
                                              unsigned int* __restrict__ maxbits, int force_order,
                                              const StepParams p) {
  using C = Codec<P>;
  using R = typename C::R;
  constexpr int Q = L::Q, D = L::D;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const int y = D == 2 ? p.a0 + (int)blockIdx.y : (int)blockIdx.y;
  const int z = D == 3 ? p.a0 + (int)blockIdx.z : 0;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int site = (z * ny + y) * nx + x;
  const size_t N = (size_t)p.N;
  if (p.solid && p.solid[site]) return;
  double gd[3];
  site_force<D>(p, x, y, z, site, gd);
  const R g[3] = {R(gd[0]), R(gd[1]), R(gd[2])};
  const R uu[3] = {R(u[site]), R(u[N + site]), D == 3 ? R(u[2 * N + site]) : R(0)};
  MidState<L, R> m;
  given_state<L, R>(R(rho[site] - 1.0), uu, R(T[site] - 1.0), g, m);
  R d[Q];
  if (force_order == 0) init_site<L, 0, R>(m, d);
  else if (force_order == 1) init_site<L, 1, R>(m, d);
  else init_site<L, 2, R>(m, d);
  if (MODE == 0) {
    float mx = 0.f;
    static_for<0, Q>([&](auto I) {
      constexpr int i = I;
      mx = fmaxf(mx, (float)fabs(double(d[i]) / L::W(i)));
    });
    atomicMax(maxbits, __float_as_uint(mx));
    return;
  }
  const int a = D == 2 ? y : z;
  const int nA = D == 2 ? ny : nz;
  const int lineA = D == 2 ? nx : nx * ny;
  const int colbase = D == 2 ? x : (y * nx + x);
  if constexpr (P == P_FP64) {  // storage probe: the initial state as a float codec stores it
    if (p.storage_probe)
      static_for<0, Q>([&](auto I) {
        constexpr int i = I;
        d[i] = probe_round<i>(d[i], p);
      });
  }
  static_for<0, Q>([&](auto I) {
    constexpr int i = I;
    constexpr int ex = L::E(i, 0), ey = L::E(i, 1), ez = L::E(i, 2);
    constexpr int eA = L::E(i, D - 1);
    const int sA = a - eA;
    if (p.wall != W_NONE && (sA < 0 || sA >= nA)) {
      constexpr int io = opposite<i>();
      const int mA = sA < 0 ? eA - 1 - a : 2 * nA - 1 - sA;
      fout[io * N + colbase + mA * lineA] = C::template encode<L, io>(d[i], p);
    } else {
      const int sx = wrap3(x - ex, nx);
      const int sy = wrap3(y - ey, ny);
      const int sz = D == 3 ? wrap3(z - ez, nz) : 0;
      const int src = (sz * ny + sy) * nx + sx;
      if (p.solid && p.solid[src]) {
        // pulled from a solid site: the wall emits it; the slot the wall
        // absorbs (-e_i, at this site) holds the local value
        constexpr int io = opposite<i>();
        fout[io * N + site] = C::template encode<L, io>(d[io], p);
      } else {
        fout[i * N + src] = C::template encode<L, i>(d[i], p);
      }
    }
  });
}

// ------------------------------------------------------------ moments
// Physical rho, u, T and heat flux q in double (the FP64 diagnostic), with
// q = 1/2 (1 - 1/(2 tau)) sum_i (f~_i - f0_i + F_i/2) |xi_i - u|^2 (xi_i - u).
// Each of the three sums is a combination of moments of order <= 3, which
// the quadrature integrates exactly for f0 and F (degree 9 >= 4 + 3 on
// D2Q37, 7 >= 3 + 3 on D3Q39), so only the pulled f~ is summed per site:
//   sum f0 |c|^2 c = 0 (the Maxwellian carries no heat flux), and with
//   S = the second moment the force's n = 3 term contracts (rho (u u + theta
//   delta), minus sigma-bar for FO 3; rho delta for orders 0 and 1) and
//   M2 = sum F xi xi (rho (g u + u g) for orders >= 1, else 0),
//   sum F |c|^2 c_a = 2 (S g)_a + g_a tr S - u_a tr M2 - 2 (M2 u)_a
//                     + 2 rho u_a (u.g) + rho u^2 g_a,
// which is (D + 2) rho theta g_a at order 2.  sum f~ |c|^2 c comes from the
// raw moments of the deviations d = f~ - w: m0 = sum d, m1 = sum d e,
// m2 = sum d e e, m3 = sum d |e|^2 e (c = xi - u, xi = c_lat e).
template <class L>
struct HeatMoments {
  double m0, m1[3], m2[6], m3[3];  // m2 as (xx, yy, zz, xy, xz, yz)
};

template <class L>
__device__ __forceinline__ HeatMoments<L> heat_moments(const double (&d)[L::Q]) {
  constexpr int NP = (L::Q - 1) / 2;
  HeatMoments<L> h{};
  h.m0 = d[0];
  static_for<0, NP>([&](auto K) {
    constexpr int ip = 2 * K + 1, im = ip + 1;
    constexpr int ex = L::E(ip, 0), ey = L::E(ip, 1), ez = L::E(ip, 2);
    constexpr int e2 = ex * ex + ey * ey + ez * ez;
    const double s = d[ip] + d[im];
    const double a = d[ip] - d[im];
    h.m0 += s;
    h.m1[0] = mac<ex>(a, h.m1[0]);
    h.m1[1] = mac<ey>(a, h.m1[1]);
    h.m2[0] = mac<ex * ex>(s, h.m2[0]);
    h.m2[1] = mac<ey * ey>(s, h.m2[1]);
    h.m2[3] = mac<ex * ey>(s, h.m2[3]);
    h.m3[0] = mac<e2 * ex>(a, h.m3[0]);
    h.m3[1] = mac<e2 * ey>(a, h.m3[1]);
    if constexpr (L::D == 3) {
      h.m1[2] = mac<ez>(a, h.m1[2]);
      h.m2[2] = mac<ez * ez>(s, h.m2[2]);
      h.m2[4] = mac<ex * ez>(s, h.m2[4]);
      h.m2[5] = mac<ey * ez>(s, h.m2[5]);
      h.m3[2] = mac<e2 * ez>(a, h.m3[2]);
    }
  });
  return h;
}

// The same raw moments from float deviations without FP64 arithmetic: each
// moment is a float pair s + c, the pair sums d_+ +- d_- are split exactly
// (Knuth's two-sum), products by the small integer weights keep their FMA
// residual, and every rounding error goes into c.  The result equals the
// FP64 sum to a few units in 2^-48 of the terms' magnitude.
struct FF {
  float s = 0.f, c = 0.f;
};
// (explicit round-to-nearest operations: a product fused into a following
// sum would break these error-free transformations)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// acc += K (hi + lo) for a compile-time integer K
template <int K>
__device__ __forceinline__ void ff_mac(FF& acc, float hi, float lo) {
  if constexpr (K != 0) {
    const float p = __fmul_rn(float(K), hi);
    const float pe = fmaf(float(K), hi, -p);
    float t, e;
    two_sum(acc.s, p, t, e);
    acc.s = t;
    acc.c += e + pe + float(K) * lo;
  }
}

// Symmetric 3x3 (xx, yy, zz, xy, xz, yz) times a vector.
template <class R>
__device__ __forceinline__ void sym_mul(const R (&S)[6], const R (&v)[3], R (&o)[3]) {
  o[0] = S[0] * v[0] + S[3] * v[1] + S[4] * v[2];
  o[1] = S[3] * v[0] + S[1] * v[1] + S[5] * v[2];
  o[2] = S[4] * v[0] + S[5] * v[1] + S[2] * v[2];
}

// The same raw moments as float-float values: each compensated pair s + c
// renormalised (an exact two-sum, since c may exceed ulp(s) after a
// cancellation).
template <class L>
__device__ __forceinline__ void heat_moments_df(const float (&d)[L::Q], DF& m0, DF (&m1)[3], DF (&m2)[6],
                                                DF (&m3)[3]) {
  constexpr int NP = (L::Q - 1) / 2;
  FF f0, f1[3], f2[6], f3[3];
  f0.s = d[0];
  static_for<0, NP>([&](auto K) {
    constexpr int ip = 2 * K + 1, im = ip + 1;
    constexpr int ex = L::E(ip, 0), ey = L::E(ip, 1), ez = L::E(ip, 2);
    constexpr int e2 = ex * ex + ey * ey + ez * ez;
    float sh, sl, ah, al;
    two_sum(d[ip], d[im], sh, sl);
    two_sum(d[ip], -d[im], ah, al);
    ff_mac<1>(f0, sh, sl);
    ff_mac<ex>(f1[0], ah, al);
    ff_mac<ey>(f1[1], ah, al);
    ff_mac<ex * ex>(f2[0], sh, sl);
    ff_mac<ey * ey>(f2[1], sh, sl);
    ff_mac<ex * ey>(f2[3], sh, sl);
    ff_mac<e2 * ex>(f3[0], ah, al);
    ff_mac<e2 * ey>(f3[1], ah, al);
    if constexpr (L::D == 3) {
      ff_mac<ez>(f1[2], ah, al);
      ff_mac<ez * ez>(f2[2], sh, sl);
      ff_mac<ex * ez>(f2[4], sh, sl);
      ff_mac<ey * ez>(f2[5], sh, sl);
      ff_mac<e2 * ez>(f3[2], ah, al);
    }
  });
  auto v = [](const FF& f) {
    DF r;
    df_two_sum(f.s, f.c, r.hi, r.lo);
    return r;
  };
  m0 = v(f0);
  for (int a = 0; a < 3; ++a) {
    m1[a] = v(f1[a]);
    m3[a] = v(f3[a]);
  }
  for (int c = 0; c < 6; ++c) m2[c] = v(f2[c]);
}

__device__ __forceinline__ double out_double(double x) { return x; }
__device__ __forceinline__ double out_double(DF x) { return df_to_double(x); }

// rho, u, T and q of one site from the raw moments of its pulled deviations
// (see the comment above HeatMoments), in the arithmetic type R: double for
// FP64 storage, float-float (~48 bits, lbm_df.cuh) for the float codecs,
// whose FP64 combination ran at the FP64 units' rate; each output is one
// rounding to double.
template <class L, class R>
__device__ __forceinline__ void write_moments(R m0, const R (&m1)[3], const R (&m2)[6], const R (&m3)[3],
                                              const R (&g)[3], int site, size_t N, int force_order,
                                              const StepParams& p, double* __restrict__ rho,
                                              double* __restrict__ u, double* __restrict__ T,
                                              double* __restrict__ q) {
  constexpr int D = L::D;
  const R c = R(L::c), c2 = R(L::c2);
  const R r = R(1) + m0, ir = R(1) / r;
  R J[3], uu[3];
  for (int a = 0; a < 3; ++a) {
    J[a] = c * m1[a];  // sum f~ xi = rho u~
    uu[a] = J[a] * ir + R(0.5) * g[a];
  }
  const R k2 = m2[0] + m2[1] + m2[2];
  const R ut2 = (J[0] * J[0] + J[1] * J[1] + J[2] * J[2]) * ir * ir;
  const R g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  const R Th = ((c2 * k2 - R(D) * m0) * ir - ut2) * R(1.0 / D) + g2 * R(0.25 / D);
  if (rho) rho[site] = out_double(r);
  if (T) T[site] = out_double(R(1) + Th);
  if (u)
    for (int a = 0; a < D; ++a) u[a * N + site] = out_double(uu[a]);
  if (!q) return;
  const R om = site_omega<R>(p, r, R(1) + Th);
  const R u2 = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
  const R ug = uu[0] * g[0] + uu[1] * g[1] + uu[2] * g[2];
  const R uJ = uu[0] * J[0] + uu[1] * J[1] + uu[2] * J[2];
  // sum f~ |c|^2 c with P = c^2 m2 (so sum f~ xi xi = delta + P)
  R Pm[6], Pu[3];
  for (int k = 0; k < 6; ++k) Pm[k] = c2 * m2[k];
  sym_mul<R>(Pm, uu, Pu);
  const R c3 = R(L::c * L::c2);
  R C3[3];
  for (int a = 0; a < 3; ++a)
    C3[a] = c3 * m3[a] - R(D + 2) * uu[a] - uu[a] * (c2 * k2) - R(2) * Pu[a] + R(2) * uu[a] * uJ +
            u2 * J[a] - u2 * uu[a] * r;
  // sum F |c|^2 c
  R FC3[3];
  const R th = R(1) + Th;
  if (force_order >= 2) {
    for (int a = 0; a < 3; ++a) FC3[a] = R(D + 2) * r * th * g[a];
    if (force_order == 3) {
      // S = rho (u u + theta delta) - sigma-bar, sigma-bar = -(1 - om/2) S_st
      R Sst[6], Sg[3];
      const R iso = fma(r, Th, m0);
      const R hr = R(0.5) * r;
      auto conv = [&](int a, int b) { return hr * (uu[a] * (g[b] - uu[b]) + uu[b] * (g[a] - uu[a])); };
      Sst[0] = Pm[0] - iso + conv(0, 0);
      Sst[1] = Pm[1] - iso + conv(1, 1);
      Sst[2] = D == 3 ? Pm[2] - iso + conv(2, 2) : R(0);
      Sst[3] = Pm[3] + conv(0, 1);
      Sst[4] = D == 3 ? Pm[4] + conv(0, 2) : R(0);
      Sst[5] = D == 3 ? Pm[5] + conv(1, 2) : R(0);
      sym_mul<R>(Sst, g, Sg);
      const R kf = R(1) - R(0.5) * om;
      for (int a = 0; a < 3; ++a) FC3[a] += R(2) * kf * Sg[a];
    }
  } else {
    // S = rho delta; M2 = rho (g u + u g) at order 1, 0 at order 0
    for (int a = 0; a < 3; ++a) {
      FC3[a] = R(D + 2) * r * g[a] + R(2) * r * uu[a] * ug + r * u2 * g[a];
      if (force_order == 1) FC3[a] -= R(2) * r * uu[a] * ug + R(2) * r * (g[a] * u2 + uu[a] * ug);
    }
  }
  const R kq = R(0.5) * (R(1) - R(0.5) * om);
  for (int a = 0; a < D; ++a) q[a * N + site] = out_double(kq * (C3[a] + R(0.5) * FC3[a]));
}

template <class L, int P>
__global__ void __launch_bounds__(128) k_moments(const typename Codec<P>::T* __restrict__ fin,
                                                 double* __restrict__ rho, double* __restrict__ u,
                                                 double* __restrict__ T, double* __restrict__ q,
                                                 int force_order, const StepParams p) {
  constexpr int Q = L::Q, D = L::D;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const int y = D == 2 ? p.a0 + (int)blockIdx.y : (int)blockIdx.y;
  const int z = D == 3 ? p.a0 + (int)blockIdx.z : 0;
  const int site = (z * p.ny + y) * p.nx + x;
  const size_t N = (size_t)p.N;
  if (p.solid && p.solid[site]) {  // solid sites report zeros
    if (rho) rho[site] = 0.0;
    if (T) T[site] = 0.0;
    for (int a = 0; a < D; ++a) {
      if (u) u[a * N + site] = 0.0;
      if (q) q[a * N + site] = 0.0;
    }
    return;
  }
  if (P != P_FP64 && !p.solid) {
    // float storage: the deviations are exact floats; compensated float-pair
    // sums and a float-float combination, no FP64 arithmetic but the final
    // rounding of each output
    float d[Q];
    pull<L, P, float>(fin, p, x, y, z, d);
    DF m0, m1[3], m2[6], m3[3];
    heat_moments_df<L>(d, m0, m1, m2, m3);
    DF g[3];
    site_force_r<D, DF>(p, x, y, z, site, g);
    write_moments<L, DF>(m0, m1, m2, m3, g, site, N, force_order, p, rho, u, T, q);
    return;
  }
  double d[Q];
  if (p.solid) pull_solid<L, P, double>(fin, p, x, y, z, site, d);
  else pull<L, P, double>(fin, p, x, y, z, d);
  const HeatMoments<L> h = heat_moments<L>(d);
  double g[3];
  site_force<D>(p, x, y, z, site, g);
  write_moments<L, double>(h.m0, h.m1, h.m2, h.m3, g, site, N, force_order, p, rho, u, T, q);
}

// ------------------------------------------------------ conservation sums
// Compensated (Neumaier) running sum in the arithmetic type R of a kernel:
// the exact sum is s + c up to the rounding of c.
template <class R>
struct RSum {
  R s = R(0), c = R(0);
  __device__ __forceinline__ void add(R v) {
    const R t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  __device__ __forceinline__ void merge(const RSum& o) {
    add(o.s);
    c += o.c;
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// Quantities reduced: 0 mass, 1..3 momentum, 4 energy; plus a count of bad sites.
constexpr int NCONS = 5;
// Doubles per block in the partials array: the NCONS compensated pairs of the
// block's per-site sums, stored in the kernel's type R from the start of the
// slot, then the block's number of fluid sites (a double at index 2 NCONS).
constexpr int CONS_SLOT = 2 * NCONS + 1;

// Block-wide merge of per-thread compensated pairs in a fixed order: the
// pairs go to shared memory, 8 threads per quantity merge contiguous runs of
// BS / 8, thread 0 merges the 8 runs; the counts are summed by warp shuffles.
// All in R: with float storage no FP64 instruction runs here (GB300 issues
// FP64 at a small fraction of the FP32 rate, so a double-precision tree at
// the end of every block was the tail of the pass).  The totals are valid in
// thread 0 only.
template <class R, int BS>
__device__ __forceinline__ void reduce_block(const RSum<R> (&v)[NCONS], unsigned n, unsigned bad,
                                             RSum<R> (&tot)[NCONS], unsigned& ntot,
                                             unsigned& btot) {
  static_assert(BS % 32 == 0 && BS >= 64, "block size");
  constexpr int RUN = BS / 8;
  __shared__ R sh_s[NCONS][BS], sh_c[NCONS][BS];
  __shared__ RSum<R> sh_p[NCONS][8];
  __shared__ unsigned sh_n[BS / 32], sh_b[BS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < NCONS; ++k) {
    sh_s[k][tid] = v[k].s;
    sh_c[k][tid] = v[k].c;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n += __shfl_down_sync(0xffffffffu, n, off);
    bad += __shfl_down_sync(0xffffffffu, bad, off);
  }
  if (lane == 0) {
    sh_n[warp] = n;
    sh_b[warp] = bad;
  }
  __syncthreads();
  if (tid < NCONS * 8) {
    const int k = tid / 8, r = tid % 8;
    RSum<R> a{sh_s[k][r * RUN], sh_c[k][r * RUN]};
    for (int j = 1; j < RUN; ++j) a.merge(RSum<R>{sh_s[k][r * RUN + j], sh_c[k][r * RUN + j]});
    sh_p[k][r] = a;
  }
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < NCONS; ++k) {
      RSum<R> a = sh_p[k][0];
      for (int r = 1; r < 8; ++r) a.merge(sh_p[k][r]);
      tot[k] = a;
    }
    ntot = 0u;
    btot = 0u;
    for (int w = 0; w < BS / 32; ++w) {
      ntot += sh_n[w];
      btot += sh_b[w];
    }
  }
}

// Mass, momentum and energy (as s, c pairs of doubles: out[2k], out[2k + 1])
// from the grid's sums.  Uniform g: S = (sum drho, sum j, sum k2) and, with
// n fluid sites, mass M = n + S0, momentum c J + M g / 2, energy
// (D n + c^2 K2 + c J.g + M |g|^2 / 2) / 2 (mid-point values of R1).  Other
// forces: S = (sum drho, sum of per-site momentum, sum of per-site energy
// less D / 2), so the momentum is S1..3 and the energy D n / 2 + S4.
template <class L, class R>
__device__ __forceinline__ void conserved_from_sums(const RSum<R> (&S)[NCONS], double n,
                                                    const StepParams& p, double* out) {
  constexpr int D = L::D;
  double v[NCONS];
  for (int k = 0; k < NCONS; ++k) v[k] = S[k].value();
  const double mass = n + v[0];
  double res[NCONS];
  res[0] = mass;
  res[1] = res[2] = res[3] = 0.0;
  if (p.gkind == G_UNIFORM) {
    const double g[3] = {p.g0[0], p.g0[1], D == 3 ? p.g0[2] : 0.0};
    double jg = 0.0;
    for (int a = 0; a < D; ++a) {
      res[1 + a] = L::c * v[1 + a] + 0.5 * g[a] * mass;
      jg += L::c * v[1 + a] * g[a];
    }
    const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    res[4] = 0.5 * (double(D) * n + L::c2 * v[4] + jg + 0.5 * g2 * mass);
  } else {
    for (int a = 0; a < D; ++a) res[1 + a] = v[1 + a];
    res[4] = 0.5 * double(D) * n + v[4];
  }
  for (int k = 0; k < NCONS; ++k) {
    out[2 * k] = res[k];
    out[2 * k + 1] = 0.0;
  }
}

// Merge of the partials of nblocks blocks (slot layout CONS_SLOT) by one
// block of BS threads, in a fixed order: thread t takes blocks t, t + BS, ...
// then the block merge above.  Thread 0 writes out[0 .. 2 NCONS - 1] (s, c
// pairs) and out[2 NCONS] = the bad-site count.
template <class L, class R, int BS>
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part,
                                                const unsigned* __restrict__ badcount, int nblocks,
                                                const StepParams& p, double* out) {
  RSum<R> f[NCONS];
  unsigned n = 0u, b = 0u;
  for (int blk = threadIdx.x; blk < nblocks; blk += BS) {
    const double* slot = part + (size_t)blk * CONS_SLOT;
    const R* rs = reinterpret_cast<const R*>(slot);
    for (int k = 0; k < NCONS; ++k) f[k].merge(RSum<R>{__ldcg(rs + 2 * k), __ldcg(rs + 2 * k + 1)});
    n += (unsigned)__ldcg(slot + 2 * NCONS);
    b += __ldcg(badcount + blk);
  }
  RSum<R> tot[NCONS];
  unsigned ntot, btot;
  reduce_block<R, BS>(f, n, b, tot, ntot, btot);
  if (threadIdx.x == 0) {
    conserved_from_sums<L, R>(tot, double(ntot), p, out);
    out[2 * NCONS] = double(btot);
  }
}

// Grid-stride pass: block b handles row tiles b, b + gridDim.x, ... (one
// site per thread and tile; threads past the row end contribute nothing).
// Per site only the raw moments are needed, in the codec's arithmetic
// precision: mass rho = 1 + drho, momentum rho u = c j + rho g / 2, energy
// rho (|u|^2 + D theta) / 2 = (K + c j.g + rho |g|^2 / 2) / 2 with
// K = D + c^2 k2 (mid-point values of R1, no division).  With a uniform g
// these are linear in the sums of drho, j and k2, so a thread sums only
// those; otherwise it sums the per-site momentum and energy.  Each thread
// keeps compensated pairs in R; the block merges them (reduce_block) and
// writes its slot of `part` (CONS_SLOT doubles per block) and its bad-site
// count.  The number of blocks is fixed by the caller, so the summation
// order, and the result, are deterministic for a grid.
//
// ticket != nullptr: the last block to finish (by an atomic ticket) also
// reduces all partials in block order into out (the k_conserved_final
// layout, plus out[2 NCONS + 1] = *err, the bounded-wait error flag) and
// resets the ticket; out may be mapped host memory.
// Resident 128-thread blocks per SM the conservation pass is compiled for
// (its grid is LBM_CONSERVED_BLOCKS blocks per SM, a tuning hook).
#ifndef LBM_CONSERVED_BLOCKS
#define LBM_CONSERVED_BLOCKS 4
#endif
template <class L, int P>
__global__ void __launch_bounds__(128, LBM_CONSERVED_BLOCKS) k_conserved(const typename Codec<P>::T* __restrict__ fin,
                                                   double* __restrict__ part,
                                                   unsigned* __restrict__ badcount,
                                                   unsigned* __restrict__ ticket,
                                                   double* __restrict__ out,
                                                   const int* __restrict__ err,
                                                   const StepParams p) {
  using R = typename Codec<P>::R;
  constexpr int Q = L::Q, D = L::D;
  const int ntx = (p.nx + 127) / 128;
  const int ntiles = ntx * (D == 2 ? p.na : p.ny * p.na);
  const bool uniform = p.gkind == G_UNIFORM;
  RSum<R> sums[NCONS];
  unsigned count = 0u, bad = 0u;
  const bool walls = p.wall != W_NONE;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // the wall rows, whose pull also gathers the wall sums, come first so
    // that they do not form the tail of the pass
    const int xt = t % ntx, row = t / ntx;
    const int y = D == 2 ? p.a0 + wall_rows_first(row, p.na, walls) : row % p.ny;
    const int z = D == 3 ? p.a0 + wall_rows_first(row / p.ny, p.na, walls) : 0;
    const int x = xt * 128 + threadIdx.x;
    if (x >= p.nx) continue;
    const int site = (z * p.ny + y) * p.nx + x;
    if (p.solid && p.solid[site]) continue;
    R d[Q];
    const int a = D == 2 ? y : z;
    const int nA = D == 2 ? p.ny : p.nz;
    const int wx0 = xt * 128 + (threadIdx.x & ~31);
    const bool interior = !(walls && (a < 3 || a >= nA - 3)) && wx0 >= 3 && wx0 + 31 <= p.nx - 4;
    if (p.solid) pull_solid<L, P, R>(fin, p, x, y, z, site, d);
    else if (interior) pull_interior<L, P, R>(fin + site, p, y, z, d);
    else pull<L, P, R>(fin, p, x, y, z, d);
    R g[3];
    if (sizeof(R) == sizeof(float) && p.gkind == G_FIELD && p.gtab_f == nullptr) {
      // a caller's double field without a float copy (lbm_conserved_static),
      // rounded to float as a context rounds its copy
      g[0] = R(__ldg(p.gtab + site));
      g[1] = R(__ldg(p.gtab + (size_t)p.N + site));
      g[2] = D == 3 ? R(__ldg(p.gtab + 2 * (size_t)p.N + site)) : R(0);
    } else {
      site_force_r<D, R>(p, x, y, z, site, g);
    }
    const RawMoments<L, R> r = raw_moments<L, R>(d);
    ++count;
    sums[0].add(r.drho);
    const R j0 = mul_c<L, R>(r.j[0]), j1 = mul_c<L, R>(r.j[1]), j2 = mul_c<L, R>(r.j[2]);
    const R rr = R(1) + r.drho;
    const R g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    if (uniform) {
      for (int a2 = 0; a2 < D; ++a2) sums[1 + a2].add(r.j[a2]);
      sums[4].add(r.k2);
    } else {
      const R hr = R(0.5) * rr;
      sums[1].add(fma(hr, g[0], j0));
      sums[2].add(fma(hr, g[1], j1));
      if (D == 3) sums[3].add(fma(hr, g[2], j2));
      const R jg = j0 * g[0] + j1 * g[1] + j2 * g[2];
      sums[4].add(R(0.5) * (mul_c2<L, R>(r.k2) + jg + R(0.5) * rr * g2));
    }
    // positivity check in the codec's precision, without divisions:
    // D theta = (K - |c j|^2 / rho) / rho + g^2 / 4 with K = D + c^2 k2, so
    // for rho > 0, theta > 0 exactly when e = K rho - |c j|^2 + rho^2 g^2 / 4
    // > 0; a NaN or infinite moment makes e NaN or infinite
    const R K = R(D) + mul_c2<L, R>(r.k2);
    const R e = fma(rr * rr, R(0.25) * g2, fma(K, rr, -(j0 * j0 + j1 * j1 + j2 * j2)));
    bad += (rr > R(0) && e > R(0) && isfinite(e)) ? 0u : 1u;
  }
  {
    RSum<R> tot[NCONS];
    unsigned ntot, btot;
    reduce_block<R, 128>(sums, count, bad, tot, ntot, btot);
    if (threadIdx.x == 0) {
      double* slot = part + (size_t)blockIdx.x * CONS_SLOT;
      R* rs = reinterpret_cast<R*>(slot);
      for (int k = 0; k < NCONS; ++k) {
        rs[2 * k] = tot[k].s;
        rs[2 * k + 1] = tot[k].c;
      }
      slot[2 * NCONS] = double(ntot);
      badcount[blockIdx.x] = btot;
    }
  }
  if (!ticket) return;
  // the last block to finish reduces every block's partials, in block order
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  reduce_partials<L, R, 128>(part, badcount, gridDim.x, p, out);
  if (threadIdx.x == 0) {
    out[2 * NCONS + 1] = err ? double(*(volatile const int*)err) : 0.0;
    *ticket = 0u;
  }
}

// Final pass of the two-kernel form: one block of 128 threads merges the
// partials of k_conserved (launched without a ticket) into out: 2 NCONS
// doubles (s, c pairs) followed by the bad-site count (as double).
template <class L, int P>
__global__ void __launch_bounds__(128) k_conserved_final(const double* __restrict__ part,
                                                         const unsigned* __restrict__ badcount,
                                                         int nblocks, double* __restrict__ out,
                                                         const StepParams p) {
  reduce_partials<L, typename Codec<P>::R, 128>(part, badcount, nblocks, p, out);
}

// ------------------------------------------------------ state access
template <class L, int P>
__global__ void __launch_bounds__(128) k_get_pulled(const typename Codec<P>::T* __restrict__ fin,
                                                    double* __restrict__ out, const StepParams p) {
  constexpr int Q = L::Q, D = L::D;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const int y = D == 2 ? p.a0 + (int)blockIdx.y : (int)blockIdx.y;
  const int z = D == 3 ? p.a0 + (int)blockIdx.z : 0;
  const int site = (z * p.ny + y) * p.nx + x;
  const size_t N = (size_t)p.N;
  if (p.solid && p.solid[site]) {
    static_for<0, Q>([&](auto I) { out[int(I) * N + site] = 0.0; });
    return;
  }
  double d[Q];
  if (p.solid) pull_solid<L, P, double>(fin, p, x, y, z, site, d);
  else pull<L, P, double>(fin, p, x, y, z, d);
  static_for<0, Q>([&](auto I) {
    constexpr int i = I;
    out[i * N + site] = L::W(i) + d[i];
  });
}

// DIR = 0: out = decode(f) + w ; DIR = 1: f = encode(in - w)
template <class L, int P, int DIR>
__global__ void __launch_bounds__(128) k_state(typename Codec<P>::T* __restrict__ f,
                                               double* __restrict__ io, const StepParams p) {
  using C = Codec<P>;
  constexpr int Q = L::Q, D = L::D;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const int y = D == 2 ? p.a0 + (int)blockIdx.y : (int)blockIdx.y;
  const int z = D == 3 ? p.a0 + (int)blockIdx.z : 0;
  const int site = (z * p.ny + y) * p.nx + x;
  const size_t N = (size_t)p.N;
  static_for<0, Q>([&](auto I) {
    constexpr int i = I;
    if (DIR == 0)
      io[i * N + site] = L::W(i) + double(C::template decode<L, i>(f[i * N + site], p));
    else
      f[i * N + site] = C::template encode<L, i>(typename C::R(io[i * N + site] - L::W(i)), p);
  });
}

}  // namespace lbm
