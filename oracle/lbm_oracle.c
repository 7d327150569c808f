/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the thermal compressible lattice
 * Boltzmann step with a Hermite-expanded body force, after Li & Shan,
 * "Body-force modelling in thermal compressible flows with lattice Boltzmann
 * method" (arXiv 2302.04741).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg load this library.  The CUDA
 * library never links, loads or calls it, and the two share no code, header,
 * table or generator: this file carries its own quadrature rules (rules.h,
 * written by oracle/gen_rules.py) and its own arithmetic.
 *
 * The oracle is deliberately slow and literal.  Everything is written in the
 * paper's tensor notation with rank-n tensors stored as flat D^n arrays:
 *   - Hermite tensors H^(n)(xi), n <= 4, from their explicit definitions
 *     (Sec. 2; H^(3) = xi^3 - 3 xi delta is printed before Eq. f3);
 *   - Hermite coefficients a^(n)_0 of the Maxwellian (Eq. an applied to f^(0);
 *     a^(2)_0 is the equilibrium part of Eq. f2);
 *   - discrete equilibrium f^(0)_i = w_i sum_n a^(n)_0 : H^(n)(xi_i) / n!
 *     (Eq. fN truncated, sampled with f_i = w_i f_N(xi_i)/omega(xi_i));
 *   - discrete force from its DEFINING series (Eq. F),
 *     F_i = w_i sum_{n=1}^{N+1} (g a^(n-1)) : H^(n)(xi_i) / (n-1)!,
 *     not from the expanded scalar form Eq. fi;
 *   - the update Eq. lbm with the mid-point state rho, u + g/2, theta.
 *
 * Readings of points the paper leaves open (numbered as in the design notes):
 *   R1  f in Eq. lbm is the auxiliary (pre-collision) distribution f~; the
 *       mid-point state is rho = sum f~, u = sum f~ xi / rho + g/2 and the
 *       physical temperature theta = (sum f~ xi^2/rho - |u~|^2)/D + g^2/(4D)
 *       with u~ = sum f~ xi / rho (this keeps the O(g^2) term so that the
 *       energy budget per step is exactly 2 rho g.u).
 *   R2  tau passed in is the collision divisor tau-hat of Eq. lbm.
 *   R8  sigma-bar = -(1 - 1/(2 tau)) sum_i (f~_i - f0_i)(xi_i - u)(xi_i - u)
 *       with u the mid-point velocity; it enters the force through
 *       a^(2) = a^(2)_0 - sigma (Eq. f2).  Off unless requested.
 *   R9  heat flux q = 1/2 (1 - 1/(2 tau)) sum_i (f~_i - f0_i + F_i/2)
 *       |xi_i - u|^2 (xi_i - u): the physical non-equilibrium part of the
 *       distribution (f0 carries no heat flux).
 *   R10 walls (the paper's boundary rule is unpublished): half-way bounce-back
 *       keeping the column, f~_i(x) = f*_{-i}(x with x_a -> e_ia - 1 - x_a)
 *       at the low wall (mirrored at the high wall); the thermal wall fills
 *       the same slots with rho_w f0_i(1, 0, T_wall) where rho_w makes the
 *       column's incoming mass equal its outgoing mass.  Pinned by mass
 *       conservation, the conduction profile, Fourier's law, the no-slip
 *       channel parabola and the kinetic slip; at slot level by the
 *       micro-reversibility of streaming with bounce-back and by the closed
 *       form of the thermal wall's refill of a resting fluid (as for R15's
 *       solid sites; tests/test_wall_pins.py).
 *   R11 storage holds the post-collision distribution f*; a step pulls
 *       f~_i(x) = f*_i(x - e_i) and collides.  init places f~ = f0 - F/2 at
 *       the slots the first pull reads, so the pulled state at t = 0 is
 *       exactly the requested one (periodic and bounce-back walls).
 *   R13 constant dynamic viscosity (the validation runs of Sec. 3 set
 *       tau = mu / (rho theta) so that mu and lambda stay uniform): with
 *       mu > 0 every site uses tau-hat = mu / (rho theta) + 1/2 with the
 *       mid-point rho and theta, in the update, sigma-bar and q.
 *   R15 solid sites (curved walls, staircase): a slot of a fluid site x
 *       pulled from a solid site y = x - e_i holds rho_w(x) f0_i(1, 0, T_y);
 *       rho_w(x) makes the mass x emits into solid sites (its post-collision
 *       slots -e_i) equal the mass the walls emit into x.  Links are not
 *       traced: only the source site decides.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "rules.h"

#define ORC_QMAX 39
#define ORC_T4 81 /* 3^4: largest rank-4 tensor */

enum { ORC_D2Q37 = 0, ORC_D3Q39 = 1 };
enum { ORC_PERIODIC = 0, ORC_BOUNCE_BACK = 1, ORC_THERMAL_WALL = 2 };

typedef struct {
  int D, Q, neq;
  double c;
  int e[ORC_QMAX][3];
  double w[ORC_QMAX];
  double xi[ORC_QMAX][3];
  int opp[ORC_QMAX];
  double H[5][ORC_QMAX][ORC_T4]; /* H^(n)(xi_i) for n = 0..4 */
} orc_lattice;

static long ipow(long b, int n) {
  long r = 1;
  while (n-- > 0) r *= b;
  return r;
}

static double kd(int a, int b) { return a == b ? 1.0 : 0.0; }

/* ------------------------------------------------------------------------ */
/* Hermite tensors H^(n)(xi), n <= 4, written out from their definitions:    */
/*   H0 = 1, H1 = xi_a, H2 = xi_a xi_b - d_ab,                               */
/*   H3 = xi_a xi_b xi_c - (xi_a d_bc + xi_b d_ac + xi_c d_ab),              */
/*   H4 = xi_a xi_b xi_c xi_d - (six xi xi d terms) + (three d d terms).     */
/* Flat index: ((a*D + b)*D + c)*D + d.                                      */
/* ------------------------------------------------------------------------ */
int orc_hermite_tensor(int D, int n, const double *x, double *H) {
  if (D < 1 || D > 3 || n < 0 || n > 4) return -1;
  long m = ipow(D, n);
  for (long k = 0; k < m; ++k) {
    int id[4] = {0, 0, 0, 0};
    long r = k;
    for (int p = n - 1; p >= 0; --p) {
      id[p] = (int)(r % D);
      r /= D;
    }
    int a = id[0], b = id[1], c = id[2], d = id[3];
    double v = 0.0;
    switch (n) {
      case 0: v = 1.0; break;
      case 1: v = x[a]; break;
      case 2: v = x[a] * x[b] - kd(a, b); break;
      case 3:
        v = x[a] * x[b] * x[c] - (x[a] * kd(b, c) + x[b] * kd(a, c) + x[c] * kd(a, b));
        break;
      case 4:
        v = x[a] * x[b] * x[c] * x[d]
            - (x[a] * x[b] * kd(c, d) + x[a] * x[c] * kd(b, d) + x[a] * x[d] * kd(b, c)
               + x[b] * x[c] * kd(a, d) + x[b] * x[d] * kd(a, c) + x[c] * x[d] * kd(a, b))
            + (kd(a, b) * kd(c, d) + kd(a, c) * kd(b, d) + kd(a, d) * kd(b, c));
        break;
    }
    H[k] = v;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Hermite coefficients of the Maxwellian, a^(n)_0 = int f0 H^(n) dxi:       */
/*   a0 = rho, a1 = rho u, a2 = rho (u u + (theta-1) d)  (Eq. f2),           */
/*   a3 = rho (u u u + (theta-1)(u_a d_bc + u_b d_ac + u_c d_ab)),           */
/*   a4 = rho (u u u u + (theta-1)(six u u d terms)                          */
/*             + (theta-1)^2 (three d d terms)).                             */
/* ------------------------------------------------------------------------ */
int orc_maxwell_coeff(int D, int n, double rho, const double *u, double theta, double *A) {
  if (D < 1 || D > 3 || n < 0 || n > 4) return -1;
  double t = theta - 1.0;
  long m = ipow(D, n);
  for (long k = 0; k < m; ++k) {
    int id[4] = {0, 0, 0, 0};
    long r = k;
    for (int p = n - 1; p >= 0; --p) {
      id[p] = (int)(r % D);
      r /= D;
    }
    int a = id[0], b = id[1], c = id[2], d = id[3];
    double v = 0.0;
    switch (n) {
      case 0: v = 1.0; break;
      case 1: v = u[a]; break;
      case 2: v = u[a] * u[b] + t * kd(a, b); break;
      case 3:
        v = u[a] * u[b] * u[c] + t * (u[a] * kd(b, c) + u[b] * kd(a, c) + u[c] * kd(a, b));
        break;
      case 4:
        v = u[a] * u[b] * u[c] * u[d]
            + t * (u[a] * u[b] * kd(c, d) + u[a] * u[c] * kd(b, d) + u[a] * u[d] * kd(b, c)
                   + u[b] * u[c] * kd(a, d) + u[b] * u[d] * kd(a, c) + u[c] * u[d] * kd(a, b))
            + t * t * (kd(a, b) * kd(c, d) + kd(a, c) * kd(b, d) + kd(a, d) * kd(b, c));
        break;
    }
    A[k] = rho * v;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Quadrature rules (own tables, rules.h) and per-abscissa Hermite tensors.   */
/* ------------------------------------------------------------------------ */
static int orc_lattice_build(int lat, orc_lattice *L) {
  const int(*vel)[4];
  const double *sw;
  memset(L, 0, sizeof(*L));
  if (lat == ORC_D2Q37) {
    L->D = ORC_D2Q37_D; L->Q = ORC_D2Q37_Q; L->c = orc_D2Q37_c; L->neq = 4;
    vel = orc_D2Q37_vel; sw = orc_D2Q37_shell_w;
  } else if (lat == ORC_D3Q39) {
    L->D = ORC_D3Q39_D; L->Q = ORC_D3Q39_Q; L->c = orc_D3Q39_c; L->neq = 3;
    vel = orc_D3Q39_vel; sw = orc_D3Q39_shell_w;
  } else {
    return -1;
  }
  for (int i = 0; i < L->Q; ++i) {
    L->w[i] = sw[vel[i][0]];
    for (int a = 0; a < 3; ++a) {
      L->e[i][a] = vel[i][1 + a];
      L->xi[i][a] = L->c * (double)L->e[i][a];
    }
  }
  for (int i = 0; i < L->Q; ++i) {
    L->opp[i] = -1;
    for (int k = 0; k < L->Q; ++k)
      if (L->e[k][0] == -L->e[i][0] && L->e[k][1] == -L->e[i][1] && L->e[k][2] == -L->e[i][2])
        L->opp[i] = k;
    if (L->opp[i] < 0) return -2;
    for (int n = 0; n <= 4; ++n) orc_hermite_tensor(L->D, n, L->xi[i], L->H[n][i]);
  }
  return 0;
}

int orc_lattice_info(int lat, int *D, int *Q, double *c, int *e, double *w, int *neq) {
  orc_lattice L;
  if (orc_lattice_build(lat, &L)) return -1;
  if (D) *D = L.D;
  if (Q) *Q = L.Q;
  if (c) *c = L.c;
  if (neq) *neq = L.neq;
  for (int i = 0; i < L.Q; ++i) {
    if (e)
      for (int a = 0; a < 3; ++a) e[3 * i + a] = L.e[i][a];
    if (w) w[i] = L.w[i];
  }
  return 0;
}

static double contract(long m, const double *A, const double *B) {
  double s = 0.0;
  for (long k = 0; k < m; ++k) s += A[k] * B[k];
  return s;
}

static const double inv_fact[5] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0};

/* Discrete equilibrium f0_i = w_i sum_{n<=neq} (1/n!) a^(n)_0 : H^(n)(xi_i). */
static void equilibrium(const orc_lattice *L, int neq, double rho, const double *u, double theta,
                        double *feq) {
  double A[5][ORC_T4];
  for (int n = 0; n <= neq; ++n) orc_maxwell_coeff(L->D, n, rho, u, theta, A[n]);
  for (int i = 0; i < L->Q; ++i) {
    double s = 0.0;
    for (int n = 0; n <= neq; ++n) s += inv_fact[n] * contract(ipow(L->D, n), A[n], L->H[n][i]);
    feq[i] = L->w[i] * s;
  }
}

/* Discrete force from the defining series (Eq. F with F_i = w_i F(xi_i)/omega):
 *   F_i = w_i sum_{n=1}^{N+1} (1/(n-1)!) sum_a g_a a^(n-1)_{I} H^(n)_{a I}(xi_i).
 * (n/n! = 1/(n-1)!; contracting the plain product g (x) a^(n-1) with the
 * symmetric H^(n) equals contracting the symmetrised product.)
 * sigma (D*D, may be NULL) replaces a^(2) by a^(2)_0 - sigma (Eq. f2). */
static void force(const orc_lattice *L, int order, double rho, const double *u, double theta,
                  const double *g, const double *sigma, double *F) {
  int D = L->D;
  double A[4][ORC_T4];
  for (int n = 0; n <= order && n <= 3; ++n) orc_maxwell_coeff(D, n, rho, u, theta, A[n]);
  if (sigma && order >= 2)
    for (int k = 0; k < D * D; ++k) A[2][k] -= sigma[k];
  for (int i = 0; i < L->Q; ++i) {
    double s = 0.0;
    for (int n = 1; n <= order + 1; ++n) {
      long m = ipow(D, n - 1);
      double t = 0.0;
      for (int a = 0; a < D; ++a) t += g[a] * contract(m, A[n - 1], L->H[n][i] + a * m);
      s += inv_fact[n - 1] * t;
    }
    F[i] = L->w[i] * s;
  }
}

int orc_equilibrium(int lat, int neq, double rho, const double *u, double theta, double *feq) {
  orc_lattice L;
  if (orc_lattice_build(lat, &L)) return -1;
  if (neq < 0) neq = L.neq;
  if (neq > 4) return -1;
  equilibrium(&L, neq, rho, u, theta, feq);
  return 0;
}

int orc_force(int lat, int order, double rho, const double *u, double theta, const double *g,
              const double *sigma, double *F) {
  orc_lattice L;
  if (orc_lattice_build(lat, &L)) return -1;
  if (order < 0 || order > 3) return -1;
  force(&L, order, rho, u, theta, g, sigma, F);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Simulation state.                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  orc_lattice L;
  int n[3];
  long N;
  double tau;
  double mu;              /* > 0: constant dynamic viscosity (R13) */
  int force_order, include_sigma;
  int bc[3];
  double Tw[3][2];        /* wall temperature, [axis][0 = low, 1 = high] */
  double fw[3][2][ORC_QMAX]; /* f0_i(1, 0, T_wall) per wall */
  double fw_in[3][2];     /* sum of fw over the incoming slots of one column */
  double *g;              /* D * N acceleration field */
  double *f;              /* Q * N post-collision state */
  double *fn;             /* Q * N scratch for the next state */
  double *rho_w;          /* 2 * (N / n_wall) wall densities of the current step */
  int wall_axis;          /* -1 if fully periodic */
  unsigned char *solid;   /* N flags (R15), NULL without solid sites */
  double *E_solid;        /* Q * N: f0_i(1, 0, T_wall) at solid sites */
  double *rho_ws;         /* N wall densities of the fluid sites of the current step */
} orc_sim;

static long site_index(const orc_sim *S, const int *x) {
  return x[0] + (long)S->n[0] * (x[1] + (long)S->n[1] * x[2]);
}

static void site_coords(const orc_sim *S, long s, int *x) {
  x[0] = (int)(s % S->n[0]);
  x[1] = (int)((s / S->n[0]) % S->n[1]);
  x[2] = (int)(s / ((long)S->n[0] * S->n[1]));
}

static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* Column index of a site: its coordinates other than the wall axis. */
static long column_of(const orc_sim *S, const int *x) {
  long col = 0, stride = 1;
  for (int a = 0; a < 3; ++a) {
    if (a == S->wall_axis) continue;
    col += stride * x[a];
    stride *= S->n[a];
  }
  return col;
}

void orc_destroy(void *h) {
  orc_sim *S = (orc_sim *)h;
  if (!S) return;
  free(S->g); free(S->f); free(S->fn); free(S->rho_w);
  free(S->solid); free(S->E_solid); free(S->rho_ws);
  free(S);
}

void *orc_create(int lat, int nx, int ny, int nz, double tau, double mu, int force_order,
                 int include_sigma, const int *bc, const double *T_lo, const double *T_hi,
                 const double *g) {
  orc_sim *S = (orc_sim *)calloc(1, sizeof(orc_sim));
  if (!S) return NULL;
  if (orc_lattice_build(lat, &S->L)) { free(S); return NULL; }
  int D = S->L.D;
  if (D == 2) nz = 1;
  S->n[0] = nx; S->n[1] = ny; S->n[2] = nz;
  if (nx < 1 || ny < 1 || nz < 1 || tau <= 0.5 || force_order < 0 || force_order > 3) {
    free(S);
    return NULL;
  }
  S->N = (long)nx * ny * nz;
  S->tau = tau;
  S->mu = mu > 0.0 ? mu : 0.0;
  S->force_order = force_order;
  S->include_sigma = include_sigma;
  S->wall_axis = -1;
  for (int a = 0; a < 3; ++a) {
    S->bc[a] = (bc && a < D) ? bc[a] : ORC_PERIODIC;
    S->Tw[a][0] = T_lo ? T_lo[a] : 1.0;
    S->Tw[a][1] = T_hi ? T_hi[a] : 1.0;
    if (S->bc[a] != ORC_PERIODIC) {
      if (S->wall_axis >= 0 || S->n[a] < 6) { free(S); return NULL; }
      S->wall_axis = a;
    }
  }
  if (S->wall_axis >= 0) {
    int a = S->wall_axis;
    double zero[3] = {0, 0, 0};
    for (int side = 0; side < 2; ++side) {
      equilibrium(&S->L, S->L.neq, 1.0, zero, S->Tw[a][side], S->fw[a][side]);
      double s = 0.0;
      for (int i = 0; i < S->L.Q; ++i) {
        int e = S->L.e[i][a];
        int cnt = side == 0 ? (e > 0 ? e : 0) : (e < 0 ? -e : 0); /* slots per column */
        s += cnt * S->fw[a][side][i];
      }
      S->fw_in[a][side] = s;
    }
  }
  S->g = (double *)malloc(sizeof(double) * D * S->N);
  S->f = (double *)calloc((size_t)S->L.Q * S->N, sizeof(double));
  S->fn = (double *)calloc((size_t)S->L.Q * S->N, sizeof(double));
  S->rho_w = (double *)calloc(2 * (size_t)S->N, sizeof(double));
  if (!S->g || !S->f || !S->fn || !S->rho_w) { orc_destroy(S); return NULL; }
  for (long k = 0; k < (long)D * S->N; ++k) S->g[k] = g ? g[k] : 0.0;
  return S;
}

static long neighbour(const orc_sim *S, const int *x, const int *e, int sign) {
  int y[3];
  for (int a = 0; a < 3; ++a) y[a] = wrap(x[a] + sign * e[a], S->n[a]);
  return site_index(S, y);
}

/* Solid sites (R15, fully periodic grids only): solid[s] != 0 marks a wall
 * site at temperature T[s].  Must precede orc_init.                        */
int orc_set_solid(void *h, const unsigned char *solid, const double *T) {
  orc_sim *S = (orc_sim *)h;
  if (S->wall_axis >= 0 || !solid || !T) return -1;
  const int Q = S->L.Q;
  S->solid = (unsigned char *)malloc((size_t)S->N);
  S->E_solid = (double *)calloc((size_t)Q * S->N, sizeof(double));
  S->rho_ws = (double *)calloc((size_t)S->N, sizeof(double));
  if (!S->solid || !S->E_solid || !S->rho_ws) return -1;
  double zero[3] = {0, 0, 0};
  for (long k = 0; k < S->N; ++k) {
    S->solid[k] = solid[k] ? 1 : 0;
    if (S->solid[k]) equilibrium(&S->L, S->L.neq, 1.0, zero, T[k], S->E_solid + (size_t)k * Q);
  }
  return 0;
}

/* Wall densities of the solid sites' diffuse walls (R15): at a fluid site x,
 * rho_w(x) = (mass of the slots of x about to move into solid sites) / (mass
 * of f0(1, 0, T_wall) over the slots of x pulled from solid sites).       */
static void solid_densities(orc_sim *S, const double *f) {
  const int Q = S->L.Q;
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S->N; ++s) {
    S->rho_ws[s] = 0.0;
    if (S->solid[s]) continue;
    int x[3];
    site_coords(S, s, x);
    double out = 0.0, in = 0.0;
    for (int i = 0; i < Q; ++i) {
      long src = neighbour(S, x, S->L.e[i], -1);
      if (!S->solid[src]) continue;
      out += f[(long)S->L.opp[i] * S->N + s];
      in += S->E_solid[(size_t)src * Q + i];
    }
    if (in > 0.0) S->rho_ws[s] = out / in;
  }
}

/* Wall densities of the thermal (diffuse) wall for the state f: per column and
 * side, rho_w = (mass of the slots about to leave through that wall) / (mass
 * of f0(1, 0, T_wall) over the slots the wall fills).                      */
static void wall_densities(orc_sim *S, const double *f) {
  if (S->solid) solid_densities(S, f);
  int a = S->wall_axis;
  if (a < 0 || S->bc[a] != ORC_THERMAL_WALL) return;
  long ncol = S->N / S->n[a];
  for (long k = 0; k < 2 * ncol; ++k) S->rho_w[k] = 0.0;
  for (long s = 0; s < S->N; ++s) {
    int x[3];
    site_coords(S, s, x);
    long col = column_of(S, x);
    for (int j = 0; j < S->L.Q; ++j) {
      int dst = x[a] + S->L.e[j][a];
      if (dst < 0) S->rho_w[col] += f[j * S->N + s];
      else if (dst >= S->n[a]) S->rho_w[ncol + col] += f[j * S->N + s];
    }
  }
  for (long k = 0; k < ncol; ++k) {
    S->rho_w[k] /= S->fw_in[a][0];
    S->rho_w[ncol + k] /= S->fw_in[a][1];
  }
}

/* Pull of slot (x, i): f~_i(x) = f*_i(x - e_i) with the boundary rules. */
static double pull(const orc_sim *S, const double *f, const int *x, int i) {
  int src[3];
  int wa = -1, side = 0;
  for (int a = 0; a < 3; ++a) {
    src[a] = x[a] - S->L.e[i][a];
    if (src[a] < 0 || src[a] >= S->n[a]) {
      if (S->bc[a] == ORC_PERIODIC) {
        src[a] = wrap(src[a], S->n[a]);
      } else {
        wa = a;
        side = src[a] < 0 ? 0 : 1;
      }
    }
  }
  if (wa < 0) {
    long k = site_index(S, src);
    if (S->solid && S->solid[k]) return S->rho_ws[site_index(S, x)] * S->E_solid[(size_t)k * S->L.Q + i];
    return f[i * S->N + k];
  }
  if (S->bc[wa] == ORC_BOUNCE_BACK) {
    int m[3] = {x[0], x[1], x[2]};
    m[wa] = side == 0 ? S->L.e[i][wa] - 1 - x[wa] : 2 * S->n[wa] - 1 - (x[wa] - S->L.e[i][wa]);
    return f[S->L.opp[i] * S->N + site_index(S, m)];
  }
  long ncol = S->N / S->n[wa];
  return S->rho_w[side * ncol + column_of(S, x)] * S->fw[wa][side][i];
}

/* The slot of the post-collision state that the pull of (x, i) reads, for the
 * periodic and bounce-back maps (used to place the initial state, R11).     */
static long pull_source(const orc_sim *S, const int *x, int i) {
  int src[3];
  for (int a = 0; a < 3; ++a) {
    src[a] = x[a] - S->L.e[i][a];
    if (src[a] < 0 || src[a] >= S->n[a]) {
      if (S->bc[a] == ORC_PERIODIC) {
        src[a] = wrap(src[a], S->n[a]);
      } else {
        int m[3] = {x[0], x[1], x[2]};
        m[a] = src[a] < 0 ? S->L.e[i][a] - 1 - x[a] : 2 * S->n[a] - 1 - src[a];
        return S->L.opp[i] * S->N + site_index(S, m);
      }
    }
  }
  return i * S->N + site_index(S, src);
}

typedef struct {
  double rho, u[3], theta;
} orc_state;

/* Moments of the pulled f~ and the mid-point state (Eq. rut1 and R1). */
static orc_state midpoint(const orc_lattice *L, const double *ft, const double *g) {
  orc_state m;
  double rho = 0.0, j[3] = {0, 0, 0}, K = 0.0;
  for (int i = 0; i < L->Q; ++i) {
    rho += ft[i];
    double x2 = 0.0;
    for (int a = 0; a < L->D; ++a) {
      j[a] += ft[i] * L->xi[i][a];
      x2 += L->xi[i][a] * L->xi[i][a];
    }
    K += ft[i] * x2;
  }
  double ut2 = 0.0, g2 = 0.0;
  m.rho = rho;
  for (int a = 0; a < 3; ++a) m.u[a] = 0.0;
  for (int a = 0; a < L->D; ++a) {
    double ut = j[a] / rho;
    ut2 += ut * ut;
    g2 += g[a] * g[a];
    m.u[a] = ut + 0.5 * g[a];
  }
  m.theta = (K / rho - ut2) / L->D + g2 / (4.0 * L->D);
  return m;
}

/* sigma-bar (R8). */
static void sigma_bar(const orc_lattice *L, double tau, const double *ft, const double *feq,
                      const double *u, double *sig) {
  int D = L->D;
  for (int k = 0; k < D * D; ++k) sig[k] = 0.0;
  for (int i = 0; i < L->Q; ++i) {
    double c[3];
    for (int a = 0; a < D; ++a) c[a] = L->xi[i][a] - u[a];
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) sig[a * D + b] += (ft[i] - feq[i]) * c[a] * c[b];
  }
  for (int k = 0; k < D * D; ++k) sig[k] *= -(1.0 - 0.5 / tau);
}

/* The collision divisor tau-hat at a site (R2 / R13). */
static double site_tau(const orc_sim *S, const orc_state *m) {
  return S->mu > 0.0 ? S->mu / (m->rho * m->theta) + 0.5 : S->tau;
}

/* One site of Eq. lbm given the pulled f~ (Q values) and g at the site. */
static void collide(const orc_sim *S, const double *ft, const double *g, double *out,
                    orc_state *ms, double *feq_out, double *F_out, double *sig_out) {
  const orc_lattice *L = &S->L;
  double feq[ORC_QMAX], F[ORC_QMAX], sig[9];
  orc_state m = midpoint(L, ft, g);
  const double tau = site_tau(S, &m);
  equilibrium(L, L->neq, m.rho, m.u, m.theta, feq);
  const double *sp = NULL;
  if (S->include_sigma) {
    sigma_bar(L, tau, ft, feq, m.u, sig);
    sp = sig;
  } else {
    for (int k = 0; k < 9; ++k) sig[k] = 0.0;
  }
  force(L, S->force_order, m.rho, m.u, m.theta, g, sp, F);
  if (out)
    for (int i = 0; i < L->Q; ++i)
      out[i] = ft[i] - (ft[i] - feq[i]) / tau + (1.0 - 0.5 / tau) * F[i];
  if (ms) *ms = m;
  if (feq_out) memcpy(feq_out, feq, sizeof(double) * L->Q);
  if (F_out) memcpy(F_out, F, sizeof(double) * L->Q);
  if (sig_out) memcpy(sig_out, sig, sizeof(double) * L->D * L->D);
}

int orc_init(void *h, const double *rho, const double *u, const double *T) {
  orc_sim *S = (orc_sim *)h;
  const orc_lattice *L = &S->L;
  int D = L->D;
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S->N; ++s) {
    if (S->solid && S->solid[s]) continue;
    int x[3];
    double uu[3] = {0, 0, 0}, gg[3] = {0, 0, 0}, feq[ORC_QMAX], F[ORC_QMAX];
    site_coords(S, s, x);
    for (int a = 0; a < D; ++a) {
      uu[a] = u[a * S->N + s];
      gg[a] = S->g[a * S->N + s];
    }
    equilibrium(L, L->neq, rho[s], uu, T[s], feq);
    force(L, S->force_order, rho[s], uu, T[s], gg, NULL, F);
    for (int i = 0; i < L->Q; ++i) {
      if (S->solid && S->solid[neighbour(S, x, L->e[i], -1)]) {
        /* pulled from a solid site: the wall emits it; the slot the wall
         * absorbs (the opposite direction, at x) holds the local value */
        S->f[(long)L->opp[i] * S->N + s] = feq[L->opp[i]] - 0.5 * F[L->opp[i]];
        continue;
      }
      S->f[pull_source(S, x, i)] = feq[i] - 0.5 * F[i];
    }
  }
  return 0;
}

static void gather(const orc_sim *S, const double *f, long s, double *ft, double *g) {
  int x[3];
  site_coords(S, s, x);
  for (int i = 0; i < S->L.Q; ++i) ft[i] = pull(S, f, x, i);
  for (int a = 0; a < 3; ++a) g[a] = a < S->L.D ? S->g[a * S->N + s] : 0.0;
}

int orc_step(void *h, int nsteps) {
  orc_sim *S = (orc_sim *)h;
  for (int t = 0; t < nsteps; ++t) {
    wall_densities(S, S->f);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < S->N; ++s) {
      double ft[ORC_QMAX], out[ORC_QMAX], g[3];
      if (S->solid && S->solid[s]) continue;
      gather(S, S->f, s, ft, g);
      collide(S, ft, g, out, NULL, NULL, NULL, NULL);
      for (int i = 0; i < S->L.Q; ++i) S->fn[i * S->N + s] = out[i];
    }
    double *tmp = S->f;
    S->f = S->fn;
    S->fn = tmp;
  }
  return 0;
}

/* One step evaluated only at the listed sites, from an explicit state (Q*N,
 * the oracle's velocity order).  out is nsites*Q, site-major.             */
int orc_step_sites(void *h, const double *state, const long *sites, long nsites, double *out) {
  orc_sim *S = (orc_sim *)h;
  memcpy(S->fn, state, sizeof(double) * S->L.Q * S->N);
  wall_densities(S, S->fn);
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nsites; ++k) {
    double ft[ORC_QMAX], g[3];
    gather(S, S->fn, sites[k], ft, g);
    collide(S, ft, g, out + k * S->L.Q, NULL, NULL, NULL, NULL);
  }
  return 0;
}

/* Physical mid-point moments rho, u (D*N), T (N), heat flux q (D*N, R9) and,
 * optionally, sigma-bar (D*D*N) of the current state.  Any output may be NULL. */
int orc_moments(void *h, double *rho, double *u, double *T, double *q, double *sigma) {
  orc_sim *S = (orc_sim *)h;
  const orc_lattice *L = &S->L;
  int D = L->D;
  wall_densities(S, S->f);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S->N; ++s) {
    double ft[ORC_QMAX], g[3], feq[ORC_QMAX], F[ORC_QMAX], sig[9];
    orc_state m;
    if (S->solid && S->solid[s]) {  /* solid sites report zeros */
      if (rho) rho[s] = 0.0;
      if (T) T[s] = 0.0;
      for (int a = 0; a < D; ++a) {
        if (u) u[a * S->N + s] = 0.0;
        if (q) q[a * S->N + s] = 0.0;
      }
      if (sigma)
        for (int k = 0; k < D * D; ++k) sigma[(long)k * S->N + s] = 0.0;
      continue;
    }
    gather(S, S->f, s, ft, g);
    collide(S, ft, g, NULL, &m, feq, F, sig);
    if (rho) rho[s] = m.rho;
    if (T) T[s] = m.theta;
    for (int a = 0; a < D; ++a)
      if (u) u[a * S->N + s] = m.u[a];
    if (q) {
      double qq[3] = {0, 0, 0};
      for (int i = 0; i < L->Q; ++i) {
        double c[3], c2 = 0.0;
        for (int a = 0; a < D; ++a) {
          c[a] = L->xi[i][a] - m.u[a];
          c2 += c[a] * c[a];
        }
        double fneq = ft[i] - feq[i] + 0.5 * F[i];
        for (int a = 0; a < D; ++a) qq[a] += fneq * c2 * c[a];
      }
      for (int a = 0; a < D; ++a) q[a * S->N + s] = 0.5 * (1.0 - 0.5 / site_tau(S, &m)) * qq[a];
    }
    if (sigma) {
      if (!S->include_sigma) sigma_bar(L, site_tau(S, &m), ft, feq, m.u, sig);
      for (int k = 0; k < D * D; ++k) sigma[(long)k * S->N + s] = sig[k];
    }
  }
  return 0;
}

int orc_get_state(void *h, double *f) {
  orc_sim *S = (orc_sim *)h;
  memcpy(f, S->f, sizeof(double) * S->L.Q * S->N);
  return 0;
}

int orc_set_state(void *h, const double *f) {
  orc_sim *S = (orc_sim *)h;
  memcpy(S->f, f, sizeof(double) * S->L.Q * S->N);
  return 0;
}

/* The pulled (pre-collision) distribution f~ of the current state, Q*N. */
int orc_pull_state(void *h, double *ft) {
  orc_sim *S = (orc_sim *)h;
  wall_densities(S, S->f);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S->N; ++s) {
    int x[3];
    site_coords(S, s, x);
    const int solid = S->solid && S->solid[s];
    for (int i = 0; i < S->L.Q; ++i) ft[i * S->N + s] = solid ? 0.0 : pull(S, S->f, x, i);
  }
  return 0;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
