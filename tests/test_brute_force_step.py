"""Brute-force pin of one oracle step on tiny grids.

The update of Eq. lbm is recomputed here in numpy from the definitions, by a
route that shares nothing with the oracle's tensor code:

* the Hermite equilibrium in product form.  A Maxwellian factorises over the
  axes, so its Hermite coefficients are products of 1-D ones; for X normal
  with mean u and variance theta the generating function
  E[exp(X t - t^2/2)] = exp(u t + (theta - 1) t^2 / 2) gives
  E[He_n(X)] = sum_k n! / (k! (n - 2k)! 2^k) (theta - 1)^k u^(n - 2k),
  and f0_i = w_i rho sum_{|m| <= N_eq} prod_a E[He_{m_a}] He_{m_a}(xi_ia) / m_a!;
* the force F = -g . grad_xi f_N of Eq. F by an index shift (Rodrigues):
  -d/dxi_a [omega He_m] = omega He_{m + e_a}, so
  F_i = w_i rho sum_a g_a sum_{|m| <= N} prod_b E[He_{m_b}] / m_b! He_{m + e_a}(xi_i);
* the mid-point state of Sec. 2 (u = j / rho + g / 2, theta with the g^2 / 4D
  term) and the pull with the wall rules written as loops over sites and
  directions: half-way bounce-back in the same column, the diffuse thermal
  wall that re-emits, per column, the mass leaving through the wall as a
  wall Maxwellian, and solid sites that do the same per fluid site;
* optionally the sigma-bar terms (subtracted from the second-order
  coefficients of the force) and the constant-viscosity relaxation time.

Everything is FP64 on both sides; only the summation order differs.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2302_04741_gb300 import workloads as W

from numpy.polynomial import hermite_e as He


def he(n, x):
    """Probabilists' Hermite polynomial He_n at x (numpy's coefficients)."""
    c = np.zeros(n + 1)
    c[n] = 1.0
    return He.hermeval(x, c)


def he_mean(n, u, theta):
    """E[He_n(X)] for X normal with mean u and variance theta."""
    return sum(math.factorial(n) / (math.factorial(k) * math.factorial(n - 2 * k) * 2 ** k)
               * (theta - 1.0) ** k * u ** (n - 2 * k) for k in range(n // 2 + 1))


def multi_indices(D, nmax):
    return [m for m in itertools.product(range(nmax + 1), repeat=D) if sum(m) <= nmax]


def feq_product(xi, w, rho, u, theta, neq):
    D = xi.shape[1]
    out = np.zeros(len(w))
    for m in multi_indices(D, neq):
        coef = rho * np.prod([he_mean(m[a], u[a], theta) / math.factorial(m[a]) for a in range(D)])
        out += coef * np.prod([he(m[a], xi[:, a]) for a in range(D)], axis=0)
    return w * out


def force_shift(xi, w, rho, u, theta, g, order, sigma=None):
    """sigma (D x D): the non-equilibrium stress, subtracted from the
    second-order coefficients (a^(2) = a^(2)_0 - sigma-bar, Eq. f2)."""
    D = xi.shape[1]
    out = np.zeros(len(w))
    for m in multi_indices(D, order):
        coef = rho * np.prod([he_mean(m[b], u[b], theta) / math.factorial(m[b]) for b in range(D)])
        if sigma is not None and sum(m) == 2:
            ab = [b for b in range(D) for _ in range(m[b])]        # the tensor index pair
            coef -= sigma[ab[0], ab[1]] / np.prod([math.factorial(m[b]) for b in range(D)])
        for a in range(D):
            mm = list(m)
            mm[a] += 1
            out += g[a] * coef * np.prod([he(mm[b], xi[:, b]) for b in range(D)], axis=0)
    return w * out


def brute_step(fstar, lat, shape, tau, g, order, bc_wall=0, T_lo=1.0, T_hi=1.0, solid=None,
               T_wall=None, sigma=False, mu=0.0):
    """One step of Eq. lbm from the post-collision state fstar (Q, N).
    bc_wall: 0 periodic, 1 bounce-back, 2 thermal wall on the last axis.
    solid (N flags) with T_wall (N): staircase diffuse walls on a periodic
    grid -- a fluid site re-emits the mass it sends into solid sites as wall
    Maxwellians at the temperatures of the solid sites it pulls from.
    sigma: the force's second-order coefficients less the non-equilibrium
    stress sigma-bar = -(1 - 1/(2 tau)) sum (f~ - f0)(xi - u)(xi - u);
    mu > 0: each site relaxes with tau-hat = mu / (rho theta) + 1/2."""
    D, Q, c, e, w, neq = oracle.lattice_info(lat)
    e = e[:, :D]
    xi = c * e.astype(float)
    n = list(shape[:D])
    A = D - 1                                     # wall axis
    opp = [int(np.flatnonzero((e == -e[i]).all(axis=1))[0]) for i in range(Q)]
    strides = [1, shape[0], shape[0] * shape[1]][:D]

    def site(x):
        return sum(x[a] * strides[a] for a in range(D))

    # wall densities per column (thermal wall): emitted mass / emitted shape
    rho_w = {}
    if bc_wall == 2:
        for side, Tw in ((0, T_lo), (1, T_hi)):
            f0w = feq_product(xi, w, 1.0, np.zeros(D), Tw, neq)
            den = sum((e[i, A] if side == 0 else -e[i, A]) * f0w[i]
                      for i in range(Q) if (e[i, A] > 0 if side == 0 else e[i, A] < 0))
            for col in itertools.product(*[range(n[a]) for a in range(A)]):
                leave = 0.0
                for r in range(3):
                    row = r if side == 0 else n[A] - 1 - r
                    for j in range(Q):
                        dest = row + e[j, A]
                        if (side == 0 and dest < 0) or (side == 1 and dest >= n[A]):
                            leave += fstar[j, site(list(col) + [row])]
                rho_w[(side, col)] = (leave / den, f0w)
    N = fstar.shape[1]
    out = np.zeros_like(fstar)
    gg = np.asarray(g).reshape(D, N)
    for x in itertools.product(*[range(k) for k in n]):
        x = list(x)
        s = site(x)
        if solid is not None and solid[s]:
            continue
        ft = np.zeros(Q)
        if solid is not None:
            from_solid = [i for i in range(Q)
                          if solid[site([(x[a] - e[i, a]) % n[a] for a in range(D)])]]
            emitted = {}
            for i in from_solid:
                y = site([(x[a] - e[i, a]) % n[a] for a in range(D)])
                emitted[i] = feq_product(xi, w, 1.0, np.zeros(D), T_wall[y], neq)[i]
            if from_solid:
                sent = sum(fstar[opp[i], s] for i in from_solid)
                rw = sent / sum(emitted.values())
        for i in range(Q):
            src = [x[a] - e[i, a] for a in range(D)]
            if solid is not None and i in emitted:
                ft[i] = rw * emitted[i]
            elif 0 <= src[A] < n[A] or bc_wall == 0:
                ft[i] = fstar[i, site([src[a] % n[a] for a in range(D)])]
            elif bc_wall == 1:
                # half-way bounce-back: the opposite population, same column
                mir = e[i, A] - 1 - x[A] if src[A] < 0 else 2 * n[A] - 1 - src[A]
                ft[i] = fstar[opp[i], site(x[:A] + [mir])]
            else:
                side = 0 if src[A] < 0 else 1
                rw, f0w = rho_w[(side, tuple(x[:A]))]
                ft[i] = rw * f0w[i]
        gs = gg[:, s]
        rho = ft.sum()
        ut = ft @ xi / rho
        u = ut + 0.5 * gs
        theta = ((ft @ np.sum(xi * xi, axis=1)) / rho - ut @ ut) / D + gs @ gs / (4 * D)
        f0 = feq_product(xi, w, rho, u, theta, neq)
        tau_s = mu / (rho * theta) + 0.5 if mu > 0 else tau
        sig = None
        if sigma:
            cc = xi - u
            sig = -(1.0 - 0.5 / tau_s) * np.einsum("i,ia,ib->ab", ft - f0, cc, cc)
        F = force_shift(xi, w, rho, u, theta, gs, order, sig)
        out[:, s] = ft - (ft - f0) / tau_s + (1.0 - 0.5 / tau_s) * F
    return out


def start_state(lat, shape, seed, bc, T_lo, T_hi, g, order, tau):
    """A non-trivial post-collision state: smooth random fields, two oracle steps."""
    D = W.dims(lat)
    N = int(np.prod(shape))
    rho = 1.0 + 0.02 * (W.uniform(seed, 1, N) - 0.5)
    u = 0.06 * (W.uniform(seed, 2, D * N).reshape(D, N) - 0.5)
    T = 1.0 + 0.08 * (W.uniform(seed, 3, N) - 0.5)
    sim = oracle.OracleSim(lat, *shape, tau, g, force_order=order, bc=bc, T_lo=T_lo, T_hi=T_hi)
    sim.init(rho, u, T)
    sim.step(2)
    return sim


CASES = [
    # lattice, shape, force order, wall rule on the last axis
    (oracle.D2Q37, (4, 4, 1), 2, 0),
    (oracle.D2Q37, (5, 3, 1), 1, 0),
    (oracle.D2Q37, (4, 4, 1), 0, 0),
    (oracle.D2Q37, (5, 7, 1), 2, 1),
    (oracle.D2Q37, (4, 7, 1), 2, 2),
    (oracle.D3Q39, (4, 3, 4), 2, 0),
    (oracle.D3Q39, (3, 4, 6), 1, 1),
    (oracle.D3Q39, (3, 3, 7), 2, 2),
]


@pytest.mark.parametrize("lat,shape,order,wall", CASES)
def test_one_step_equals_brute_force(lat, shape, order, wall):
    D = W.dims(lat)
    N = int(np.prod(shape))
    tau = 0.85
    g = 0.01 * (W.uniform(41, 4, D * N).reshape(D, N) - 0.5)
    bc = [0, 0, 0]
    T_lo, T_hi = [1.0, 1.0, 1.0], [1.0, 1.0, 1.0]
    if wall:
        bc[D - 1] = wall
        T_lo[D - 1], T_hi[D - 1] = 1.04, 0.97
    sim = start_state(lat, shape, 40 + order, bc, T_lo, T_hi, g, order, tau)
    fstar = sim.get_state()
    ref = brute_step(fstar, lat, shape, tau, g, order, wall, T_lo[D - 1], T_hi[D - 1])
    sim.step(1)
    got = sim.get_state()
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-15)
    # the update moved the state: the comparison is not of two copies
    assert np.max(np.abs(got - fstar)) > 1e-4


@pytest.mark.parametrize("lat,shape", [(oracle.D2Q37, (9, 8, 1)), (oracle.D3Q39, (6, 5, 7))])
def test_one_step_with_solid_sites_equals_brute_force(lat, shape):
    """The staircase diffuse wall of solid sites (periodic grid): a solid
    block with a per-site wall temperature, one step from a stepped state;
    fluid sites compared (solid sites hold no populations)."""
    D = W.dims(lat)
    N = int(np.prod(shape))
    nx, ny, nz = shape
    tau, order = 0.9, 2
    g = 0.01 * (W.uniform(43, 4, D * N).reshape(D, N) - 0.5)
    idx = np.arange(N)
    x, y, z = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    solid = ((x >= 2) & (x <= 4) & (y >= 3) & (y <= 5)).astype(np.uint8)
    if D == 3:
        solid &= ((z >= 1) & (z <= 3)).astype(np.uint8)
    T_wall = 1.0 + 0.05 * (W.uniform(43, 5, N) - 0.5)
    rho = 1.0 + 0.02 * (W.uniform(44, 1, N) - 0.5)
    u = 0.06 * (W.uniform(44, 2, D * N).reshape(D, N) - 0.5)
    T = 1.0 + 0.08 * (W.uniform(44, 3, N) - 0.5)
    sim = oracle.OracleSim(lat, *shape, tau, g, force_order=order)
    sim.set_solid(solid, T_wall)
    sim.init(rho, u, T)
    sim.step(2)
    fstar = sim.get_state()
    ref = brute_step(fstar, lat, shape, tau, g, order, solid=solid, T_wall=T_wall)
    sim.step(1)
    got = sim.get_state()
    fluid = solid == 0
    np.testing.assert_allclose(got[:, fluid], ref[:, fluid], rtol=0, atol=2e-15)
    assert np.max(np.abs(got[:, fluid] - fstar[:, fluid])) > 1e-4


@pytest.mark.parametrize("lat,shape,wall,sigma,mu", [
    (oracle.D2Q37, (5, 4, 1), 0, True, 0.0),
    (oracle.D2Q37, (4, 7, 1), 2, False, 0.05),
    (oracle.D2Q37, (4, 7, 1), 2, True, 0.05),
    (oracle.D3Q39, (4, 3, 4), 0, True, 0.08),
])
def test_one_step_with_sigma_and_constant_mu_equals_brute_force(lat, shape, wall, sigma, mu):
    """The sigma-bar terms of Eq. fi (R8: sigma-bar from the pulled f~ about
    the mid-point velocity, entering the second-order coefficients of the
    n = 3 force term) and the constant-viscosity relaxation (R13:
    tau-hat = mu / (rho theta) + 1/2 per site), in the same restatement."""
    D = W.dims(lat)
    N = int(np.prod(shape))
    tau, order = 0.85, 2
    g = 0.01 * (W.uniform(45, 4, D * N).reshape(D, N) - 0.5)
    bc = [0, 0, 0]
    T_lo, T_hi = [1.0, 1.0, 1.0], [1.0, 1.0, 1.0]
    if wall:
        bc[D - 1] = wall
        T_lo[D - 1], T_hi[D - 1] = 1.04, 0.97
    rho = 1.0 + 0.02 * (W.uniform(46, 1, N) - 0.5)
    u = 0.06 * (W.uniform(46, 2, D * N).reshape(D, N) - 0.5)
    T = 1.0 + 0.08 * (W.uniform(46, 3, N) - 0.5)
    sim = oracle.OracleSim(lat, *shape, tau, g, force_order=order, include_sigma=sigma, bc=bc,
                           T_lo=T_lo, T_hi=T_hi, mu=mu)
    sim.init(rho, u, T)
    sim.step(2)
    fstar = sim.get_state()
    ref = brute_step(fstar, lat, shape, tau, g, order, wall, T_lo[D - 1], T_hi[D - 1],
                     sigma=sigma, mu=mu)
    sim.step(1)
    got = sim.get_state()
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-15)
    assert np.max(np.abs(got - fstar)) > 1e-4


@pytest.mark.parametrize("lat,shape,order,mu", [
    (oracle.D2Q37, (4, 4, 1), 2, 0.0),
    (oracle.D2Q37, (5, 3, 1), 1, 0.0),
    (oracle.D2Q37, (4, 4, 1), 0, 0.05),
    (oracle.D3Q39, (4, 3, 4), 2, 0.08),
])
def test_moments_equal_brute_force(lat, shape, order, mu):
    """The diagnostics of the oracle (rho, u, T at the mid-point, R1, and the
    heat flux of R9, q = 1/2 (1 - 1/(2 tau)) sum (f~ - f0 + F/2) |xi - u|^2
    (xi - u)) recomputed from the pulled state by the same product-form
    equilibrium and index-shift force."""
    D, Q, c, e, w, neq = oracle.lattice_info(lat)
    xi = c * e[:, :D].astype(float)
    N = int(np.prod(shape))
    tau = 0.85
    g = 0.01 * (W.uniform(47, 4, D * N).reshape(D, N) - 0.5)
    rho0 = 1.0 + 0.02 * (W.uniform(48, 1, N) - 0.5)
    u0 = 0.06 * (W.uniform(48, 2, D * N).reshape(D, N) - 0.5)
    T0 = 1.0 + 0.08 * (W.uniform(48, 3, N) - 0.5)
    sim = oracle.OracleSim(lat, *shape, tau, g, force_order=order, mu=mu)
    sim.init(rho0, u0, T0)
    sim.step(3)
    ft = sim.pulled()
    rho, u, T, q = sim.moments()
    for s in range(N):
        f = ft[:, s]
        r = f.sum()
        ut = f @ xi / r
        uu = ut + 0.5 * g[:, s]
        th = ((f @ np.sum(xi * xi, axis=1)) / r - ut @ ut) / D + g[:, s] @ g[:, s] / (4 * D)
        tau_s = mu / (r * th) + 0.5 if mu > 0 else tau
        f0 = feq_product(xi, w, r, uu, th, neq)
        F = force_shift(xi, w, r, uu, th, g[:, s], order)
        cc = xi - uu
        qq = 0.5 * (1.0 - 0.5 / tau_s) * ((f - f0 + 0.5 * F) * np.sum(cc * cc, axis=1)) @ cc
        assert abs(rho[s] - r) < 1e-15 and abs(T[s] - th) < 1e-15
        np.testing.assert_allclose(u[:, s], uu, rtol=0, atol=1e-16)
        np.testing.assert_allclose(q[:, s], qq, rtol=0, atol=1e-15)
