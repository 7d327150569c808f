"""Slot-level pins of the wall rules (reading R10) on the CPU oracle.

With the collision switched off (tau-hat = 1e12, so 1/tau-hat = 1e-12, and
no force) a step is the streaming of Eq. lbm plus the wall rule alone:
  * half-way bounce-back is then a permutation of the stored slots that must
    be micro-reversible: stepping, reversing every velocity (slot i <-> -i),
    stepping again and reversing once more restores the state exactly -- an
    off-by-one mirror row or a wrong column breaks this;
  * the diffuse thermal wall fills the slots it owns with
    rho_w f0_i(1, 0, T_wall), rho_w set by the column's mass balance; for a
    fluid at rest at T = 1 (f = w) that is the closed form
    rho_w = sum_{e_ia < 0} |e_ia| w_i / sum_{e_ia > 0} e_ia f0_i(1, 0, T_wall)
    (mass leaving the column through the wall over the Maxwellian mass of
    the slots the wall refills), with f0 the pinned Hermite equilibrium.
"""
import numpy as np
import pytest

import oracle

TAU_OFF = 1e12


def setup(lat, shape, bc, T_lo=(1.0, 1.0, 1.0), T_hi=(1.0, 1.0, 1.0)):
    D, Q, c, e, w, neq = oracle.lattice_info(lat)
    nx, ny, nz = shape
    N = nx * ny * nz
    sim = oracle.OracleSim(lat, nx, ny, nz, TAU_OFF, np.zeros((D, N)), bc=bc, T_lo=T_lo, T_hi=T_hi)
    return sim, D, Q, e, w, N


def opposite(e):
    idx = {tuple(v): k for k, v in enumerate(e)}
    return np.array([idx[tuple(-v)] for v in e])


@pytest.mark.parametrize("lat,shape", [(0, (9, 10, 1)), (1, (5, 6, 9))])
def test_bounce_back_streaming_is_micro_reversible(lat, shape):
    D = oracle.lattice_info(lat)[0]
    bc = (0, 1) if D == 2 else (0, 0, 1)
    sim, D, Q, e, w, N = setup(lat, shape, bc)
    rng = np.random.default_rng(7)
    f0 = w[:, None] * (1.0 + 0.01 * rng.standard_normal((Q, N)))
    opp = opposite(e)
    sim.set_state(f0)
    sim.step(4)  # every particle within 3 rows of a wall meets it
    moved = sim.get_state()
    assert np.max(np.abs(moved - f0)) > 1e-4  # the state did move
    sim.set_state(moved[opp])
    sim.step(4)
    back = sim.get_state()[opp]
    assert np.max(np.abs(back - f0)) <= 1e-12, np.max(np.abs(back - f0))


@pytest.mark.parametrize("lat,shape", [(0, (6, 12, 1)), (1, (4, 5, 12))])
def test_thermal_wall_refills_with_the_wall_maxwellian(lat, shape):
    D = oracle.lattice_info(lat)[0]
    bc = (0, 2) if D == 2 else (0, 0, 2)
    T_lo, T_hi = 1.1, 0.92
    Tl = (1.0, T_lo, 1.0) if D == 2 else (1.0, 1.0, T_lo)
    Th = (1.0, T_hi, 1.0) if D == 2 else (1.0, 1.0, T_hi)
    sim, D, Q, e, w, N = setup(lat, shape, bc, Tl, Th)
    sim.set_state(np.repeat(w[:, None], N, axis=1))  # rest, rho = 1, T = 1: f = w
    sim.step(1)
    f = sim.get_state().reshape(Q, *shape[::-1])  # [Q][z][y][x]
    a = D - 1  # wall axis
    nA = shape[a]
    eA = e[:, a]
    for side, Tw in ((0, T_lo), (1, T_hi)):
        f0 = oracle.equilibrium(lat, 1.0, np.zeros(D), Tw)
        inward = eA > 0 if side == 0 else eA < 0
        rho_w = (np.abs(eA[~inward & (eA != 0)]) * w[~inward & (eA != 0)]).sum() / \
                (np.abs(eA[inward]) * f0[inward]).sum()
        for i in np.nonzero(inward)[0]:
            for r in range(abs(eA[i])):  # rows whose pull of direction i crosses the wall
                row = r if side == 0 else nA - 1 - r
                got = f[i, row] if D == 3 else f[i, 0, row]
                assert np.allclose(got, rho_w * f0[i], rtol=0, atol=1e-12), (side, i, r)
    # and the fluid's mass is unchanged (each column's balance)
    assert abs(f.sum() - w.sum() * N) <= 1e-11 * N


@pytest.mark.parametrize("lat,shape", [(0, (14, 12, 1)), (1, (9, 8, 10))])
def test_solid_sites_refill_with_the_wall_maxwellian(lat, shape):
    """R15: a fluid site x next to solid sites at T_s receives, in each slot i
    pulled from a solid site, rho_w(x) f0_i(1, 0, T_s), where rho_w(x) makes
    the mass x sends into solid sites equal the mass it receives from them:
    for a fluid at rest at T = 1 (f = w),
    rho_w(x) = sum_{i: x + e_i solid} w_i / sum_{i: x - e_i solid} f0_i(1, 0, T_s)."""
    D, Q, c, e, w, neq = oracle.lattice_info(lat)
    nx, ny, nz = shape
    N = nx * ny * nz
    sim = oracle.OracleSim(lat, nx, ny, nz, TAU_OFF, np.zeros((D, N)))
    zz, yy, xx = np.indices((nz, ny, nx)).reshape(3, N)
    solid = (np.abs(xx - nx // 2) <= 1) & (np.abs(yy - ny // 2) <= 1)
    if D == 3:
        solid &= np.abs(zz - nz // 2) <= 1
    Ts = 1.08
    sim.set_solid(solid, np.where(solid, Ts, 1.0))
    sim.set_state(np.repeat(w[:, None], N, axis=1))
    sim.step(1)
    f = sim.get_state()
    f0 = oracle.equilibrium(lat, 1.0, np.zeros(D), Ts)
    n = np.array([nx, ny, nz])

    def is_solid(p):
        p = np.mod(p, n)
        return solid[(p[2] * ny + p[1]) * nx + p[0]]

    checked = 0
    for k in np.nonzero(~solid)[0]:
        p = np.array([xx[k], yy[k], zz[k]])
        into = [i for i in range(Q) if is_solid(p + e[i])]
        frm = [i for i in range(Q) if is_solid(p - e[i])]
        if not frm:
            continue
        rho_w = w[into].sum() / f0[frm].sum()
        assert np.allclose(f[frm, k], rho_w * f0[frm], rtol=0, atol=1e-12), k
        checked += 1
    assert checked > 0
    # fluid mass is conserved
    assert abs(f[:, ~solid].sum() - w.sum() * (~solid).sum()) <= 1e-11 * N
