"""Heat transfer between concentric cylinders under centrifugal force (Sec.
3.2, Fig. 2) on the GPU: solid-site walls against the oracle, and the steady
radial profiles against the analytic solution.

In the frame rotating with both cylinders the fluid is static; the walls are
staircases of solid sites (the library's diffuse-wall rule for solid sites).
Six FP64 runs -- theta_i / theta_o = 1.0 / 1.1 and 1.4 / 0.7, force order N
= 0, 1, 2 -- step concurrently, one stream each, to the steady state.
"""
import numpy as np
import pytest

import paper_2302_04741_gb300 as lbm
from oracle import cylinders_ref as cr
from paper_2302_04741_gb300 import workloads as W
from helpers import compare_fields, oracle_sim, perm_to_oracle

pytestmark = pytest.mark.gpu

THETAS = [(1.0, 1.1), (1.4, 0.7)]
ORDERS = [0, 1, 2]
CHUNK = 4000
MAX_STEPS = 400_000


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2302_04741_gb300 import build
    build.build()


def small_annulus(precision, force_order=2, include_sigma=False):
    """A 44 x 44 annulus (radii 5 and 19 sites) with the paper's kind of
    setup: field force alpha^2 R, walls at 1.2 (inner) and 0.9 (outer),
    constant mu, and a seeded perturbation so that it flows."""
    w = W.cylinders(1.2, 0.9, force_order=force_order, L=38, margin=3, precision=precision,
                    ratio=38 / 10.0, Uc=0.3, Re=20.0)
    N = w["shape"][0] * w["shape"][1]
    w["u"] = 0.02 * (W.uniform(5, 1, 2 * N).reshape(2, N) - 0.5)
    w["rho"] = w["rho"] * (1 + 0.01 * (W.uniform(5, 2, N) - 0.5))
    w["include_sigma"] = include_sigma
    return w


@pytest.mark.parametrize("precision,fo,sig", [(0, 2, False), (0, 1, False), (0, 2, True),
                                              (1, 2, False)])
def test_solid_sites_parity_with_oracle(precision, fo, sig):
    w = small_annulus(precision, fo, sig)
    sim = lbm.Sim(w).init()
    ref = oracle_sim(w)
    sim.step(15)
    ref.step(15)
    fluid = w["solid"] == 0
    perm = perm_to_oracle(w["lattice"])
    if precision == 0:
        fg = sim.populations()[:, fluid]
        fo_ = ref.pulled()[perm][:, fluid]
        assert np.max(np.abs(fg - fo_)) < 1e-14
    g = [np.asarray(a)[..., fluid] for a in sim.moments()]
    r = [np.asarray(a)[..., fluid] for a in ref.moments()]
    err = compare_fields(g, r, 1e-3 * 0.01 * np.sqrt(2 * fluid.sum()))
    tol = 1e-12 if precision == 0 else 1e-6
    assert all(err[k] <= tol for k in ("rho", "u", "T")), err
    solid_out = sim.moments()
    assert np.all(solid_out[0][~fluid] == 0.0)


def test_solid_sites_conserve_mass():
    w = small_annulus(1)
    sim = lbm.Sim(w).init()
    m0 = sim.conserved()[1]
    sim.step(500)
    m1 = sim.conserved()[1]
    fluid = int((w["solid"] == 0).sum())
    assert abs(m0 - fluid) < 1e-3 * fluid  # rho ~ 1 on the fluid sites only
    assert abs(m1 - m0) < 1e-6 * m0


def test_solid_sites_rejections():
    w = small_annulus(2)  # FP16 storage
    sim = lbm.Sim(w)
    with pytest.raises(lbm.LbmError) as ei:
        sim.init()
    assert ei.value.status == lbm.LBM_EINVAL
    w = small_annulus(0)
    sim = lbm.Sim(w).init()
    with pytest.raises(lbm.LbmError) as ei:  # after init
        lbm.lbm_set_solid(sim.ctx, w["solid"], w["T_wall"])
    assert ei.value.status == lbm.LBM_ESTATE


def radial_profiles(sim, w):
    rho, u, T, _ = sim.moments()
    fluid = w["solid"] == 0
    return np.stack([rho[fluid], T[fluid]]), float(np.max(np.abs(u[:, fluid])))


@pytest.fixture(scope="module")
def steady():
    torch = pytest.importorskip("torch")
    runs = []
    for ti, to in THETAS:
        for fo in ORDERS:
            w = W.cylinders(ti, to, force_order=fo)
            st = torch.cuda.Stream()
            sim = lbm.Sim(w, stream=st.cuda_stream, graph_steps=100).init()
            runs.append(dict(w=w, sim=sim, stream=st, prev=None, steps=0, done=False))
    while not all(r["done"] for r in runs):
        live = [r for r in runs if not r["done"]]
        for r in live:
            r["sim"].step(CHUNK)
        for r in live:
            r["steps"] += CHUNK
            prof, umax = radial_profiles(r["sim"], r["w"])
            if r["prev"] is not None:
                r["change"] = float(np.max(np.abs(prof - r["prev"])))
                if r["change"] < 1e-10 or r["steps"] >= MAX_STEPS:
                    r["done"], r["prof"], r["umax"] = True, prof, umax
            r["prev"] = prof
    table = {}
    for r in runs:
        w, prm = r["w"], r["w"]["params"]
        fluid = w["solid"] == 0
        R = w["radius"][fluid]
        rho_ref, th_ref = cr.profiles(R, prm["Ri"], prm["Ro"], prm["theta_i"], prm["theta_o"],
                                      prm["alpha"], prm["rho0"], mean_over=R)
        drho = np.abs(r["prof"][0] - rho_ref)
        dth = np.abs(r["prof"][1] - th_ref)
        key = (prm["theta_i"], prm["theta_o"], w["force_order"])
        # away from the staircase walls (3 sites)
        band = (R > prm["Ri"] + 3 * prm["c"]) & (R < prm["Ro"] - 3 * prm["c"])
        table[key] = dict(rho=float(drho.max()), theta=float(dth.max()),
                          theta_band=float(dth[band].max()), rho_band=float(drho[band].max()),
                          theta_rms=float(np.sqrt(np.mean(dth[band] ** 2))), umax=r["umax"],
                          steps=r["steps"], change=r["change"], T=r["prof"][1])
        r["sim"].close()
    print("\ntheta_i theta_o N | max|d rho| max|d theta| (band) rms(d theta, band) | max|u| | steps")
    for k, v in table.items():
        print(f"{k[0]:.1f} {k[1]:.1f} {k[2]} | {v['rho']:.3e} {v['theta']:.3e} ({v['theta_band']:.3e}) "
              f"{v['theta_rms']:.3e} | {v['umax']:.1e} | {v['steps']} (last change {v['change']:.1e})")
    return table


def test_cylinders_reach_steady_state(steady):
    for k, v in steady.items():
        assert v["change"] < 1e-10, (k, v)


# measured N = 2 errors (rms of theta in the band, max in the band): 1.0e-3 /
# 3.3e-3 at 10 % temperature variation, 8.1e-3 / 2.6e-2 at 100 %; they are
# set by the staircase diffuse walls (temperature jump ~ mean free path x
# dtheta/dR, largest at the inner wall), not by the force term
BOUNDS = {(1.0, 1.1): (2e-3, 6e-3), (1.4, 0.7): (1.2e-2, 4e-2)}


@pytest.mark.parametrize("thetas", THETAS)
def test_cylinders_third_order_force_matches_analytic(steady, thetas):
    v = steady[(*thetas, 2)]
    rms, mx = BOUNDS[thetas]
    assert v["theta_rms"] < rms and v["theta_band"] < mx and v["rho_band"] < mx, v


@pytest.mark.parametrize("thetas", THETAS)
def test_cylinders_force_order_ranking(steady, thetas):
    """Without the third-moment term the temperature error is larger (N = 0
    and 1 coincide up to the small spurious flow: u = 0)."""
    e = {fo: steady[(*thetas, fo)]["theta_rms"] for fo in ORDERS}
    assert e[1] > 1.8 * e[2] and e[0] > 1.8 * e[2], e  # measured 3.5x and 2.2x
    d01 = np.max(np.abs(steady[(*thetas, 0)]["T"] - steady[(*thetas, 1)]["T"]))
    assert d01 < 0.1 * abs(e[1] - e[2]) + 1e-12, (d01, e)
