"""Seeded synthetic workloads shaped like the paper's runs.

This module only builds INPUTS: grid shapes, relaxation times, body-force
descriptors and initial fields (rho, u, T).  It contains none of the lattice
Boltzmann arithmetic, so the CUDA path and the CPU oracle can both consume its
arrays without sharing any of the method.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: value k of stream (seed, tag) is mix(seed * 2^32 + tag + (k + 1) *
0x9E3779B97F4A7C15), so every array is reproducible element by element.

Field layout everywhere: scalars (N,), vectors (D, N), with N = nx*ny*nz and x
fastest ("row-major [nz][ny][nx]").
"""
import math

import numpy as np

D2Q37, D3Q39 = 0, 1
PERIODIC, BOUNCE_BACK, THERMAL_WALL = 0, 1, 2
G_UNIFORM, G_SINE, G_FIELD = 0, 1, 2
FP64, FP32_SHIFTED, FP16_SCALED = 0, 1, 2

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, tag, n):
    """n uint64 values of the counter-based SplitMix64 stream (seed, tag)."""
    with np.errstate(over="ignore"):
        base = np.uint64((int(seed) << 32) + int(tag) & 0xFFFFFFFFFFFFFFFF)
        z = base + (np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, tag, n, lo=0.0, hi=1.0):
    """n doubles uniform in [lo, hi) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, tag, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def dims(lattice):
    return 2 if lattice == D2Q37 else 3


def g_field_array(lattice, shape, g):
    """Materialise a body-force descriptor as a (D, N) array.

    g = {"kind": G_UNIFORM, "g0": (gx, gy, gz)}
      | {"kind": G_SINE, "g0": ..., "wave_axis": a}  -> g0 * sin(2 pi x_a / n_a)
      | {"kind": G_FIELD, "field": (D, N) array}
    """
    D = dims(lattice)
    nx, ny, nz = shape
    N = nx * ny * nz
    if g["kind"] == G_FIELD:
        return np.ascontiguousarray(np.asarray(g["field"], dtype=np.float64).reshape(D, N))
    g0 = np.zeros(3)
    g0[:len(g["g0"])] = g["g0"]
    out = np.empty((D, N))
    if g["kind"] == G_UNIFORM:
        for a in range(D):
            out[a] = g0[a]
        return out
    axis = g["wave_axis"]
    n_axis = shape[axis]
    coord = np.indices((nz, ny, nx)).reshape(3, N)[2 - axis]
    s = np.sin(2.0 * math.pi * coord / n_axis)
    for a in range(D):
        out[a] = g0[a] * s
    return out


def _coords(shape):
    nx, ny, nz = shape
    zz, yy, xx = np.indices((nz, ny, nx)).reshape(3, nx * ny * nz)
    return xx, yy, zz


def kolmogorov(nx=64, ny=64, tau=0.8, g0=1e-5, seed=1, rho_noise=1e-6, T_amp=0.01,
               lattice=D2Q37, nz=1, precision=FP64, force_order=2):
    """Periodic Kolmogorov flow: g_x = g0 sin(2 pi y / ny), T = 1 + T_amp sin(2 pi x / nx),
    rho = 1 + U(-rho_noise, rho_noise), u = 0 (the 64x64 D2Q37 FP64 configuration)."""
    D = dims(lattice)
    if D == 2:
        nz = 1
    shape = (nx, ny, nz)
    N = nx * ny * nz
    xx, _, _ = _coords(shape)
    rho = 1.0 + uniform(seed, 1, N, -rho_noise, rho_noise)
    T = 1.0 + T_amp * np.sin(2.0 * math.pi * xx / nx)
    u = np.zeros((D, N))
    return dict(lattice=lattice, shape=shape, tau=tau, precision=precision,
                force_order=force_order, bc=(PERIODIC,) * 3, T_lo=(1.0,) * 3, T_hi=(1.0,) * 3,
                g={"kind": G_SINE, "g0": (g0, 0.0, 0.0), "wave_axis": 1},
                rho=rho, u=u, T=T, name=f"kolmogorov_{nx}x{ny}" + (f"x{nz}" if D == 3 else ""))


def rayleigh_benard(nx=1024, ny=512, nz=1, lattice=D2Q37, tau=0.6, g=-1e-5, T_bottom=1.05,
                    T_top=0.95, seed=2, T_noise=1e-4, precision=FP32_SHIFTED, force_order=2):
    """Thermal Rayleigh-Benard cell: walls normal to the last axis (y in 2-D, z in 3-D) at
    T_bottom / T_top, periodic elsewhere, uniform gravity g along that axis, rho = 1, u = 0,
    T linear between the wall values plus U(-T_noise, T_noise)."""
    D = dims(lattice)
    if D == 2:
        nz = 1
    shape = (nx, ny, nz)
    N = nx * ny * nz
    wall = D - 1
    xx, yy, zz = _coords(shape)
    h = (yy if wall == 1 else zz).astype(np.float64)
    n_wall = shape[wall]
    T = T_bottom + (T_top - T_bottom) * (h + 0.5) / n_wall
    T = T + uniform(seed, 2, N, -T_noise, T_noise)
    rho = np.ones(N)
    u = np.zeros((D, N))
    bc = [PERIODIC] * 3
    bc[wall] = THERMAL_WALL
    T_lo = [1.0] * 3
    T_hi = [1.0] * 3
    T_lo[wall] = T_bottom
    T_hi[wall] = T_top
    g0 = [0.0] * 3
    g0[wall] = g
    return dict(lattice=lattice, shape=shape, tau=tau, precision=precision,
                force_order=force_order, bc=tuple(bc), T_lo=tuple(T_lo), T_hi=tuple(T_hi),
                g={"kind": G_UNIFORM, "g0": tuple(g0)}, rho=rho, u=u, T=T,
                name=f"rayleigh_benard_{nx}x{ny}" + (f"x{nz}" if D == 3 else ""))


# Lattice constant of the D2Q37 rule as the paper prints it (Sec. 3): the
# lattice spacing in units of the reference thermal speed.
C_D2Q37 = 1.196979770393


def poiseuille_parameters(theta_b, theta_t, Uc=1.5, Re=1800.0, Ly=150, Pr=1.0,
                          gy_over_gx=-50.0, rho0=1.0, c=C_D2Q37, D=2):
    """Parameters of the compressible Poiseuille validation case (Sec. 3.1):
    channel height H = L_y c, dynamic viscosity mu = rho0 U_c H / Re,
    conductivity lambda = c_p mu / Pr with c_p = (D + 2) / 2, and g_x from the
    definition U_c = rho0 g_x H^2 / (8 mu), i.e. g_x = 8 U_c^2 / (Re H) (the
    printed U_c^2 / (Re H) lacks the factor 8 this definition implies);
    g_y = (g_y / g_x) g_x points down."""
    H = Ly * c
    mu = rho0 * Uc * H / Re
    lam = (D + 2) / 2.0 * mu / Pr
    gx = 8.0 * Uc * Uc / (Re * H)
    return dict(H=H, mu=mu, lam=lam, gx=gx, gy=gy_over_gx * gx, rho0=rho0, theta_b=theta_b,
                theta_t=theta_t, Uc=Uc, Re=Re, Ly=Ly)


def poiseuille(theta_b=1.0, theta_t=1.1, force_order=2, include_sigma=False, Lx=3, Ly=150,
               precision=FP64, **kw):
    """Compressible Poiseuille flow under cross gravity on an L_x x L_y D2Q37
    lattice (Sec. 3.1): thermal walls at y = -1/2 and L_y - 1/2 (theta_b below,
    theta_t above, no slip), periodic in x, uniform g = (g_x, g_y), constant mu
    (tau = mu / (rho theta) per site).  Starts from rest at rho = rho0 with theta
    linear between the wall values."""
    prm = poiseuille_parameters(theta_b, theta_t, Ly=Ly, **kw)
    shape = (Lx, Ly, 1)
    N = Lx * Ly
    _, yy, _ = _coords(shape)
    T = theta_b + (theta_t - theta_b) * (yy + 0.5) / Ly
    return dict(lattice=D2Q37, shape=shape, tau=1.0, mu=prm["mu"], precision=precision,
                force_order=force_order, include_sigma=include_sigma,
                bc=(PERIODIC, THERMAL_WALL, PERIODIC), T_lo=(1.0, theta_b, 1.0),
                T_hi=(1.0, theta_t, 1.0), g={"kind": G_UNIFORM, "g0": (prm["gx"], prm["gy"], 0.0)},
                rho=np.full(N, prm["rho0"]), u=np.zeros((2, N)), T=T, params=prm,
                name=f"poiseuille_{Lx}x{Ly}_theta{theta_b}-{theta_t}_N{force_order}"
                     + ("_sigma" if include_sigma else ""))


def cylinders_parameters(theta_i, theta_o, L=250, ratio=5.0, Uc=0.3, Re=100.0, rho0=1.0,
                         c=C_D2Q37):
    """Parameters of the concentric-cylinder test (Sec. 3.2): outer radius
    R_o = L c / 2, inner R_i = R_o / ratio, centre-line speed U_c = alpha (R_o
    + R_i) / 2 (which fixes the angular speed alpha), Re = rho0 alpha (R_o^2 -
    R_i^2) / (2 mu) (which fixes mu)."""
    Ro = L * c / 2.0
    Ri = Ro / ratio
    alpha = Uc / (0.5 * (Ro + Ri))
    mu = rho0 * alpha * (Ro * Ro - Ri * Ri) / (2.0 * Re)
    return dict(Ro=Ro, Ri=Ri, alpha=alpha, mu=mu, rho0=rho0, theta_i=theta_i, theta_o=theta_o,
                Uc=Uc, Re=Re, L=L, c=c)


def cylinders(theta_i=1.0, theta_o=1.1, force_order=2, L=250, margin=3, precision=FP64, **kw):
    """Heat transfer between concentric cylinders rotating together (Sec. 3.2),
    in the co-rotating frame: static fluid under the centrifugal acceleration
    g = alpha^2 R (radially outward) on an (L + 2 margin)^2 periodic D2Q37 grid.
    Sites farther than R_o from the centre, or nearer than R_i, are solid walls
    at theta_o and theta_i (a staircase); the margin keeps >= 3 solid rows
    between the outer wall and the periodic edges.  Constant mu; starts from
    rho = rho0, u = 0 and the conduction profile theta(R) ~ ln R."""
    prm = cylinders_parameters(theta_i, theta_o, L=L, **kw)
    n = L + 2 * margin
    shape = (n, n, 1)
    N = n * n
    xx, yy, _ = _coords(shape)
    cx = cy = 0.5 * (n - 1)
    X, Y = prm["c"] * (xx - cx), prm["c"] * (yy - cy)
    R = np.hypot(X, Y)
    inner, outer = R < prm["Ri"], R > prm["Ro"]
    solid = inner | outer
    T_wall = np.where(inner, theta_i, theta_o)
    Rc = np.clip(R, prm["Ri"], prm["Ro"])
    T = theta_i + (theta_o - theta_i) * np.log(Rc / prm["Ri"]) / math.log(prm["Ro"] / prm["Ri"])
    a2 = prm["alpha"] ** 2
    field = np.stack([a2 * X, a2 * Y])
    return dict(lattice=D2Q37, shape=shape, tau=1.0, mu=prm["mu"], precision=precision,
                force_order=force_order, bc=(PERIODIC,) * 3, T_lo=(1.0,) * 3, T_hi=(1.0,) * 3,
                g={"kind": G_FIELD, "field": field}, rho=np.full(N, prm["rho0"]),
                u=np.zeros((2, N)), T=T, solid=solid.astype(np.uint8), T_wall=T_wall, radius=R,
                params=prm, name=f"cylinders_{n}x{n}_theta{theta_i}-{theta_o}_N{force_order}")


RAGGED_SIDES = (128, 192, 256, 384, 512)


def ragged_batch(count=64, seed=3, sides=RAGGED_SIDES, tau_range=(0.55, 1.0),
                 g_range=(1e-6, 1e-4), precision=FP32_SHIFTED):
    """Independent periodic D2Q37 Kolmogorov grids: nx, ny drawn from ``sides``,
    tau ~ U[tau_range], g0 ~ U[g_range] (the ragged-batch configuration)."""
    r = uniform(seed, 3, 4 * count)
    grids = []
    for k in range(count):
        nx = sides[int(r[4 * k] * len(sides))]
        ny = sides[int(r[4 * k + 1] * len(sides))]
        tau = tau_range[0] + (tau_range[1] - tau_range[0]) * r[4 * k + 2]
        g0 = g_range[0] + (g_range[1] - g_range[0]) * r[4 * k + 3]
        w = kolmogorov(nx=nx, ny=ny, tau=tau, g0=g0, seed=seed * 1000 + k, precision=precision)
        w["name"] = f"ragged[{k}]_{nx}x{ny}"
        grids.append(w)
    return grids


SERVING_SIDES = (32, 48, 64, 96)


def serving_trace(n_requests=2000, rate=200.0, seed=4, sides=SERVING_SIDES, g_range=(1e-6, 1e-5),
                  steps_range=(500, 5000), tau=0.8):
    """Poisson arrivals of D3Q39 periodic thermal boxes: side from ``sides``, gravity
    magnitude ~ U[g_range] along -z, steps ~ U{steps_range}.  Returns a list of dicts with
    the arrival time and the request's workload (fields built lazily by make_request)."""
    r = uniform(seed, 5, 4 * n_requests)
    t = 0.0
    reqs = []
    for k in range(n_requests):
        t += -math.log(1.0 - r[4 * k]) / rate
        side = sides[int(r[4 * k + 1] * len(sides))]
        gmag = g_range[0] + (g_range[1] - g_range[0]) * r[4 * k + 2]
        steps = steps_range[0] + int(r[4 * k + 3] * (steps_range[1] - steps_range[0] + 1))
        reqs.append(dict(id=k, arrival=t, side=side, g=gmag, steps=steps, tau=tau, seed=seed))
    return reqs


def make_request(req, precision=FP32_SHIFTED):
    """Workload of one serving request: a periodic thermal box with a small T wave."""
    s = req["side"]
    N = s ** 3
    shape = (s, s, s)
    xx, _, zz = _coords(shape)
    T = 1.0 + 0.01 * np.sin(2.0 * math.pi * xx / s) * np.cos(2.0 * math.pi * zz / s)
    rho = 1.0 + uniform(req["seed"] * 100000 + req["id"], 6, N, -1e-6, 1e-6)
    u = np.zeros((3, N))
    return dict(lattice=D3Q39, shape=shape, tau=req["tau"], precision=precision, force_order=2,
                bc=(PERIODIC,) * 3, T_lo=(1.0,) * 3, T_hi=(1.0,) * 3,
                g={"kind": G_UNIFORM, "g0": (0.0, 0.0, -req["g"])}, rho=rho, u=u, T=T,
                name=f"serve[{req['id']}]_{s}^3")
