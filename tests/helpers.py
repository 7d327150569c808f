"""Test helpers: run the same seeded workload on the CUDA library and on the
CPU oracle and compare them.  Nothing here computes any part of the method."""
import numpy as np

import oracle
import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import workloads as W


def rel_l2(a, b, floor=0.0):
    """||a - b||_2 / max(||b||_2, floor) over every site and component."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), floor))


def perm_to_oracle(lat):
    """perm[k] = oracle index of the library's direction k (matched by vector)."""
    e = lbm.lbm_lattice_info(lat)[3]
    eo = oracle.lattice_info(lat)[3]
    idx = {tuple(v): k for k, v in enumerate(eo)}
    return np.array([idx[tuple(v)] for v in e])


def oracle_sim(w):
    g = W.g_field_array(w["lattice"], w["shape"], w["g"])
    s = oracle.OracleSim(w["lattice"], *w["shape"], w["tau"], g, force_order=w.get("force_order", 2),
                         bc=w.get("bc", (0, 0, 0)), T_lo=w.get("T_lo", (1, 1, 1)),
                         T_hi=w.get("T_hi", (1, 1, 1)), mu=w.get("mu", 0.0),
                         include_sigma=w.get("include_sigma", False))
    if w.get("solid") is not None:
        s.set_solid(w["solid"], w["T_wall"])
    s.init(w["rho"], w["u"], w["T"])
    return s


def _modes(shape, seed, tag, n_modes=3):
    """Sum of a few seeded Fourier modes of the periodic box, scaled to [-1, 1]."""
    nx, ny, nz = shape
    zz, yy, xx = np.indices((nz, ny, nx)).reshape(3, nx * ny * nz)
    r = W.uniform(seed, tag, 4 * n_modes)
    f = np.zeros(nx * ny * nz)
    for m in range(n_modes):
        kx, ky = 1 + int(r[4 * m] * 2), int(r[4 * m + 1] * 3)
        kz = int(r[4 * m + 2] * 2) if nz > 1 else 0
        ph = 2 * np.pi * r[4 * m + 3]
        f += np.sin(2 * np.pi * (kx * xx / nx + ky * yy / ny + kz * zz / nz) + ph)
    return f / n_modes


def smooth_state(lat, shape, seed, amp_u=0.02, amp_T=0.03, amp_rho=0.01, noise=1e-4):
    """Seeded resolved initial fields (rho, u, T): a few Fourier modes plus a
    small white-noise component that still exercises every code path."""
    D = W.dims(lat)
    N = shape[0] * shape[1] * shape[2]
    wn = lambda tag, n: 2 * noise * (W.uniform(seed, tag, n) - 0.5)
    rho = 1.0 + amp_rho * _modes(shape, seed, 31) + amp_rho * wn(21, N)
    u = np.stack([amp_u * _modes(shape, seed, 32 + a) for a in range(D)]) + amp_u * wn(22, D * N).reshape(D, N)
    T = 1.0 + amp_T * _modes(shape, seed, 36) + amp_T * wn(23, N)
    return rho, u, T


def white_noise_state(lat, shape, seed, amp_u=0.02, amp_T=0.03, amp_rho=0.01):
    """Grid-scale white-noise fields (unresolved; used only where stated)."""
    D = W.dims(lat)
    N = shape[0] * shape[1] * shape[2]
    rho = 1.0 + amp_rho * (W.uniform(seed, 21, N) - 0.5)
    u = 2 * amp_u * (W.uniform(seed, 22, D * N).reshape(D, N) - 0.5)
    T = 1.0 + 2 * amp_T * (W.uniform(seed, 23, N) - 0.5)
    return rho, u, T


def workload(lat, shape, tau=0.8, g=None, seed=1, precision=0, force_order=2, bc=(0, 0, 0),
             T_lo=(1.0, 1.0, 1.0), T_hi=(1.0, 1.0, 1.0), white_noise=False, **amps):
    D = W.dims(lat)
    if g is None:
        g = {"kind": W.G_UNIFORM, "g0": (2e-5, -1e-5, 5e-6)[:D] + (0.0,) * (3 - D)}
    make = white_noise_state if white_noise else smooth_state
    rho, u, T = make(lat, shape, seed, **amps)
    return dict(lattice=lat, shape=shape, tau=tau, g=g, precision=precision,
                force_order=force_order, bc=bc, T_lo=T_lo, T_hi=T_hi, rho=rho, u=u, T=T,
                name=f"test_{lat}_{shape}")


def compare_fields(gpu, ref, q_floor):
    """Relative L2 errors of (rho, u, T, q) as a dict."""
    names = ("rho", "u", "T", "q")
    out = {}
    for n, a, b in zip(names, gpu, ref):
        out[n] = rel_l2(a, b, q_floor if n == "q" else 0.0)
    return out
