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


def q_floor(w, u_ref):
    D = W.dims(w["lattice"])
    N = w["shape"][0] * w["shape"][1] * w["shape"][2]
    Ma = max(float(np.max(np.abs(u_ref))), 1e-3)
    return 1e-3 * Ma * np.sqrt(D * N)


def q_roundoff(ref, lat):
    """L2 norm over sites of 8 eps_64 sum_i |f~_i| |xi_i - u|^3 (per component)."""
    D, Q, c, e, _, _ = oracle.lattice_info(lat)
    ft = ref.pulled()
    u = ref.moments()[1]
    xi = c * e[:, :D].astype(float)
    cc = xi[:, :, None] - u[None, :, :]
    mag3 = np.sqrt((cc * cc).sum(axis=1)) ** 3
    B = 8 * 2.0 ** -53 * (np.abs(ft) * mag3).sum(axis=0)
    return float(np.linalg.norm(B) * np.sqrt(D))


# Unit roundoff of each float codec's stored value (the deviation f - w).
STORAGE_UNIT_ROUNDOFF = {1: 2.0 ** -24, 2: 2.0 ** -11}


def q_codec_bound(ref, w):
    """L2 norm over sites of the q error a float codec's rounding of the
    stored deviations d_i = f~_i - w_i can cause.  q = 1/2 (1 - 1/(2 tau))
    sum_i (...)_i |c_i|^2 c_i (c_i = xi_i - u) is a strongly cancelling third
    moment; a relative perturbation of at most u_s of every d_i changes it by
    at most k_i = 1/2 (1 - 1/(2 tau)) u_s |d_i| |c_i|^3 per direction.
      FP16 (u_s = 2^-11): storage-dominated (its float arithmetic is 2^13
      times finer, and the codec's error equals its storage floor), the
      rounding errors are independent and uniform, so twice the rms,
      2 sqrt(sum_i k_i^2 / 3), bounds the L2 over many sites.
      FP32 (u_s = 2^-24): dominated by the float arithmetic of the collision,
      whose rounding of intermediates shared by many directions is coherent
      (measured 3-30x the rms of one storage rounding), so the first-order
      worst case sum_i k_i (all roundings aligned).
    Zero for FP64 (q_roundoff covers its own rounding)."""
    prec = w.get("precision", 0)
    us = STORAGE_UNIT_ROUNDOFF.get(prec, 0.0)
    if us == 0.0:
        return 0.0
    D, Q, c, e, wt, _ = oracle.lattice_info(w["lattice"])
    ft = ref.pulled()
    rho, u, T, _ = ref.moments()
    mu = w.get("mu", 0.0)
    tau = mu / (rho * T) + 0.5 if mu > 0 else np.full(rho.shape, float(w["tau"]))
    xi = c * e[:, :D].astype(float)
    cc = xi[:, :, None] - u[None, :, :]
    mag3 = np.sqrt((cc * cc).sum(axis=1)) ** 3
    k = 0.5 * (1.0 - 0.5 / tau) * us * np.abs(ft - wt[:, None]) * mag3
    per_site = 2.0 * np.sqrt((k * k).sum(axis=0) / 3.0) if prec == 2 else k.sum(axis=0)
    return float(np.linalg.norm(per_site) * (np.sqrt(D) if prec != 2 else 1.0))


def check_fields(sim, ref, w, tol):
    """Relative L2 of rho, u, T and q of ``sim`` (a Sim, or its moments as a
    tuple) against the oracle ``ref`` within ``tol``.  q is normalised by
    max(||q_ref||, q_floor); its bound adds the round-off of its defining FP64
    sum (q_roundoff) and, for the float codecs, the error the codec's
    rounding of the stored deviations can cause in that sum (q_codec_bound):
    q is the small remainder of a cancelling third moment, which a codec
    resolves only to that level."""
    g = sim.moments() if hasattr(sim, "moments") else sim
    r = ref.moments()
    qf = q_floor(w, r[1])
    err = compare_fields(g, r, qf)
    dq = float(np.linalg.norm((g[3] - r[3]).ravel()))
    q_ok = dq <= (tol * max(float(np.linalg.norm(r[3].ravel())), qf) + q_roundoff(ref, w["lattice"])
                  + q_codec_bound(ref, w))
    ok = all(err[k] <= tol for k in ("rho", "u", "T")) and q_ok
    assert ok, err
    return err
