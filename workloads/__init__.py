"""Seeded synthetic inputs shared, as data, by the CUDA path and the oracle.

This module holds no arithmetic of the solver: only the parameter sets of the
workloads (grating shape, wavenumbers, discretisation sizes, incidence angles)
and the seeded random placement of the disks.  Both the library binding and the
oracle consume its output; neither depends on the other.

Conventions (Sec. 2 of the paper, "Problem formulation"):
  * one period d, unit cell x in [-d/2, d/2];
  * interface j is the graph y = h_j(x) = h0 + sum_m (a_m cos(2 pi m x/d) + b_m sin(2 pi m x/d));
  * wavenumbers k = (k1 top, k2 middle, k3 bottom), TM polarisation;
  * the incident angle theta follows the paper: u_inc = exp(i k1 (cos(theta) x + sin(theta) y)),
    with sin(theta) < 0 for a wave travelling downwards.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "grating", "disks", "config", "CONFIG_NAMES", "wood_angle",
    "batched_angles", "batched_geometries", "sweep_points",
]


def _iface(h0, cos=(), sin=()):
    return {"h0": float(h0), "cos": [float(c) for c in cos], "sin": [float(s) for s in sin]}


def grating(name: str) -> dict:
    """Layer/periodic parameters of a named grating.

    Keys: d, gamma1, gamma2 (interface Fourier descriptions), k (k1,k2,k3), N (nodes per
    interface), y0 (Gamma_u at +y0, Gamma_d at -y0), Q (J-expansion orders for layers 1,2,3),
    K_rb (Rayleigh-Bloch orders -K..K), n_wall (Gauss-Legendre nodes on the walls of layers
    1,2,3), n_bound (equispaced nodes on Gamma_u and on Gamma_d), eps_pinv (Sec. 5, pseudo-inverse
    regularisation 1e-10).
    """
    if name == "fig2":
        # Sec. 3, Fig. 2: empty grating k=(10,5,10), Gamma1 y=1+0.1 sin 2pi x, Gamma2 y=-1+0.1 cos 2pi x,
        # N=120, 50 points on Gamma_u/Gamma_d, 2Q+1=73, 41 Rayleigh-Bloch modes (Sec. 6).
        return dict(d=1.0, gamma1=_iface(1.0, sin=[0.1]), gamma2=_iface(-1.0, cos=[0.1]),
                    k=(10.0, 5.0, 10.0), N=120, y0=1.6, Q=(36, 36, 36), K_rb=20,
                    n_wall=(50, 70, 50), n_bound=50, eps_pinv=1e-10)
    if name in ("small", "c1"):
        # k=(10,15,20); interfaces y=+-0.5+0.05 cos 2pi x with 128 nodes each.
        return dict(d=1.0, gamma1=_iface(0.5, cos=[0.05]), gamma2=_iface(-0.5, cos=[0.05]),
                    k=(10.0, 15.0, 20.0), N=128, y0=1.0, Q=(36, 36, 36), K_rb=20,
                    n_wall=(40, 60, 40), n_bound=50, eps_pinv=1e-10)
    if name in ("headline", "c2"):
        # k=(40,60,80); interfaces y=+-0.5+0.05 cos 2pi x with 256 nodes each.
        return dict(d=1.0, gamma1=_iface(0.5, cos=[0.05]), gamma2=_iface(-0.5, cos=[0.05]),
                    k=(40.0, 60.0, 80.0), N=256, y0=1.0, Q=(90, 90, 90), K_rb=30,
                    n_wall=(80, 120, 80), n_bound=80, eps_pinv=1e-10)
    if name == "tiny":
        # A cheap grating for unit tests of the layer block (few nodes, low wavenumbers).
        return dict(d=1.0, gamma1=_iface(0.5, cos=[0.05]), gamma2=_iface(-0.5, cos=[0.05]),
                    k=(6.0, 8.0, 7.0), N=64, y0=1.0, Q=(20, 24, 20), K_rb=10,
                    n_wall=(24, 36, 24), n_bound=32, eps_pinv=1e-10)
    raise KeyError(name)


def scaled_grating(base: str, k_top: float) -> dict:
    """The grating `base` with all wavenumbers scaled so that k1 == k_top (a frequency sweep)."""
    g = dict(grating(base))
    s = k_top / g["k"][0]
    g["k"] = tuple(float(kk * s) for kk in g["k"])
    return g


def wood_angle(k1: float, d: float = 1.0, n: int = 1) -> float:
    """Incidence angle (paper convention, sin < 0) at which kappa_n = kappa + 2 pi n / d = k1, so that
    k_{1,n} = 0 (a Wood anomaly, Sec. 2)."""
    return -math.acos(1.0 - 2.0 * math.pi * n / (k1 * d))


def _min_image_ok(cand, pts, dmin, d):
    if len(pts) == 0:
        return True
    dx = np.abs(pts[:, 0] - cand[0])
    dx = np.minimum(dx, d - dx)
    dy = pts[:, 1] - cand[1]
    return bool(np.all(dx * dx + dy * dy >= dmin * dmin))


def disks(M: int, radius: float, gap: float, index: float, k_top: float, seed: int,
          d: float = 1.0, ymax: float = 0.4, iface_min: float = 0.45, clearance: float = 0.04,
          p: int = 12, max_tries: int = 2_000_000) -> dict:
    """Seeded non-overlapping disks, centres uniform in the middle layer.

    Centres are drawn uniformly in x in [-d/2, d/2) and |y| < min(ymax, iface_min - clearance - r),
    and accepted when the minimum-image distance (periodic in x) to every accepted centre is at
    least 2r + gap.  Disks may cross the unit-cell walls.  k_p = index * k_top.
    Returns {"xy": (M,2), "radius": (M,), "kp": (M,), "p": p}.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ylim = min(ymax, iface_min - clearance - radius)
    dmin = 2.0 * radius + gap
    # cell list over the strip for fast rejection
    ncx = max(1, int(d / dmin))
    cells: dict = {}
    pts = []
    tries = 0
    while len(pts) < M:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"disk placement failed after {max_tries} tries ({len(pts)} of {M})")
        x = rng.uniform(-0.5 * d, 0.5 * d)
        y = rng.uniform(-ylim, ylim)
        cx = int((x + 0.5 * d) / d * ncx) % ncx
        cy = int(math.floor(y / dmin))
        near = []
        for ox in (-1, 0, 1):
            for oy in (-1, 0, 1):
                near.extend(cells.get(((cx + ox) % ncx, cy + oy), ()))
        if near and not _min_image_ok((x, y), np.asarray(near), dmin, d):
            continue
        pts.append((x, y))
        cells.setdefault((cx, cy), []).append((x, y))
    xy = np.asarray(pts, dtype=np.float64)
    return {"xy": xy, "radius": np.full(M, float(radius)), "kp": np.full(M, float(index * k_top)),
            "p": int(p)}


def batched_angles(k1: float = 40.0, n: int = 256, d: float = 1.0) -> np.ndarray:
    """256 angles phi uniform in [-pi/3, pi/3] (measured from the downward normal), with the one
    nearest the k1 Wood anomaly replaced by it exactly; returned in the paper's convention
    theta = -pi/2 + phi."""
    phi = np.linspace(-math.pi / 3, math.pi / 3, n)
    phi_w = wood_angle(k1, d) + 0.5 * math.pi
    j = int(np.argmin(np.abs(phi - phi_w)))
    phi[j] = phi_w
    return -0.5 * math.pi + phi


def batched_geometries(n_geom: int = 64, seed: int = 4, k_top: float = 40.0, p: int = 12,
                       m_lo: int = 250, m_hi: int = 4000, d: float = 1.0) -> list:
    """Geometries of uneven size: M log-uniform in [m_lo, m_hi], radius uniform in
    [0.004, min(0.01, r_max(M))] with r_max(M) = sqrt(0.4*0.8/(pi M))/1.25 (keeps the packing
    feasible), index uniform in [1.5, 2.5]; gap r/2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for g in range(n_geom):
        M = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        rmax = min(0.01, math.sqrt(0.4 * 0.8 / (math.pi * M)) / 1.25)
        r = rng.uniform(0.004, max(0.004, rmax))
        idx = rng.uniform(1.5, 2.5)
        out.append(disks(M, r, 0.5 * r, idx, k_top, seed=1000 * seed + g, d=d, p=p))
    return out


def sweep_points(n: int = 4096, seed: int = 5, phi_range=(-math.pi / 3, math.pi / 3),
                 k_range=(35.0, 45.0)) -> np.ndarray:
    """(phi, k_top) pairs, iid uniform in phi_range x k_range (default [-pi/3, pi/3] x [35, 45])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    phi = rng.uniform(phi_range[0], phi_range[1], n)
    kt = rng.uniform(k_range[0], k_range[1], n)
    return np.stack([phi, kt], axis=1)


CONFIG_NAMES = ("small", "headline", "mixed4000", "batched", "warmstart")


def config(name: str, seed: int = 1) -> dict:
    """A full workload: grating, incidence angle(s), disks, solver tolerance.

    small      M=10 disks r=0.04 index 2, k=(10,15,20), p=10, theta=-pi/5, GMRES tol 1e-12.
    headline   M=1000 disks r=0.008 gap 0.004 index 2, k=(40,60,80), p=12, theta=-pi/5, tol 1e-11.
    mixed4000  M=4000 disks r=0.004 gap 0.002 on the headline grating, Bragg target 1e-9.
    """
    if name == "small":
        g = grating("small")
        return {"name": name, "grating": g, "theta": -math.pi / 5,
                "disks": disks(10, 0.04, 0.02, 2.0, g["k"][0], seed=seed, p=10), "tol": 1e-12}
    if name == "headline":
        g = grating("headline")
        return {"name": name, "grating": g, "theta": -math.pi / 5,
                "disks": disks(1000, 0.008, 0.004, 2.0, g["k"][0], seed=seed, p=12), "tol": 1e-11}
    if name == "mixed4000":
        g = grating("headline")
        return {"name": name, "grating": g, "theta": -math.pi / 5,
                "disks": disks(4000, 0.004, 0.002, 2.0, g["k"][0], seed=seed, p=12), "tol": 1e-11,
                "bragg_target": 1e-9}
    raise KeyError(name)


def mlp_init(p: int, seed: int = 11) -> np.ndarray:
    """Seeded initial weights of the warm-start network for multipole order p, flat float32 in the
    order W1[64][128], b1[128], W2[128][128], b2[128], W3[128][2(2p+1)], b3[2(2p+1)]: weights
    N(0, 1/fan_in), biases zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    no = 2 * (2 * p + 1)
    parts = []
    for fan_in, fan_out in ((64, 128), (128, 128), (128, no)):
        parts.append(rng.normal(0.0, 1.0 / math.sqrt(fan_in), (fan_in, fan_out)).ravel())
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)
