"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module computes INITIAL DATA only. It holds none of the finite-volume
step's arithmetic (no reconstruction, flux, EMF, source, update, inversion or
floor). To express analytic solutions in the native coordinates it carries its
own few Kerr-Schild metric components and its own coordinate map, written
separately from both the CUDA library and the oracle.

Problems (the paper's test and performance workloads; every input is
synthetic):
  * linear MHD slow mode in a periodic Minkowski box (regression tests,
    "Readiness and Testing" section);
  * Bondi accretion on Schwarzschild in MKS coordinates (same section;
    Michel's transonic polytrope solution);
  * Fishbone-Moncrief torus with a single-loop poloidal field on Kerr in funky
    MKS (the torus workload of the "Performance" section).

Arrays are numpy float64 of shape (8, N3, N2, N1), ghosts included, slot
order (rho, u, u~1, u~2, u~3, B1, B2, B3).
"""
from __future__ import annotations

import math

import numpy as np

NG = 3

# ---------------------------------------------------------------------------
# Counter-based noise: splitmix64 (Steele, Lea & Flood 2014) of
# seed XOR global interior zone index, top 53 bits scaled to [0, 1).
# ---------------------------------------------------------------------------
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
    with np.errstate(over="ignore"):
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, index: np.ndarray) -> np.ndarray:
    z = splitmix64(np.uint64(seed) ^ np.asarray(index, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def interior_index(cfg: dict) -> np.ndarray:
    """Global interior zone index (k n2 + j) n1 + i over the interior, shape (n3, n2, n1).
    For a block of a refined mesh (cfg["block"] = (level, i0, j0, k0, N1l, N2l)),
    the index of the zone in its level's grid, offset by level * 2^40."""
    n1, n2, n3 = cfg["n1"], cfg["n2"], cfg["n3"]
    k, j, i = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    if "block" in cfg:
        lev, i0, j0, k0, N1l, N2l = cfg["block"]
        return (((k + k0) * N2l + (j + j0)) * N1l + (i + i0) + lev * (1 << 40)).astype(np.uint64)
    return ((k * n2 + j) * n1 + i).astype(np.uint64)


# ---------------------------------------------------------------------------
# Grid helpers
# ---------------------------------------------------------------------------
def shape(cfg: dict):
    ng = cfg.get("ng", NG)
    n3 = cfg["n3"]
    return (8, n3 + 2 * ng if n3 > 1 else 1, cfg["n2"] + 2 * ng, cfg["n1"] + 2 * ng)


def interior(cfg: dict):
    """Slices selecting the interior of a (…, N3, N2, N1) array."""
    ng = cfg.get("ng", NG)
    g3 = ng if cfg["n3"] > 1 else 0
    return (slice(g3, g3 + cfg["n3"]), slice(ng, ng + cfg["n2"]), slice(ng, ng + cfg["n1"]))


def centers(cfg: dict, axis: int, face: bool = False) -> np.ndarray:
    """Native coordinates of cell centres (or lower faces) along an axis, ghosts included."""
    ng = cfg.get("ng", NG)
    n = cfg[("n1", "n2", "n3")[axis]]
    lo, hi = cfg[("x1", "x2", "x3")[axis]]
    d = (hi - lo) / n
    g = ng if (axis < 2 or cfg["n3"] > 1) else 0
    idx = np.arange(n + 2 * g)
    return lo + (idx - g + (0.0 if face else 0.5)) * d


# ---------------------------------------------------------------------------
# Problem configurations
# ---------------------------------------------------------------------------
def linear_mode_cfg(n: int, ndim: int = 3, recon: str = "mc") -> dict:
    """Slow-mode box: Minkowski, [0,1]^3 periodic, gamma = 4/3, MC, CFL 0.9."""
    return dict(
        name=f"linear slow mode {n}^{ndim}", coords="minkowski", n1=n, n2=n, n3=n if ndim == 3 else 1,
        recon=recon, bc=["periodic"] * 6, a=0.0, gam=4.0 / 3.0,
        x1=(0.0, 1.0), x2=(0.0, 1.0), x3=(0.0, 1.0), cfl=0.9, floors={},
    )


def bondi_cfg(n1: int = 128, n2: int = 128, recon: str = "mc") -> dict:
    """Bondi: a = 0, MKS h = 0.3, r in [1.8, 50], gamma = 4/3."""
    return dict(
        name=f"bondi mks {n1}x{n2}", coords="mks", n1=n1, n2=n2, n3=1, recon=recon,
        bc=["outflow", "dirichlet", "polar", "polar", "periodic", "periodic"], a=0.0, gam=4.0 / 3.0,
        x1=(math.log(1.8), math.log(50.0)), x2=(0.0, 1.0), x3=(0.0, 2.0 * math.pi), hslope=0.3, cfl=0.9,
        floors=dict(rho_min=1e-6, u_min=1e-8, bsq_rho_max=100.0, bsq_u_max=5000.0, u_rho_max=100.0,
                    gamma_max=50.0),
        r_sonic=8.0,
    )


def torus_cfg(n1: int = 192, n2: int = 96, n3: int = 96, a: float = 0.9375, recon: str = "weno5",
              r_out: float = 1000.0) -> dict:
    """FM torus: funky MKS, spin a, r_out = 1000, 5.5 zones inside the horizon."""
    rh = 1.0 + math.sqrt(1.0 - a * a)
    x1in = (n1 * math.log(rh) - 5.5 * math.log(r_out)) / (n1 - 5.5)
    return dict(
        name=f"fm torus fmks {n1}x{n2}x{n3}", coords="fmks", n1=n1, n2=n2, n3=n3, recon=recon,
        bc=["outflow", "outflow", "polar", "polar", "periodic", "periodic"], a=a, gam=13.0 / 9.0,
        x1=(x1in, math.log(r_out)), x2=(0.0, 1.0), x3=(0.0, 2.0 * math.pi), hslope=0.3, poly_xt=0.82,
        poly_alpha=14.0, mks_smooth=0.5, cfl=0.9,
        floors=dict(rho_min=1e-6, u_min=1e-8, bsq_rho_max=100.0, bsq_u_max=5000.0, u_rho_max=100.0,
                    gamma_max=50.0),
        r_in=6.0, r_max=12.0, beta=100.0,
    )


# ---------------------------------------------------------------------------
# Initial-data geometry (this module's own): native (x1, x2) -> (r, theta),
# the theta derivatives by complex-step differentiation, and the few
# Kerr-Schild quantities needed to express a 4-velocity as u~^i.
# ---------------------------------------------------------------------------
def _theta(cfg: dict, x1, x2):
    if cfg["coords"] == "ks":
        return x2
    h = cfg.get("hslope", 0.3)
    thg = np.pi * x2 + 0.5 * (1.0 - h) * np.sin(2.0 * np.pi * x2)
    if cfg["coords"] == "mks":
        return thg
    xt, al, s = cfg["poly_xt"], cfg["poly_alpha"], cfg["mks_smooth"]
    # continued past the poles by reflection: theta(-x2) = -theta(x2), theta(2 - x2) = 2 pi - theta(x2)
    x2r = np.real(x2)
    if np.any(x2r < 0.0) or np.any(x2r > 1.0):
        lo = x2r < 0.0
        hi = x2r > 1.0
        mid = ~(lo | hi)
        x2m = np.where(lo, -x2, np.where(hi, 2.0 - x2, x2))
        t = _theta(cfg, x1, x2m)
        return np.where(mid, t, np.where(lo, -t, 2.0 * np.pi - t))
    y = 2.0 * x2 - 1.0
    nrm = 0.5 * np.pi / (1.0 + xt ** (-al) / (al + 1.0))
    thj = 0.5 * np.pi + nrm * y * (1.0 + (y / xt) ** int(al) / (al + 1.0))
    return thg + np.exp(s * (cfg.get("x1ref", cfg["x1"][0]) - x1)) * (thj - thg)


def embed(cfg: dict, x1, x2):
    """(r, theta, dtheta/dx1, dtheta/dx2) at native points (MKS family: r = e^x1)."""
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    hstep = 1e-30
    r = np.exp(x1) if cfg["coords"] != "ks" else x1
    th = _theta(cfg, x1, x2)
    th1 = np.imag(_theta(cfg, x1 + 1j * hstep, x2)) / hstep
    th2 = np.imag(_theta(cfg, x1, x2 + 1j * hstep)) / hstep
    return r, th, th1, th2


def _ks_lapse_gtr(a, r, th):
    sig = r * r + a * a * np.cos(th) ** 2
    alpha = 1.0 / np.sqrt(1.0 + 2.0 * r / sig)
    gtr = 2.0 * r / sig  # g^{tr} of Kerr-Schild
    return alpha, gtr, sig


def utilde_from_ks(cfg: dict, x1, x2, ut, ur, uth, uph):
    """Native u~^i from Kerr-Schild u^mu at native points (MKS family).

    u^i_native = (d x^i / d x^a) u^a and u~^i = u^i + gamma alpha g^{0i}, with
    gamma = alpha u^t and g^{0i}_native = g^{tr}_KS d x^i / d r (Kerr-Schild has
    g^{t theta} = g^{t phi} = 0)."""
    a = cfg.get("a", 0.0)
    r, th, th1, th2 = embed(cfg, x1, x2)
    alpha, gtr, _ = _ks_lapse_gtr(a, r, th)
    dx1_dr = 1.0 / r
    dx2_dr = -th1 / (th2 * r)
    dx2_dth = 1.0 / th2
    u1 = dx1_dr * ur
    u2 = dx2_dr * ur + dx2_dth * uth
    u3 = uph
    gamma = alpha * ut
    return (u1 + gamma * alpha * gtr * dx1_dr, u2 + gamma * alpha * gtr * dx2_dr, u3)


def gdet_native(cfg: dict, x1, x2):
    """sqrt(-g) in native coordinates: 1 for Minkowski (Cartesian); for Kerr
    Sigma |sin theta| (dr/dx1) (dtheta/dx2), dr/dx1 = r in the MKS family."""
    if cfg["coords"] == "minkowski":
        return np.ones(np.broadcast(np.asarray(x1), np.asarray(x2)).shape)
    a = cfg.get("a", 0.0)
    r, th, th1, th2 = embed(cfg, x1, x2)
    sig = r * r + a * a * np.cos(th) ** 2
    return sig * np.abs(np.sin(th)) * (r if cfg["coords"] != "ks" else 1.0) * th2


# ---------------------------------------------------------------------------
# Linear slow mode: P = P0 + amp * dP cos(k.x); the eigenvector (dP, omega) is
# supplied by the caller (it is derived from the oracle's flux Jacobians and
# stored as a text fixture).
# ---------------------------------------------------------------------------
LINEAR_BACKGROUND = np.array([1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0])
LINEAR_K = (2.0 * np.pi, 2.0 * np.pi, 0.0)


def linear_mode_state(cfg: dict, dP: np.ndarray, omega: float, t: float = 0.0, amp: float = 1e-4) -> np.ndarray:
    """Analytic mode at time t sampled at cell centres (ghosts included)."""
    x1 = centers(cfg, 0)
    x2 = centers(cfg, 1)
    x3 = centers(cfg, 2)
    X3, X2, X1 = np.meshgrid(x3, x2, x1, indexing="ij")
    phase = LINEAR_K[0] * X1 + LINEAR_K[1] * X2 + LINEAR_K[2] * X3 - omega * t
    P = np.empty(shape(cfg))
    for v in range(8):
        P[v] = LINEAR_BACKGROUND[v] + amp * dP[v] * np.cos(phase)
    return P


def linear_mode_face_field(cfg: dict, dP: np.ndarray, omega: float, t: float = 0.0, amp: float = 1e-4):
    """The mode's field on faces (Minkowski: sqrt(-g) = 1): the uniform
    background plus the curl of the edge potential A = amp (dB x k)/|k|^2
    sin(k.x - omega t), periodic and discretely divergence-free (k.dB = 0)."""
    k = np.array(LINEAR_K)
    dB = np.asarray(dP[5:8], dtype=np.float64)
    Ahat = amp * np.cross(dB, k) / (k @ k)
    c = [centers(cfg, q) for q in range(3)]
    f = [centers(cfg, q, face=True) for q in range(3)]

    def phase(x1, x2, x3):
        X3, X2, X1 = np.meshgrid(x3, x2, x1, indexing="ij")
        return np.sin(k[0] * X1 + k[1] * X2 + k[2] * X3 - omega * t)

    three = cfg["n3"] > 1
    # A1 on x1-edges (i, j-1/2, k-1/2), A2 on x2-edges (i-1/2, j, k-1/2),
    # A3 on x3-edges (i-1/2, j-1/2, k); on a 2-D grid x3 sits at the centre
    z = f[2] if three else c[2]
    A1 = Ahat[0] * phase(c[0], f[1], z)
    A2 = Ahat[1] * phase(f[0], c[1], z)
    A3 = Ahat[2] * phase(f[0], f[1], c[2])
    fB = face_field_from_potential(cfg, A1, A2, A3)
    for q in range(3):
        fB[q] += LINEAR_BACKGROUND[5 + q]
    return fB


def load_eigvec(path: str):
    """(dP[8], omega) from a fixture written by tests/golden/make_linear_mode.py."""
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split("=")
            vals[key.strip()] = val.strip()
    dP = np.array([float(x) for x in vals["dP"].split()])
    return dP, float(vals["omega"])


# ---------------------------------------------------------------------------
# Bondi accretion (Michel 1972 transonic polytrope, M = 1, a = 0):
#   p = K rho^Gamma, n = 1/(Gamma-1), T = p/rho;
#   C1 = r^2 T^n u^r, C2 = (1 + (1+n) T)^2 (1 - 2/r + (u^r)^2);
#   sonic point r_s: u_s^2 = 1/(2 r_s), V_s^2 = u_s^2 / (1 - 3 u_s^2),
#   T_s = n V_s^2 / ((1+n)(1 - n V_s^2)); K such that mdot = 4 pi r^2 rho |u^r| = 1.
# ---------------------------------------------------------------------------
def bondi_constants(gam: float, r_s: float):
    n = 1.0 / (gam - 1.0)
    us = math.sqrt(1.0 / (2.0 * r_s))
    Vs2 = us * us / (1.0 - 3.0 * us * us)
    Ts = n * Vs2 / ((1.0 + n) * (1.0 - n * Vs2))
    C1 = us * r_s * r_s * Ts ** n
    C2 = (1.0 + (1.0 + n) * Ts) ** 2 * (1.0 - 2.0 / r_s + us * us)
    K = (4.0 * math.pi * C1) ** (1.0 / n)
    return n, C1, C2, K, Ts


def bondi_T(r: np.ndarray, gam: float, r_s: float) -> np.ndarray:
    """Temperature T(r) on the accreting branch (subsonic outside r_s, supersonic inside)."""
    n, C1, C2, K, Ts = bondi_constants(gam, r_s)
    r = np.asarray(r, dtype=np.float64)

    def F(T):
        ur = C1 / (r * r * T ** n)
        return (1.0 + (1.0 + n) * T) ** 2 * (1.0 - 2.0 / r + ur * ur) - C2

    # F is convex-like in log T with one minimum; locate it by golden section on log T.
    lo = np.full_like(r, math.log(1e-12))
    hi = np.full_like(r, math.log(1e3))
    g = (math.sqrt(5.0) - 1.0) / 2.0
    for _ in range(200):
        m1 = hi - g * (hi - lo)
        m2 = lo + g * (hi - lo)
        f1 = F(np.exp(m1))
        f2 = F(np.exp(m2))
        left = f1 < f2
        hi = np.where(left, m2, hi)
        lo = np.where(left, lo, m1)
    tmin = np.exp(0.5 * (lo + hi))
    # subsonic (larger-T) root outside r_s, supersonic (smaller-T) root inside
    outside = r >= r_s
    a_ = np.where(outside, tmin, np.full_like(r, 1e-12))
    b_ = np.where(outside, np.full_like(r, 1e3), tmin)
    fa = F(a_)
    for _ in range(400):
        m = 0.5 * (a_ + b_)
        fm = F(m)
        same = np.sign(fm) == np.sign(fa)
        a_ = np.where(same, m, a_)
        fa = np.where(same, fm, fa)
        b_ = np.where(same, b_, m)
    return 0.5 * (a_ + b_)


def bondi_fluid(r: np.ndarray, gam: float, r_s: float):
    """(rho, u, u^r, u^t_KS) of the Bondi solution at radii r."""
    n, C1, C2, K, Ts = bondi_constants(gam, r_s)
    T = bondi_T(r, gam, r_s)
    ur = -C1 / (r * r * T ** n)
    rho = (T / K) ** n
    uint = n * rho * T
    X = 1.0 - 2.0 / r + ur * ur
    # u^t in Kerr-Schild (a = 0), written without the 0/0 at r = 2:
    ut = (r + ur * ur * (r + 2.0)) / (r * np.sqrt(X) - 2.0 * ur)
    return rho, uint, ur, ut


def bondi_prims(cfg: dict, x1, x2):
    r, th, _, _ = embed(cfg, x1, x2)
    rho, uint, ur, ut = bondi_fluid(r, cfg["gam"], cfg["r_sonic"])
    u1, u2, u3 = utilde_from_ks(cfg, x1, x2, ut, ur, 0.0 * ur, 0.0 * ur)
    return rho, uint, u1, u2, u3


def bondi_state(cfg: dict, seed: int = 1, noise: float = 1e-3):
    """(P, dirichlet) for the Bondi problem: analytic solution everywhere, the
    interior's u multiplied by 1 + noise (xi - 1/2), xi = uniform01(seed, zone);
    dirichlet = (None, ghosts of the outer x1 face [8][N3][N2][ng])."""
    ng = cfg.get("ng", NG)
    x1 = centers(cfg, 0)
    x2 = centers(cfg, 1)
    X2, X1 = np.meshgrid(x2, x1, indexing="ij")
    rho, uint, u1, u2, u3 = bondi_prims(cfg, X1, X2)
    P = np.zeros(shape(cfg))
    for v, q in enumerate((rho, uint, u1, u2, u3)):
        P[v] = q[None, :, :]
    if noise:
        sl = interior(cfg)
        xi = uniform01(seed, interior_index(cfg))
        P[1][sl] = P[1][sl] * (1.0 + noise * (xi - 0.5))
    hi = np.ascontiguousarray(P[:, :, :, ng + cfg["n1"]:])
    # the analytic (noise-free) values in the outer ghosts
    for v, q in enumerate((rho, uint, u1, u2, u3)):
        hi[v] = q[None, :, ng + cfg["n1"]:]
    return P, (None, hi)


def bondi_analytic(cfg: dict) -> np.ndarray:
    P, _ = bondi_state(cfg, noise=0.0)
    return P


# ---------------------------------------------------------------------------
# Fishbone & Moncrief (1976) torus, constant l = u^t u_phi, on Kerr (M = 1).
# ---------------------------------------------------------------------------
def _bl_metric_eq(a, r, th):
    """Boyer-Lindquist g_tt, g_tphi, g_phiphi."""
    sig = r * r + a * a * np.cos(th) ** 2
    s2 = np.sin(th) ** 2
    gtt = -(1.0 - 2.0 * r / sig)
    gtp = -2.0 * a * r * s2 / sig
    gpp = s2 * (r * r + a * a + 2.0 * a * a * r * s2 / sig)
    return gtt, gtp, gpp


def fm_angular_momentum(a: float, r_max: float) -> float:
    """l = u^t u_phi of the prograde circular equatorial orbit at r_max
    (Omega = 1 / (r^{3/2} + a))."""
    gtt, gtp, gpp = _bl_metric_eq(a, r_max, 0.5 * math.pi)
    om = 1.0 / (r_max ** 1.5 + a)
    ut = 1.0 / math.sqrt(-(gtt + 2.0 * om * gtp + om * om * gpp))
    uphi_cov = ut * (gtp + om * gpp)
    return ut * uphi_cov


def fm_lnh(a: float, l: float, r, th):
    """ln h of the FM solution, not yet offset by its value at the inner edge
    (NaN inside the horizon, where the torus does not exist)."""
    with np.errstate(invalid="ignore", divide="ignore"):
        return _fm_lnh(a, l, r, th)


def _fm_lnh(a, l, r, th):
    sth = np.sin(th)
    cth = np.cos(th)
    sig = r * r + a * a * cth * cth
    dl = r * r - 2.0 * r + a * a
    A = (r * r + a * a) ** 2 - dl * a * a * sth * sth
    q = np.sqrt(1.0 + 4.0 * l * l * sig * sig * dl / (A * A * sth * sth))
    return 0.5 * np.log((1.0 + q) / (sig * dl / A)) - 0.5 * q - 2.0 * a * r * l / A


def fm_velocity(a: float, l: float, r, th):
    """(u^t, u^phi) in Boyer-Lindquist with u^r = u^theta = 0 and u^t u_phi = l:
    with D = g_tphi^2 - g_tt g_phiphi, (u^t)^2 = (g_phiphi + sqrt(g_phiphi^2 + 4 D l^2)) / (2 D)
    and u^phi = (l/u^t - g_tphi u^t) / g_phiphi."""
    gtt, gtp, gpp = _bl_metric_eq(a, r, th)
    D = gtp * gtp - gtt * gpp
    with np.errstate(invalid="ignore", divide="ignore"):
        ut = np.sqrt((gpp + np.sqrt(gpp * gpp + 4.0 * D * l * l)) / (2.0 * D))
        uph = (l / ut - gtp * ut) / gpp
    return ut, uph


def fm_density(cfg: dict, r, th, kappa: float = 1e-3):
    """(rho, u, inside) of the unnormalised torus (ln h > 0 and r > r_in)."""
    a, gam = cfg["a"], cfg["gam"]
    l = fm_angular_momentum(a, cfg["r_max"])
    lnh = fm_lnh(a, l, r, th) - fm_lnh(a, l, cfg["r_in"], 0.5 * np.pi)
    inside = (lnh > 0.0) & (r > cfg["r_in"])
    h = np.exp(np.where(inside, lnh, 0.0))
    rho = np.where(inside, ((h - 1.0) * (gam - 1.0) / (kappa * gam)) ** (1.0 / (gam - 1.0)), 0.0)
    uint = kappa * rho ** gam / (gam - 1.0)
    return rho, uint, inside


def torus_norms(cfg: dict, kappa: float = 1e-3):
    """(rho_max, field normalisation) of the torus on the grid of cfg."""
    _, info = torus_state(cfg, noise=0.0, kappa=kappa, return_norms=True)
    return info


def torus_state(cfg: dict, seed: int = 2, noise: float = 4e-2, kappa: float = 1e-3, field: bool = True,
                norms=None, return_norms: bool = False):
    """FM torus (rho_max = 1) in an atmosphere at the floors, single poloidal
    loop from A_phi = max(rho/rho_max - 0.2, 0) at corners normalised to
    beta = max(p_gas) / max(p_mag) (p_mag = g_ij B^i B^j / 2), multiplicative
    u noise inside the torus. Returns P with ghosts filled by value (the
    boundary rules refill them)."""
    a = cfg["a"]
    fl = cfg["floors"]
    x1 = centers(cfg, 0)
    x2 = centers(cfg, 1)
    X2, X1 = np.meshgrid(x2, x1, indexing="ij")
    r, th, th1, th2 = embed(cfg, X1, X2)
    rho, uint, inside = fm_density(cfg, r, th, kappa)
    ut_bl, uph = fm_velocity(cfg["a"], fm_angular_momentum(a, cfg["r_max"]), r, th)
    # the torus velocity is defined inside the torus only (NaN e.g. inside the
    # horizon); outside, the atmosphere is at rest: mask before transforming
    ut_bl = np.where(inside, ut_bl, 1.0)
    uph = np.where(inside, uph, 0.0)
    # BL -> KS with u^r = 0: u^t and u^phi are unchanged.
    u1, u2, u3 = utilde_from_ks(cfg, X1, X2, ut_bl, 0.0 * r, 0.0 * r, uph)
    rho_max = rho.max() if norms is None else norms[0]
    rho = rho / rho_max
    uint = uint / rho_max
    rho_atm = np.maximum(fl["rho_min"] * r ** -1.5, 1e-20)
    u_atm = np.maximum(fl["u_min"] * r ** -2.5, 1e-20)
    norm = 0.0
    P2 = np.zeros((8,) + r.shape)
    P2[0] = np.where(inside, rho, rho_atm)
    P2[1] = np.where(inside, uint, u_atm)
    P2[2] = np.where(inside, u1, 0.0)
    P2[3] = np.where(inside, u2, 0.0)
    P2[4] = np.where(inside, u3, 0.0)
    P2[0] = np.maximum(P2[0], rho_atm)
    P2[1] = np.maximum(P2[1], u_atm)
    if field:
        # corner vector potential from the analytic density at the corners
        x1f = centers(cfg, 0, face=True)
        x2f = centers(cfg, 1, face=True)
        Y2, Y1 = np.meshgrid(x2f, x1f, indexing="ij")
        rc, thc, _, _ = embed(cfg, Y1, Y2)
        rhoc, _, insc = fm_density(cfg, rc, thc, kappa)
        Aphi = np.maximum(np.where(insc, rhoc / rho_max, 0.0) - 0.2, 0.0)
        dx1 = x1[1] - x1[0]
        dx2 = x2[1] - x2[0]
        gd = gdet_native(cfg, X1, X2)
        B1 = np.zeros_like(r)
        B2 = np.zeros_like(r)
        # cell (j, i) has corners (j, i), (j, i+1), (j+1, i), (j+1, i+1)
        d2A = (Aphi[1:, :-1] + Aphi[1:, 1:] - Aphi[:-1, :-1] - Aphi[:-1, 1:]) / (2.0 * dx2)
        d1A = (Aphi[:-1, 1:] + Aphi[1:, 1:] - Aphi[:-1, :-1] - Aphi[1:, :-1]) / (2.0 * dx1)
        B1[:-1, :-1] = d2A / gd[:-1, :-1]
        B2[:-1, :-1] = -d1A / gd[:-1, :-1]
        # native spatial metric for the magnetic-pressure proxy (B^3 = 0)
        sig = r * r + a * a * np.cos(th) ** 2
        g_rr = 1.0 + 2.0 * r / sig
        g11 = r * r * g_rr + th1 * th1 * sig
        g12 = th1 * th2 * sig
        g22 = th2 * th2 * sig
        pmag = 0.5 * (g11 * B1 * B1 + 2.0 * g12 * B1 * B2 + g22 * B2 * B2)
        pgas = (cfg["gam"] - 1.0) * P2[1]
        sl = interior(cfg)
        if norms is None:
            norm = math.sqrt((pgas[sl[1], sl[2]].max() / pmag[sl[1], sl[2]].max()) / cfg["beta"])
        else:
            norm = norms[1]
        P2[5] = B1 * norm
        P2[6] = B2 * norm
    P = np.zeros(shape(cfg))
    P[:] = P2[:, None, :, :]
    if noise:
        sl = interior(cfg)
        xi = uniform01(seed, interior_index(cfg))
        ins3 = np.broadcast_to(inside[None, sl[1], sl[2]], xi.shape)
        fac = np.where(ins3, 1.0 + noise * (xi - 0.5), 1.0)
        P[1][sl] = P[1][sl] * fac
    if return_norms:
        return P, (rho_max, norm if field else 0.0)
    return P


# ---------------------------------------------------------------------------
# Minkowski test problems the paper cites beside the linear modes ("Readiness
# and Testing" section): the Orszag-Tang vortex and Komissarov's (1999)
# magnetised cylindrical explosion, in the relativistic setting below (the
# paper names the problems, not their parameters).
# ---------------------------------------------------------------------------
def orszag_tang_cfg(n: int = 256, recon: str = "mc") -> dict:
    """[0, 2 pi)^2 periodic, gamma = 5/3, CFL 0.9."""
    return dict(
        name=f"orszag-tang {n}^2", coords="minkowski", n1=n, n2=n, n3=1, recon=recon, bc=["periodic"] * 6,
        a=0.0, gam=5.0 / 3.0, x1=(0.0, 2 * math.pi), x2=(0.0, 2 * math.pi), x3=(0.0, 1.0), cfl=0.9,
        floors=dict(rho_min=1e-6, u_min=1e-8),
    )


def orszag_tang_state(cfg: dict, v0: float = 0.5, B0: float = 1.0) -> np.ndarray:
    """rho = 25/9, p = 5/3, 3-velocity v = v0 (-sin y, sin x), B = B0 (-sin y,
    sin 2x); u~ = W v. The state is odd under the half-turn about the
    centre ((x, y) -> (2 pi - x, 2 pi - y), v -> -v, B -> -B)."""
    X2, X1 = np.meshgrid(centers(cfg, 1), centers(cfg, 0), indexing="ij")
    v1, v2 = -v0 * np.sin(X2), v0 * np.sin(X1)
    W = 1.0 / np.sqrt(1.0 - v1 * v1 - v2 * v2)
    P = np.zeros(shape(cfg))
    P[0] = 25.0 / 9.0
    P[1] = (5.0 / 3.0) / (cfg["gam"] - 1.0)
    P[2], P[3] = W * v1, W * v2
    P[5], P[6] = -B0 * np.sin(X2), B0 * np.sin(2.0 * X1)
    return P


def explosion_cfg(n: int = 256, recon: str = "mc", B0: float = 0.1) -> dict:
    """[-6, 6]^2, outflow boundaries, gamma = 4/3, CFL 0.5."""
    return dict(
        name=f"cylindrical explosion {n}^2", coords="minkowski", n1=n, n2=n, n3=1, recon=recon,
        bc=["outflow", "outflow", "outflow", "outflow", "periodic", "periodic"], a=0.0, gam=4.0 / 3.0,
        x1=(-6.0, 6.0), x2=(-6.0, 6.0), x3=(0.0, 1.0), cfl=0.5, B0=B0,
        floors=dict(rho_min=1e-8, u_min=1e-10, bsq_rho_max=1e4, bsq_u_max=1e6),
    )


def explosion_state(cfg: dict) -> np.ndarray:
    """Komissarov (1999): rho = 1e-2, p = 1 for r < 0.8; rho = 1e-4, p = 5e-4
    for r > 1; log-linear in r between; at rest; uniform B = (B0, 0, 0).
    Mirror-symmetric about both axes (x -> -x with u~1, B2, B3 odd; y -> -y
    with u~2, B2 odd)."""
    X2, X1 = np.meshgrid(centers(cfg, 1), centers(cfg, 0), indexing="ij")
    r = np.sqrt(X1 * X1 + X2 * X2)
    w = np.clip((r - 0.8) / 0.2, 0.0, 1.0)
    rho = np.exp((1 - w) * np.log(1e-2) + w * np.log(1e-4))
    p = np.exp((1 - w) * np.log(1.0) + w * np.log(5e-4))
    P = np.zeros(shape(cfg))
    P[0] = rho
    P[1] = p / (cfg["gam"] - 1.0)
    P[5] = cfg.get("B0", 0.1)
    return P


# ---------------------------------------------------------------------------
# Face-centred fields (for face-centred constrained transport): arrays
# (3, N3, N2, N1), entry a = sqrt(-g) B^(a+1) on the lower x^(a+1) face of
# each cell (a 2-D grid keeps sqrt(-g) B^3 per cell).
# ---------------------------------------------------------------------------
def _fwd(A, axis: int, d: float):
    """Forward difference along an array axis / d; the last entry (no upper
    neighbour) is 0."""
    out = np.zeros_like(A)
    sl_hi = [slice(None)] * 3
    sl_lo = [slice(None)] * 3
    sl_hi[axis] = slice(1, None)
    sl_lo[axis] = slice(None, -1)
    out[tuple(sl_lo)] = (A[tuple(sl_hi)] - A[tuple(sl_lo)]) / d
    return out


def face_field_from_potential(cfg: dict, A1=None, A2=None, A3=None) -> np.ndarray:
    """The discrete curl of an edge vector potential: A1 on x1-edges
    (i, j-1/2, k-1/2), A2 on x2-edges (i-1/2, j, k-1/2), A3 on x3-edges
    (i-1/2, j-1/2, k), each (N3, N2, N1) or None (= 0); on a 2-D grid A1 sits on
    x2 faces and A2 on x1 faces. sqrt(-g) B^a = eps^{abc} d_b A_c, so the face
    divergence is zero up to rounding."""
    N = shape(cfg)[1:]
    z = np.zeros(N)
    A1 = z if A1 is None else np.asarray(A1, dtype=np.float64)
    A2 = z if A2 is None else np.asarray(A2, dtype=np.float64)
    A3 = z if A3 is None else np.asarray(A3, dtype=np.float64)
    dx = [(cfg[k][1] - cfg[k][0]) / cfg[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3"))]
    three = cfg["n3"] > 1
    # array axes: 0 = x3, 1 = x2, 2 = x1
    fB = np.zeros((3,) + N)
    fB[0] = _fwd(A3, 1, dx[1]) - (_fwd(A2, 0, dx[2]) if three else 0.0)
    fB[1] = (_fwd(A1, 0, dx[2]) if three else 0.0) - _fwd(A3, 2, dx[0])
    fB[2] = _fwd(A2, 2, dx[0]) - _fwd(A1, 1, dx[1])
    return fB


def random_face_field(cfg: dict, seed: int, scale: float = 1.0) -> np.ndarray:
    """A divergence-free face field of magnitude ~scale with grid-scale
    structure: the curl of seeded uniform edge potentials, drawn per interior
    edge and repeated periodically into the ghost rows (so that on a periodic
    grid a face and its periodic image carry the same value)."""
    N = shape(cfg)[1:]
    ng = cfg.get("ng", NG)
    g3 = ng if cfg["n3"] > 1 else 0
    dx = min((cfg[k][1] - cfg[k][0]) / cfg[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3")))
    k, j, i = np.meshgrid((np.arange(N[0]) - g3) % cfg["n3"], (np.arange(N[1]) - ng) % cfg["n2"],
                          (np.arange(N[2]) - ng) % cfg["n1"], indexing="ij")
    idx = (k * cfg["n2"] + j) * cfg["n1"] + i
    A = [scale * dx * (uniform01(seed + 101 * q, idx) - 0.5) for q in range(3)]
    return face_field_from_potential(cfg, *A)


def cell_field_from_faces(cfg: dict, fB: np.ndarray, P: np.ndarray) -> np.ndarray:
    """P with the B^i of every cell that has both faces (all but the last
    row along each axis) set to the face means over sqrt(-g)."""
    P = np.array(P, dtype=np.float64, copy=True)
    X2, X1 = np.meshgrid(centers(cfg, 1), centers(cfg, 0), indexing="ij")
    gd = gdet_native(cfg, X1, X2)[None, :, :]
    m1 = np.zeros_like(fB[0])
    m2 = np.zeros_like(fB[1])
    m1[:, :, :-1] = 0.5 * (fB[0][:, :, :-1] + fB[0][:, :, 1:])
    m2[:, :-1, :] = 0.5 * (fB[1][:, :-1, :] + fB[1][:, 1:, :])
    if cfg["n3"] > 1:
        m3 = np.zeros_like(fB[2])
        m3[:-1] = 0.5 * (fB[2][:-1] + fB[2][1:])
    else:
        m3 = fB[2].copy()
    P[5], P[6], P[7] = m1 / gd, m2 / gd, m3 / gd
    return P


def torus_face_field(cfg: dict, kappa: float = 1e-3, norms=None) -> np.ndarray:
    """The FM torus's poloidal loop as a face field: A_phi at cell corners as in
    torus_state (the same normalisation), curled onto the faces. Its face means
    over sqrt(-g) are torus_state's cell-centred B^1, B^2."""
    if norms is None:
        _, norms = torus_state(cfg, noise=0.0, kappa=kappa, return_norms=True)
    rho_max, norm = norms
    x1f = centers(cfg, 0, face=True)
    x2f = centers(cfg, 1, face=True)
    Y2, Y1 = np.meshgrid(x2f, x1f, indexing="ij")
    rc, thc, _, _ = embed(cfg, Y1, Y2)
    rhoc, _, insc = fm_density(cfg, rc, thc, kappa)
    Aphi = np.maximum(np.where(insc, rhoc / rho_max, 0.0) - 0.2, 0.0) * norm
    A3 = np.broadcast_to(Aphi[None, :, :], shape(cfg)[1:])
    return face_field_from_potential(cfg, None, None, A3)


# ---------------------------------------------------------------------------
# Random physical states for single-kernel parity (p2c / c2p).
# ---------------------------------------------------------------------------
def random_prims(cfg: dict, seed: int, rho_range=(1e-4, 1.0), u_range=(1e-6, 1.0), ut_scale=(1.0, 1.0, 1.0),
                 b_scale=(1.0, 1.0, 1.0), b_sqrt_rho: bool = True) -> np.ndarray:
    """Log-uniform rho and u, uniform u~^i in [-s_i, s_i], uniform B^i in
    [-b_i, b_i] (times sqrt(rho) when b_sqrt_rho, so that b^2/rho stays of
    order sum b_i^2), every cell (ghosts included) from the counter-based stream."""
    shp = shape(cfg)
    n = int(np.prod(shp[1:]))
    base = np.arange(n, dtype=np.uint64)
    P = np.zeros(shp)

    def draw(slot):
        return uniform01(seed * 16 + slot, base).reshape(shp[1:])

    # in curved coordinates scale u~^i and B^i by 1/sqrt(g_ii) so that the
    # ranges are orthonormal-frame magnitudes
    if cfg["coords"] != "minkowski":
        x1 = centers(cfg, 0)
        x2 = centers(cfg, 1)
        X2, X1 = np.meshgrid(x2, x1, indexing="ij")
        a = cfg.get("a", 0.0)
        r, th, th1, th2 = embed(cfg, X1, X2)
        sig = r * r + a * a * np.cos(th) ** 2
        s2 = np.sin(th) ** 2
        z = 2.0 * r / sig
        diag = [np.sqrt(r * r * (1.0 + z) + th1 * th1 * sig), np.sqrt(th2 * th2 * sig),
                np.sqrt(s2 * (sig + a * a * s2 * (1.0 + z)))]
        diag = [np.broadcast_to(dd[None], shp[1:]) for dd in diag]
    else:
        diag = [1.0, 1.0, 1.0]
    lr = np.log(rho_range)
    lu = np.log(u_range)
    P[0] = np.exp(lr[0] + (lr[1] - lr[0]) * draw(0))
    P[1] = np.exp(lu[0] + (lu[1] - lu[0]) * draw(1))
    for q in range(3):
        P[2 + q] = ut_scale[q] * (2.0 * draw(2 + q) - 1.0) / diag[q]
        P[5 + q] = b_scale[q] * (2.0 * draw(5 + q) - 1.0) / diag[q]
        if b_sqrt_rho:
            P[5 + q] *= np.sqrt(P[0])
    return P


# ---------------------------------------------------------------------------
# Statically refined meshes: per-block problem configurations.
# ---------------------------------------------------------------------------
def block_cfg(base: dict, blk: dict) -> dict:
    """Configuration of one block (level l, interior box [i0, i0+n1) x ... in
    level-l indices) of a mesh whose level-0 grid is base: same coordinates and
    scheme, the block's box as the native extent, base's x1 start as the FMKS
    reference, boundaries that are physical only where the block touches them."""
    lev = blk["level"]
    r3 = 2 if base["n3"] > 1 else 1
    rr = (2 ** lev, 2 ** lev, r3 ** lev)
    cfg = dict(base)
    ext = []
    for d, key, nk, ok in ((0, "x1", "n1", "i0"), (1, "x2", "n2", "j0"), (2, "x3", "n3", "k0")):
        lo, hi = base[key]
        dx = (hi - lo) / (base[nk] * rr[d])
        ext.append((lo + blk[ok] * dx, lo + (blk[ok] + blk[nk]) * dx))
        cfg[nk] = blk[nk]
    cfg["x1"], cfg["x2"], cfg["x3"] = ext
    cfg["x1ref"] = base["x1"][0]
    bc = list(base["bc"])
    nl = [base["n1"] * rr[0], base["n2"] * rr[1], base["n3"] * rr[2]]
    for d, ok, nk in ((0, "i0", "n1"), (1, "j0", "n2"), (2, "k0", "n3")):
        if blk[ok] != 0:
            bc[2 * d] = "outflow" if bc[2 * d] == "polar" else bc[2 * d]
        if blk[ok] + blk[nk] != nl[d]:
            bc[2 * d + 1] = "outflow" if bc[2 * d + 1] == "polar" else bc[2 * d + 1]
    cfg["bc"] = bc
    cfg["block"] = (lev, blk["i0"], blk["j0"], blk["k0"], nl[0], nl[1])
    return cfg


def _tile(level, box, size):
    """Blocks of `size` (n1, n2, n3) tiling the level-`level` index box
    ((i0, i1), (j0, j1), (k0, k1)); every extent must divide evenly."""
    (i0, i1), (j0, j1), (k0, k1) = box
    s1, s2, s3 = size
    assert (i1 - i0) % s1 == 0 and (j1 - j0) % s2 == 0 and (k1 - k0) % s3 == 0
    return [dict(level=level, i0=i, j0=j, k0=k, n1=s1, n2=s2, n3=s3)
            for k in range(k0, k1, s3) for j in range(j0, j1, s2) for i in range(i0, i1, s1)]


def smr_torus_layout(n1: int = 128, n2: int = 64, n3: int = 64):
    """Three-level static refinement of the torus grid (base n1 x n2 x n3 at
    level 0): level 2 over the inner half in x1 and the middle quarter in x2
    (the disc), level 1 around it (the inner three quarters in x1, the middle
    half in x2), level 0 elsewhere (the polar caps and the outer x1 quarter).
    Blocks: 16x16x32 at level 2; 16x32x32 and 32x16x32 at level 1; 32^3 and
    32x16x32 at level 0. At the default size: 592 blocks, 5,570,560 zones."""
    q1, q2 = n1 // 4, n2 // 8
    L2 = _tile(2, ((0, 8 * q1), (4 * 3 * q2, 4 * 5 * q2), (0, 4 * n3)), (16, 16, 32))
    L1 = (_tile(1, ((2 * 2 * q1, 2 * 3 * q1), (2 * 2 * q2, 2 * 6 * q2), (0, 2 * n3)), (16, 32, 32))
          + _tile(1, ((0, 2 * 2 * q1), (2 * 2 * q2, 2 * 3 * q2), (0, 2 * n3)), (32, 16, 32))
          + _tile(1, ((0, 2 * 2 * q1), (2 * 5 * q2, 2 * 6 * q2), (0, 2 * n3)), (32, 16, 32)))
    L0 = (_tile(0, ((3 * q1, n1), (0, n2), (0, n3)), (32, 32, 32))
          + _tile(0, ((0, 3 * q1), (0, 2 * q2), (0, n3)), (32, 16, 32))
          + _tile(0, ((0, 3 * q1), (6 * q2, n2), (0, n3)), (32, 16, 32)))
    return torus_cfg(n1, n2, n3), L0 + L1 + L2
