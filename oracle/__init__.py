"""Python binding of the FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA library
in ``paper_2408_01361_gb300``; the two meet only through the seeded inputs of
``paper_2408_01361_gb300.inputs`` (which holds none of the method's arithmetic).

Arrays are numpy float64 of shape (8, N3, N2, N1), ghosts included and not
padded, slot order (rho, u, u~1, u~2, u~3, B1, B2, B3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, f) for f in ("harm_oracle.cpp", "harm_oracle.hpp", "dual.hpp", "opcount.hpp")]

KIND = {"minkowski": 0, "ks": 1, "mks": 2, "fmks": 3}
BC = {"periodic": 0, "outflow": 1, "polar": 2, "dirichlet": 3}
RECON = {"mc": 0, "weno5": 1, "donor": 2}


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (plain g++, OpenMP, no CPU-specific flags;
    no fused multiply-add contraction, so that it rounds alike on every host)."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        cmd = ["g++", "-std=c++17", "-O3", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", _LIB_PATH,
               os.path.join(_HERE, "harm_oracle.cpp")]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("ng", C.c_int),
        ("recon", C.c_int), ("bc", C.c_int * 6),
        ("a", C.c_double), ("gam", C.c_double),
        ("x1min", C.c_double), ("x1max", C.c_double), ("x2min", C.c_double),
        ("x2max", C.c_double), ("x3min", C.c_double), ("x3max", C.c_double),
        ("hslope", C.c_double), ("poly_xt", C.c_double), ("poly_alpha", C.c_double),
        ("mks_smooth", C.c_double), ("cfl", C.c_double),
        ("rho_min", C.c_double), ("u_min", C.c_double), ("bsq_rho_max", C.c_double),
        ("bsq_u_max", C.c_double), ("u_rho_max", C.c_double), ("gamma_max", C.c_double),
        ("x1ref", C.c_double), ("fofc", C.c_int), ("bfield", C.c_int), ("emf", C.c_int),
        ("integrator", C.c_int),
    ]


BFIELD = {"fluxct": 0, "face": 1}
EMF = {"average": 0, "gs05": 1}
INTEGRATOR = {"vl2": 0, "rk1": 1, "rk2": 2, "ssprk54": 3}


def params(cfg: dict) -> Params:
    """ctypes parameter block from a problem configuration dict."""
    p = Params()
    p.kind = KIND[cfg["coords"]]
    p.n1, p.n2, p.n3 = cfg["n1"], cfg["n2"], cfg["n3"]
    p.ng = cfg.get("ng", 3)
    p.recon = RECON[cfg["recon"]]
    for q, b in enumerate(cfg["bc"]):
        p.bc[q] = BC[b]
    p.a = cfg.get("a", 0.0)
    p.gam = cfg["gam"]
    (p.x1min, p.x1max), (p.x2min, p.x2max), (p.x3min, p.x3max) = cfg["x1"], cfg["x2"], cfg["x3"]
    p.hslope = cfg.get("hslope", 0.3)
    p.poly_xt = cfg.get("poly_xt", 0.82)
    p.poly_alpha = cfg.get("poly_alpha", 14.0)
    p.mks_smooth = cfg.get("mks_smooth", 0.5)
    p.cfl = cfg.get("cfl", 0.9)
    fl = cfg.get("floors", {})
    p.rho_min = fl.get("rho_min", 1e-20)
    p.u_min = fl.get("u_min", 1e-20)
    p.bsq_rho_max = fl.get("bsq_rho_max", 1e300)
    p.bsq_u_max = fl.get("bsq_u_max", 1e300)
    p.u_rho_max = fl.get("u_rho_max", 1e300)
    p.gamma_max = fl.get("gamma_max", 1e300)
    p.x1ref = cfg.get("x1ref", cfg["x1"][0])
    p.fofc = int(bool(cfg.get("fofc", False)))
    p.bfield = BFIELD[cfg.get("bfield", "fluxct")]
    p.emf = EMF[cfg.get("emf", "gs05")]
    p.integrator = INTEGRATOR[cfg.get("integrator", "vl2")]
    return p


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        PP = C.POINTER(Params)
        L.or_set_threads.argtypes = [C.c_int]
        L.or_get_threads.restype = C.c_int
        L.or_geometry.argtypes = [PP, C.c_int, _dp, _dp, _dp, _dp]
        L.or_connection.argtypes = [PP, _dp]
        L.or_metric_points.argtypes = [PP, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_native_to_ks.argtypes = [PP, C.c_int, _dp, _dp, _dp, _dp]
        L.or_prim_to_cons.argtypes = [PP, _dp, _dp]
        L.or_cons_to_prim.argtypes = [PP, _dp, _dp, C.c_void_p]
        L.or_cons_to_prim.restype = C.c_long
        L.or_apply_bc.argtypes = [PP, _dp, C.c_void_p, C.c_void_p]
        L.or_fluxes.argtypes = [PP, _dp] + [C.c_void_p] * 6
        L.or_cfl_dt.argtypes = [PP, _dp, C.c_void_p, C.c_void_p]
        L.or_cfl_dt.restype = C.c_double
        L.or_step.argtypes = [PP, _dp, _dp, C.c_double, C.c_void_p, C.c_void_p, C.POINTER(C.c_long)]
        L.or_step.restype = C.c_double
        L.or_step_jvp.argtypes = [PP, _dp, _dp, _dp, _dp, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.POINTER(C.c_long)]
        L.or_step_jvp.restype = C.c_double
        L.or_evolve.argtypes = [PP, _dp, _dp, C.c_int, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                C.POINTER(C.c_long)]
        L.or_evolve.restype = C.c_double
        L.or_divb.argtypes = [PP, _dp, _dp, C.c_void_p]
        L.or_stage.argtypes = [PP, _dp, _dp, C.c_double, _dp, _dp, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(C.c_long), C.c_void_p, C.c_void_p]
        L.or_rk_table.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp]
        L.or_rk_table.restype = C.c_int
        L.or_point_flux.argtypes = [C.c_double, _dp, _dp, C.c_int, _dp]
        L.or_point_state.argtypes = [_dp, _dp, _dp]
        L.or_point_speeds.argtypes = [C.c_double, _dp, _dp, C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]
        L.or_point_llf.argtypes = [C.c_double, _dp, _dp, _dp, C.c_int, _dp, C.POINTER(C.c_double)]
        L.or_point_c2p.argtypes = [C.c_double, _dp, _dp, _dp]
        L.or_point_c2p.restype = C.c_int
        L.or_point_jacobians.argtypes = [C.c_double, _dp, _dp, C.c_int, _dp, _dp]
        L.or_point_source.argtypes = [PP, C.c_double, C.c_double, _dp, _dp]
        L.or_recon.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
        L.or_point_floors.argtypes = [PP, C.c_double, C.c_double, _dp]
        L.or_point_floors.restype = C.c_int
        L.or_count_ops.argtypes = [PP, C.c_double, C.c_double, _dp, _dp]
        L.or_fofc_flags.argtypes = [PP, _dp, _dp, C.c_double, _ip]
        L.or_step_face.argtypes = [PP, _dp, _dp, _dp, C.c_double, C.c_void_p, C.c_void_p, C.POINTER(C.c_long)]
        L.or_step_face.restype = C.c_double
        L.or_face_divb.argtypes = [PP, _dp, _dp, C.c_void_p]
        L.or_face_to_cell.argtypes = [PP, _dp, _dp]
        L.or_face_emfs.argtypes = [PP, _dp, _dp]
        L.or_stage_face.argtypes = [PP, _dp, _dp, C.c_double, _dp, _dp, _dp, _dp, _dp, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_long)]
        L.or_fofc_flags.restype = C.c_long
    return _lib


# zones flagged by the first-order flux correction in the last step/stage call
last_nfofc = 0


def _note(st):
    global last_nfofc
    last_nfofc = int(st[3])


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return lib().or_get_threads()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def shape(cfg: dict):
    ng = cfg.get("ng", 3)
    n3 = cfg["n3"]
    return (8, n3 + 2 * ng if n3 > 1 else 1, cfg["n2"] + 2 * ng, cfg["n1"] + 2 * ng)


def geometry(cfg: dict, loc: int = 0):
    """(gcov, gcon, gdet, alpha) over the (N2, N1) ghosted grid at a location
    (0 centre, 1 x1 face, 2 x2 face, 3 x3 face, 4 corner)."""
    _, _, N2, N1 = shape(cfg)
    gcov = np.zeros((N2, N1, 4, 4)); gcon = np.zeros((N2, N1, 4, 4))
    gdet = np.zeros((N2, N1)); alpha = np.zeros((N2, N1))
    lib().or_geometry(C.byref(params(cfg)), loc, gcov, gcon, gdet, alpha)
    return gcov, gcon, gdet, alpha


def connection(cfg: dict):
    _, _, N2, N1 = shape(cfg)
    out = np.zeros((N2, N1, 4, 4, 4))
    lib().or_connection(C.byref(params(cfg)), out)
    return out


def metric_points(cfg: dict, x1, x2):
    x1 = np.ascontiguousarray(x1, dtype=np.float64); x2 = np.ascontiguousarray(x2, dtype=np.float64)
    n = x1.size
    gcov = np.zeros((n, 4, 4)); gcon = np.zeros((n, 4, 4)); gdet = np.zeros(n); conn = np.zeros((n, 4, 4, 4))
    lib().or_metric_points(C.byref(params(cfg)), n, x1, x2, gcov, gcon, gdet, conn)
    return gcov, gcon, gdet, conn


def native_to_ks(cfg: dict, x1, x2):
    x1 = np.ascontiguousarray(x1, dtype=np.float64); x2 = np.ascontiguousarray(x2, dtype=np.float64)
    r = np.zeros(x1.size); th = np.zeros(x1.size)
    lib().or_native_to_ks(C.byref(params(cfg)), x1.size, x1, x2, r, th)
    return r, th


def prim_to_cons(cfg: dict, P):
    P = np.ascontiguousarray(P, dtype=np.float64)
    U = np.zeros_like(P)
    lib().or_prim_to_cons(C.byref(params(cfg)), P, U)
    return U


def cons_to_prim(cfg: dict, U, P_guess):
    """Returns (P, pflag, nfail); P keeps the guess where the inversion failed."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    P = np.array(P_guess, dtype=np.float64, order="C", copy=True)
    pflag = np.zeros(P.shape[1:], dtype=np.int32)
    nfail = lib().or_cons_to_prim(C.byref(params(cfg)), U, P, _ptr(pflag))
    return P, pflag, int(nfail)


def apply_bc(cfg: dict, P, dirichlet=None):
    P = np.array(P, dtype=np.float64, order="C", copy=True)
    lo, hi = (dirichlet or (None, None))
    lib().or_apply_bc(C.byref(params(cfg)), P, _ptr(lo), _ptr(hi))
    return P


def fluxes(cfg: dict, P):
    """Fluxes after polar zeroing and Flux-CT from P (ghosts must be filled)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    F = [np.zeros_like(P) for _ in range(3)]
    ct = [np.zeros(P.shape[1:]) for _ in range(3)]
    lib().or_fluxes(C.byref(params(cfg)), P, *[_ptr(f) for f in F], *[_ptr(c) for c in ct])
    return F, ct


def cfl_dt(cfg: dict, P, dirichlet=None) -> float:
    P = np.ascontiguousarray(P, dtype=np.float64)
    lo, hi = (dirichlet or (None, None))
    return lib().or_cfl_dt(C.byref(params(cfg)), P, _ptr(lo), _ptr(hi))


def step(cfg: dict, U, P, dt: float, dirichlet=None):
    """One two-stage step. Returns (U, P, dt_next, stats[nfail, nfloor, nunfixed])."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    P = np.array(P, dtype=np.float64, order="C", copy=True)
    lo, hi = (dirichlet or (None, None))
    st = (C.c_long * 4)()
    dtn = lib().or_step(C.byref(params(cfg)), U, P, float(dt), _ptr(lo), _ptr(hi), st)
    _note(st)
    return U, P, dtn, list(st)[:3]


def step_jvp(cfg: dict, U, P, dU, dP, dgam: float, dt: float, dirichlet=None, flux: bool = False):
    """One step and its directional derivative (dual numbers through the same
    stages; dt fixed). Returns (U, P, dU, dP, dt_next, stats, zflag) -- zflag
    per zone: 1 = an inversion failed (fixed up, frozen), 2 = a floor acted --
    and, with flux=True, also the tangent of the stage-2 x1 fluxes (cell
    layout)."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    P = np.array(P, dtype=np.float64, order="C", copy=True)
    dU = np.array(dU, dtype=np.float64, order="C", copy=True)
    dP = np.array(dP, dtype=np.float64, order="C", copy=True)
    dF1 = np.zeros_like(P) if flux else None
    zflag = np.zeros(P.shape[1:], dtype=np.int32)
    lo, hi = (dirichlet or (None, None))
    st = (C.c_long * 4)()
    dtn = lib().or_step_jvp(C.byref(params(cfg)), U, P, dU, dP, float(dgam), float(dt), _ptr(lo), _ptr(hi),
                            _ptr(dF1), _ptr(zflag), st)
    _note(st)
    out = (U, P, dU, dP, dtn, list(st)[:3], zflag)
    return out + (dF1,) if flux else out


def evolve(cfg: dict, U, P, nsteps: int, dt: float, t_end: float = 0.0, dirichlet=None):
    """nsteps steps (or until t_end); dt > 0 fixed, dt < 0: first step -dt, then CFL.
    Returns (U, P, t, stats)."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    P = np.array(P, dtype=np.float64, order="C", copy=True)
    lo, hi = (dirichlet or (None, None))
    st = (C.c_long * 4)()
    t = lib().or_evolve(C.byref(params(cfg)), U, P, int(nsteps), float(dt), float(t_end), _ptr(lo), _ptr(hi), st)
    _note(st)
    return U, P, t, list(st)[:3]


def divb(cfg: dict, P, field: bool = False):
    P = np.ascontiguousarray(P, dtype=np.float64)
    out = np.zeros(2)
    div = np.zeros(P.shape[1:]) if field else None
    lib().or_divb(C.byref(params(cfg)), P, out, _ptr(div))
    return (out[0], out[1], div) if field else (out[0], out[1])


# ---- point-level helpers -------------------------------------------------
def _g16(gcov):
    return np.ascontiguousarray(np.asarray(gcov, dtype=np.float64).reshape(16))


def point_flux(gam, gcov, P, d):
    F = np.zeros(8)
    lib().or_point_flux(float(gam), _g16(gcov), np.ascontiguousarray(P, dtype=np.float64), int(d), F)
    return F


def point_state(gcov, P):
    out = np.zeros(9)
    lib().or_point_state(_g16(gcov), np.ascontiguousarray(P, dtype=np.float64), out)
    return out[:4], out[4:8], out[8]


def point_speeds(gam, gcov, P, d):
    cmax = C.c_double(); cmin = C.c_double()
    lib().or_point_speeds(float(gam), _g16(gcov), np.ascontiguousarray(P, dtype=np.float64), int(d),
                          C.byref(cmax), C.byref(cmin))
    return cmax.value, cmin.value


def point_llf(gam, gcov, PL, PR, d):
    F = np.zeros(8); ct = C.c_double()
    lib().or_point_llf(float(gam), _g16(gcov), np.ascontiguousarray(PL, dtype=np.float64),
                       np.ascontiguousarray(PR, dtype=np.float64), int(d), F, C.byref(ct))
    return F, ct.value


def point_c2p(gam, gcov, U, P_guess):
    P = np.array(P_guess, dtype=np.float64, copy=True)
    flag = lib().or_point_c2p(float(gam), _g16(gcov), np.ascontiguousarray(U, dtype=np.float64), P)
    return P, flag


def point_jacobians(gam, gcov, P, d):
    dF = np.zeros((8, 8)); dU = np.zeros((8, 8))
    lib().or_point_jacobians(float(gam), _g16(gcov), np.ascontiguousarray(P, dtype=np.float64), int(d), dF, dU)
    return dF, dU


def point_source(cfg, x1, x2, P):
    S = np.zeros(8)
    lib().or_point_source(C.byref(params(cfg)), float(x1), float(x2), np.ascontiguousarray(P, dtype=np.float64), S)
    return S


def point_floors(cfg, x1, x2, P):
    """Floors of one state at native (x1, x2): (floored P, bit mask 1 density or
    energy floor, 2 u/rho ceiling, 4 Lorentz-factor ceiling)."""
    P = np.array(P, dtype=np.float64, copy=True)
    flag = lib().or_point_floors(C.byref(params(cfg)), float(x1), float(x2), P)
    return P, flag


def recon(kind: str, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    lo = np.full_like(q, np.nan); hi = np.full_like(q, np.nan)
    lib().or_recon(RECON[kind], q.size, q, lo, hi)
    return lo, hi


def stage(cfg: dict, U0, Pin, cdt: float, Uout, Pout, dU=None, fofc_flags=None):
    """One stage on a grid with caller-filled ghosts; Uout/Pout updated in place
    (interior); dU (optional, full array) receives the raw increment
    cdt (-div F + S) of every interior zone; fofc_flags (optional, int32 per
    cell, ghosts included; cfg with "fofc"): the flux correction's flagged
    zones, used instead of the grid's own trial. Returns (ctop[3] arrays,
    stats)."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    Pin = np.ascontiguousarray(Pin, dtype=np.float64)
    ct = [np.zeros(Pin.shape[1:]) for _ in range(3)]
    st = (C.c_long * 4)()
    fl = None if fofc_flags is None else np.ascontiguousarray(fofc_flags, dtype=np.int32)
    lib().or_stage(C.byref(params(cfg)), U0, Pin, float(cdt), Uout, Pout, *[_ptr(c) for c in ct], st, _ptr(dU),
                   _ptr(fl))
    _note(st)
    return ct, list(st)[:3]


def rk_table(integrator: str):
    """The stages of a Runge-Kutta integrator ("rk1", "rk2", "ssprk54") in
    Shu-Osher form: a list of (sources, weights, c_s, weight of stage 4's raw
    increment); stage s forms sum_t w_t U_src_t (+ that increment term) and adds
    c_s dt L(P_{s-1})."""
    n = np.zeros(5, dtype=np.int32); src = np.zeros(15, dtype=np.int32)
    a = np.zeros(15); cdt = np.zeros(5); du4 = np.zeros(5)
    ns = lib().or_rk_table(INTEGRATOR[integrator], n, src, a, cdt, du4)
    return [([int(src[3 * s + t]) for t in range(n[s])], [float(a[3 * s + t]) for t in range(n[s])],
             float(cdt[s]), float(du4[s])) for s in range(ns)]


def count_ops(cfg: dict, x1: float, x2: float, P):
    """Floating-point operations of the method's per-item formulas (oracle
    point physics on the counting type): dict with weno5 (one face value),
    mc (one cell), llf (one face from its two states), sources (one zone),
    p2c (one zone)."""
    out = np.zeros(5)
    lib().or_count_ops(C.byref(params(cfg)), float(x1), float(x2), np.ascontiguousarray(P, dtype=np.float64), out)
    return dict(zip(("weno5", "mc", "llf", "sources", "p2c"), out.tolist()))


def fofc_flags(cfg: dict, U0, Pin, cdt: float):
    """Zones the first-order flux correction flags in one stage (Pin with its
    ghosts filled): int array over the cells, 1 = flagged."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    Pin = np.ascontiguousarray(Pin, dtype=np.float64)
    flags = np.zeros(Pin.shape[1:], dtype=np.int32)
    lib().or_fofc_flags(C.byref(params(cfg)), U0, Pin, float(cdt), flags)
    return flags


def step_face(cfg: dict, U, P, fB, dt: float, dirichlet=None):
    """One two-stage step with face-centred constrained transport (cfg
    "bfield": "face"). fB: [3][N3][N2][N1], sqrt(-g) B^(a+1) on the lower
    x^(a+1) face of each cell. Returns (U, P, fB, dt_next, stats[3])."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    P = np.array(P, dtype=np.float64, order="C", copy=True)
    fB = np.array(fB, dtype=np.float64, order="C", copy=True)
    lo, hi = (dirichlet or (None, None))
    st = (C.c_long * 4)()
    dtn = lib().or_step_face(C.byref(params(cfg)), U, P, fB, float(dt), _ptr(lo), _ptr(hi), st)
    if dtn < 0:
        raise ValueError("or_step_face: needs bfield 'face' and no flux correction")
    _note(st)
    return U, P, fB, dtn, list(st)[:3]


def face_divb(cfg: dict, fB, field: bool = False):
    """Face divergence of a face field: (max |div|, mean |div|[, per cell])."""
    fB = np.ascontiguousarray(fB, dtype=np.float64)
    out = np.zeros(2)
    div = np.zeros(fB.shape[1:]) if field else None
    lib().or_face_divb(C.byref(params(cfg)), fB, out, _ptr(div))
    return (out[0], out[1], div) if field else (out[0], out[1])


def face_to_cell(cfg: dict, fB, P):
    """P with the interior cells' B^i replaced by the face means / sqrt(-g)."""
    P = np.array(P, dtype=np.float64, order="C", copy=True)
    lib().or_face_to_cell(C.byref(params(cfg)), np.ascontiguousarray(fB, dtype=np.float64), P)
    return P


def face_emfs(cfg: dict, Pin):
    """Edge EMFs of face-centred CT from a ghost-filled state: (3, N3, N2, N1)."""
    Pin = np.ascontiguousarray(Pin, dtype=np.float64)
    E = np.zeros((3,) + Pin.shape[1:])
    lib().or_face_emfs(C.byref(params(cfg)), Pin, E)
    return E


def stage_face(cfg: dict, U0, Pin, cdt: float, E, fB0, fBout, Uout, Pout):
    """One face-CT stage with caller-supplied edge EMFs; fBout, Uout, Pout
    updated in place. Returns (ctop[3] arrays, stats)."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    Pin = np.ascontiguousarray(Pin, dtype=np.float64)
    ct = [np.zeros(Pin.shape[1:]) for _ in range(3)]
    st = (C.c_long * 4)()
    lib().or_stage_face(C.byref(params(cfg)), U0, Pin, float(cdt), np.ascontiguousarray(E, dtype=np.float64),
                        np.ascontiguousarray(fB0, dtype=np.float64), fBout, Uout, Pout, *[_ptr(c) for c in ct], st)
    _note(st)
    return ct, list(st)[:3]
