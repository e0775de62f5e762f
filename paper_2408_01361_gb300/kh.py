"""Thin Python binding of the C ABI in include/kharma_gb300.h.

Argument marshalling only: every step of the method runs in the CUDA library
(libkharma_gb300.so, built in place by ``build.py``). PyTorch supplies device
memory and the stream. There is no CPU fallback: if the library or a GPU is
missing, the calls raise.

Arrays handed to the library are torch float64 CUDA tensors in the library
layout [var][n3s][n2s][n1s] (see ``Context.shape``); ``to_device`` /
``to_host`` convert from/to the unpadded (8, N3, N2, N1) numpy layout used by
the input generators (slots rho, u, u~1..3, B1..3).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# KH_LIBRARY selects another in-tree build of the library (the bounds-checked
# variant libkharma_gb300_bounds.so that build.build(bounds=True) makes)
_LIB = os.environ.get("KH_LIBRARY") or os.path.join(_HERE, "libkharma_gb300.so")

MINKOWSKI, KS, MKS, FMKS = 0, 1, 2, 3
KIND = {"minkowski": MINKOWSKI, "ks": KS, "mks": MKS, "fmks": FMKS}
BC = {"periodic": 0, "outflow": 1, "polar": 2, "dirichlet": 3}
RECON = {"mc": 0, "weno5": 1}
PRECISION = {"fp64": 0, "mixed": 1}
BFIELD = {"fluxct": 0, "face": 1}
EMF = {"average": 0, "gs05": 1}
INVERTER = {"noble2d": 0, "1dw": 1, "kastaun": 2}
INTEGRATOR = {"vl2": 0, "rk1": 1, "rk2": 2, "ssprk54": 3}
MIXED_INVERSION = {"df": 0, "fp64": 1}
WAIT_POLLS = 1 << 22  # KH_WAIT_POLLS
ERRORS = {0: "KH_OK", -1: "KH_EINVAL", -2: "KH_ECUDA", -3: "KH_ENOMEM", -4: "KH_ETIMEOUT", -5: "KH_ENAN"}


class KHError(RuntimeError):
    pass


class Coords(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("recon", C.c_int),
        ("precision", C.c_int), ("bc", C.c_int * 6),
        ("x1min", C.c_double), ("x1max", C.c_double), ("x2min", C.c_double), ("x2max", C.c_double),
        ("x3min", C.c_double), ("x3max", C.c_double),
        ("hslope", C.c_double), ("poly_xt", C.c_double), ("poly_alpha", C.c_double), ("mks_smooth", C.c_double),
        ("cfl", C.c_double), ("rho_min", C.c_double), ("u_min", C.c_double), ("bsq_rho_max", C.c_double),
        ("bsq_u_max", C.c_double), ("u_rho_max", C.c_double), ("gamma_max", C.c_double),
        ("newton_max_iter", C.c_int), ("newton_tol", C.c_double), ("fofc", C.c_int),
        ("bfield", C.c_int), ("emf", C.c_int), ("inverter", C.c_int), ("integrator", C.c_int),
        ("mixed_inversion", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [("nfail", C.c_int64), ("nfloor", C.c_int64), ("nunfixed", C.c_int64), ("dt_cfl", C.c_double),
                ("nfp64", C.c_int64), ("nfofc", C.c_int64), ("nbounds", C.c_int64)]


class Block(C.Structure):
    _fields_ = [("level", C.c_int), ("i0", C.c_int), ("j0", C.c_int), ("k0", C.c_int),
                ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int)]


_lib = None


def lib():
    """Load libkharma_gb300.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise KHError(f"CUDA library not built: {_LIB} (run __graft_entry__.build())")
        L = C.CDLL(_LIB)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.kh_geometry_init.argtypes = [C.c_double, C.POINTER(Coords), C.c_double, C.POINTER(C.c_void_p)]
        L.kh_shape.argtypes = [vp, ip, ip, ip, ip]
        L.kh_set_stream.argtypes = [vp, vp]
        L.kh_set_dirichlet.argtypes = [vp, C.c_int, vp]
        L.kh_prim_to_cons.argtypes = [vp, vp, vp, vp]
        L.kh_cons_to_prim.argtypes = [vp, vp, vp, vp, vp, C.POINTER(C.c_int64)]
        L.kh_step.argtypes = [vp, vp, vp, vp, C.c_double, dp]
        L.kh_cfl_dt.argtypes = [vp, vp, vp, dp]
        L.kh_divb.argtypes = [vp, vp, dp, dp]
        L.kh_set_face_field.argtypes = [vp, vp]
        L.kh_pack_state.argtypes = [vp, vp, vp, vp, vp]
        L.kh_unpack_state.argtypes = [vp, vp, vp, vp, vp]
        L.kh_face_to_cell.argtypes = [vp, vp, vp]
        L.kh_face_divb.argtypes = [vp, vp, dp, dp]
        L.kh_fluxes.argtypes = [vp, vp, vp, vp, vp, vp]
        L.kh_fill_ghosts.argtypes = [vp, vp, vp]
        L.kh_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.kh_profile.argtypes = [vp, C.c_int]
        L.kh_set_graph.argtypes = [vp, C.c_int]
        L.kh_set_launch.argtypes = [vp, C.c_int, C.c_int]
        L.kh_get_launch.argtypes = [vp, ip, ip]
        L.kh_autotune.argtypes = [vp, vp, vp, vp, C.c_double, ip, ip]
        L.kh_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.kh_set_wait_limit.argtypes = [vp, C.c_uint]
        L.kh_launch_count.argtypes = [vp]
        L.kh_launch_count.restype = C.c_int64
        L.kh_destroy.argtypes = [vp]
        L.kh_strerror.argtypes = [C.c_int]
        L.kh_strerror.restype = C.c_char_p
        L.kh_step_adjoint.argtypes = [vp, vp, vp, vp, C.c_double, vp, vp, vp, vp, vp, vp, vp, dp]
        L.kh_prim_to_cons_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, dp]
        L.kh_get_stage_flux.argtypes = [vp, C.c_int, vp]
        L.kh_mesh_init.argtypes = [C.c_double, C.POINTER(Coords), C.c_double, C.c_int, C.POINTER(Block),
                                   C.POINTER(C.c_void_p)]
        L.kh_mesh_block_shape.argtypes = [vp, C.c_int, ip, ip, ip, C.POINTER(C.c_int64)]
        for f in ("kh_mesh_cells", "kh_mesh_zones", "kh_mesh_ghost_cells", "kh_mesh_launch_count"):
            getattr(L, f).argtypes = [vp]
            getattr(L, f).restype = C.c_int64
        L.kh_mesh_set_stream.argtypes = [vp, vp]
        L.kh_mesh_prim_to_cons.argtypes = [vp, vp, vp, vp]
        L.kh_mesh_fill_ghosts.argtypes = [vp, vp, vp]
        L.kh_mesh_cfl_dt.argtypes = [vp, vp, vp, dp]
        L.kh_mesh_step.argtypes = [vp, vp, vp, vp, C.c_double, dp]
        L.kh_mesh_set_graph.argtypes = [vp, C.c_int]
        L.kh_mesh_set_staged_update.argtypes = [vp, C.c_int]
        L.kh_mesh_divb.argtypes = [vp, vp, dp, dp]
        L.kh_mesh_set_launch.argtypes = [vp, C.c_int, C.c_int]
        L.kh_mesh_get_launch.argtypes = [vp, ip, ip]
        L.kh_mesh_autotune.argtypes = [vp, vp, vp, vp, C.c_double, ip, ip]
        L.kh_mesh_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.kh_mesh_set_face_field.argtypes = [vp, vp]
        L.kh_mesh_destroy.argtypes = [vp]
        _lib = L
    return _lib


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise KHError(f"{what}: {ERRORS.get(rc, rc)} ({lib().kh_strerror(rc).decode()})")
    return rc


def coords_from_cfg(cfg: dict) -> Coords:
    c = Coords()
    c.kind = KIND[cfg["coords"]]
    c.n1, c.n2, c.n3 = cfg["n1"], cfg["n2"], cfg["n3"]
    c.recon = RECON[cfg["recon"]]
    c.precision = PRECISION[cfg.get("precision", "fp64")]
    for q, b in enumerate(cfg["bc"]):
        c.bc[q] = BC[b]
    (c.x1min, c.x1max), (c.x2min, c.x2max), (c.x3min, c.x3max) = cfg["x1"], cfg["x2"], cfg["x3"]
    c.hslope = cfg.get("hslope", 0.3)
    c.poly_xt = cfg.get("poly_xt", 0.82)
    c.poly_alpha = cfg.get("poly_alpha", 14.0)
    c.mks_smooth = cfg.get("mks_smooth", 0.5)
    c.cfl = cfg.get("cfl", 0.9)
    fl = cfg.get("floors", {})
    c.rho_min = fl.get("rho_min", 1e-20)
    c.u_min = fl.get("u_min", 1e-20)
    c.bsq_rho_max = fl.get("bsq_rho_max", 1e300)
    c.bsq_u_max = fl.get("bsq_u_max", 1e300)
    c.u_rho_max = fl.get("u_rho_max", 1e300)
    c.gamma_max = fl.get("gamma_max", 1e300)
    c.newton_max_iter = cfg.get("newton_max_iter", 30)
    c.newton_tol = cfg.get("newton_tol", 1e-14)
    c.fofc = 1 if cfg.get("fofc") else 0
    c.bfield = BFIELD[cfg.get("bfield", "fluxct")]
    c.emf = EMF[cfg.get("emf", "gs05")]
    c.inverter = INVERTER[cfg.get("inverter", "noble2d")]
    c.integrator = INTEGRATOR[cfg.get("integrator", "vl2")]
    c.mixed_inversion = MIXED_INVERSION[cfg.get("mixed_inversion", "df")]
    return c


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(0 if t is None else t.data_ptr())


class Context:
    """One kh_ctx: geometry cache + scratch for one problem on the current GPU."""

    def __init__(self, cfg: dict, device=None):
        import torch

        if not torch.cuda.is_available():
            raise KHError("no CUDA device: the GB300 path has no CPU fallback")
        self.torch = torch
        self.device = torch.device(device or "cuda:0")
        torch.cuda.set_device(self.device)
        self.cfg = cfg
        self._c = coords_from_cfg(cfg)
        h = C.c_void_p()
        _check(lib().kh_geometry_init(float(cfg.get("a", 0.0)), C.byref(self._c), float(cfg["gam"]), C.byref(h)),
               "kh_geometry_init")
        self._h = h
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(lib().kh_shape(h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "kh_shape")
        self.n1s, self.n2s, self.n3s, self.ng = a.value, b.value, c.value, d.value
        self.stream = None

    # ---- lifetime ----
    def close(self):
        if getattr(self, "_h", None):
            lib().kh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        _check(lib().kh_set_stream(self._h, C.c_void_p(stream.cuda_stream if stream is not None else 0)),
               "kh_set_stream")

    # ---- layout helpers ----
    def shape(self, nvar: int):
        return (nvar, self.n3s, self.n2s, self.n1s)

    def empty(self, nvar: int):
        return self.torch.zeros(self.shape(nvar), dtype=self.torch.float64, device=self.device)

    def to_device(self, A: np.ndarray, pinned_src=None):
        """(nvar, N3, N2, N1) numpy -> padded device tensor."""
        t = self.empty(A.shape[0])
        src = self.torch.from_numpy(np.ascontiguousarray(A))
        t[:, :, :, : A.shape[3]].copy_(src)
        return t

    def to_host(self, t, N1: int) -> np.ndarray:
        return t[:, :, :, :N1].cpu().numpy()

    def split(self, PB):
        """Device (8, ...) tensor -> (P view of 5 slots, B view of 3 slots), both contiguous."""
        return PB[:5], PB[5:]

    # ---- the C ABI ----
    def set_dirichlet(self, face: int, PB_ghost):
        _check(lib().kh_set_dirichlet(self._h, face, _ptr(PB_ghost)), "kh_set_dirichlet")

    def prim_to_cons(self, P, B, U):
        _check(lib().kh_prim_to_cons(self._h, _ptr(P), _ptr(B), _ptr(U)), "kh_prim_to_cons")

    def cons_to_prim(self, U, P, B, pflag=None) -> int:
        n = C.c_int64()
        _check(lib().kh_cons_to_prim(self._h, _ptr(U), _ptr(P), _ptr(B), _ptr(pflag), C.byref(n)),
               "kh_cons_to_prim")
        return n.value

    def step(self, U, P, B, dt: float, sync: bool = True):
        """One step; returns (dt_cfl, nfail) when sync, else (None, None)."""
        if sync:
            d = C.c_double()
            rc = _check(lib().kh_step(self._h, _ptr(U), _ptr(P), _ptr(B), float(dt), C.byref(d)), "kh_step")
            return d.value, rc
        _check(lib().kh_step(self._h, _ptr(U), _ptr(P), _ptr(B), float(dt), None), "kh_step")
        return None, None

    def cfl_dt(self, P, B) -> float:
        d = C.c_double()
        _check(lib().kh_cfl_dt(self._h, _ptr(P), _ptr(B), C.byref(d)), "kh_cfl_dt")
        return d.value

    def divb(self, B):
        mx, l1 = C.c_double(), C.c_double()
        _check(lib().kh_divb(self._h, _ptr(B), C.byref(mx), C.byref(l1)), "kh_divb")
        return mx.value, l1.value

    # ---- compact interior state ----
    def pack_state(self, U, P, B, out):
        """out (16 x interior zones; device, or pinned host memory written over
        the host link): U's 8 slots, then P's 5 and B's 3."""
        _check(lib().kh_pack_state(self._h, _ptr(U), _ptr(P), _ptr(B), _ptr(out)), "kh_pack_state")

    def unpack_state(self, inp, U, P, B):
        _check(lib().kh_unpack_state(self._h, _ptr(inp), _ptr(U), _ptr(P), _ptr(B)), "kh_unpack_state")

    # ---- face-centred constrained transport ----
    def set_face_field(self, fB):
        """Register the face field (3 planes, kept by the caller) that kh_step
        advances (bfield "face")."""
        self._fB = fB
        _check(lib().kh_set_face_field(self._h, _ptr(fB)), "kh_set_face_field")

    def face_to_cell(self, fB, B):
        _check(lib().kh_face_to_cell(self._h, _ptr(fB), _ptr(B)), "kh_face_to_cell")

    def face_divb(self, fB):
        mx, l1 = C.c_double(), C.c_double()
        _check(lib().kh_face_divb(self._h, _ptr(fB), C.byref(mx), C.byref(l1)), "kh_face_divb")
        return mx.value, l1.value

    def fluxes(self, P, B, F1, F2, F3=None):
        _check(lib().kh_fluxes(self._h, _ptr(P), _ptr(B), _ptr(F1), _ptr(F2), _ptr(F3)), "kh_fluxes")

    def fill_ghosts(self, P, B):
        _check(lib().kh_fill_ghosts(self._h, _ptr(P), _ptr(B)), "kh_fill_ghosts")

    def stats(self) -> Stats:
        s = Stats()
        _check(lib().kh_get_stats(self._h, C.byref(s)), "kh_get_stats")
        return s

    def set_graph(self, enable: bool):
        _check(lib().kh_set_graph(self._h, 1 if enable else 0), "kh_set_graph")

    def set_wait_limit(self, polls: int = WAIT_POLLS):
        """Polls of a mixed face CTA's wait for its TMA tile (kh_set_wait_limit)."""
        _check(lib().kh_set_wait_limit(self._h, C.c_uint(int(polls))), "kh_set_wait_limit")

    def step_rc(self, U, P, B, dt: float):
        """kh_step with a dt_cfl pointer; returns the raw return code (no raise)."""
        d = C.c_double()
        return lib().kh_step(self._h, _ptr(U), _ptr(P), _ptr(B), float(dt), C.byref(d))

    def set_launch(self, tpb_flux: int, tpb_update: int):
        _check(lib().kh_set_launch(self._h, int(tpb_flux), int(tpb_update)), "kh_set_launch")

    def get_launch(self):
        a, b = C.c_int(), C.c_int()
        _check(lib().kh_get_launch(self._h, C.byref(a), C.byref(b)), "kh_get_launch")
        return a.value, b.value

    def autotune(self, U, P, B, dt: float):
        a, b = C.c_int(), C.c_int()
        _check(lib().kh_autotune(self._h, _ptr(U), _ptr(P), _ptr(B), float(dt), C.byref(a), C.byref(b)),
               "kh_autotune")
        return a.value, b.value

    def step_adjoint(self, U, P, B, dt: float, gU=None, gP=None, gB=None, gF1=None):
        """Gradient through one step (kh_step_adjoint) at the checkpoint
        (U, P, B): returns (gU_in, gP_in, gB_in, g_gamma) as new tensors."""
        gU_in, gP_in, gB_in = self.empty(8), self.empty(5), self.empty(3)
        gg = C.c_double()
        _check(lib().kh_step_adjoint(self._h, _ptr(U), _ptr(P), _ptr(B), float(dt), _ptr(gU), _ptr(gP), _ptr(gB),
                                     _ptr(gF1), _ptr(gU_in), _ptr(gP_in), _ptr(gB_in), C.byref(gg)),
               "kh_step_adjoint")
        return gU_in, gP_in, gB_in, gg.value

    def prim_to_cons_adjoint(self, P, B, gU):
        """(dU/dP)^T gU at interior cells: returns (gP, gB, g_gamma)."""
        gP, gB = self.empty(5), self.empty(3)
        gg = C.c_double()
        _check(lib().kh_prim_to_cons_adjoint(self._h, _ptr(P), _ptr(B), _ptr(gU), _ptr(gP), _ptr(gB), C.byref(gg)),
               "kh_prim_to_cons_adjoint")
        return gP, gB, gg.value

    def stage_flux(self, d: int = 1):
        """Fluxes through the lower x^d faces from the last stage run (8 planes)."""
        F = self.empty(8)
        _check(lib().kh_get_stage_flux(self._h, int(d), _ptr(F)), "kh_get_stage_flux")
        return F

    TIMERS = ("bc", "flux_x1", "flux_x2", "flux_x3", "flux_ct", "update", "fixup", "cfl", "fofc")

    def profile(self, enable: bool):
        _check(lib().kh_profile(self._h, 1 if enable else 0), "kh_profile")

    def profile_read(self) -> dict:
        ms = (C.c_double * len(self.TIMERS))()
        n = (C.c_int64 * len(self.TIMERS))()
        _check(lib().kh_profile_read(self._h, ms, n), "kh_profile_read")
        return {name: (ms[q], n[q]) for q, name in enumerate(self.TIMERS)}

    def launches(self) -> int:
        return int(lib().kh_launch_count(self._h))


def divb_noalloc(B, gdet, n1: int, n2: int, n3: int, n1s: int, n2s: int, dx, out, stream=None) -> int:
    """kh_divb_noalloc: corner divB without a context and without any
    allocation (for callers that cannot call cudaMalloc); B, gdet, out are
    device tensors, out receives (max |divB|, mean |divB|) asynchronously."""
    L = lib()
    f = L.kh_divb_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                  C.c_double, C.c_void_p, C.c_void_p]
    rc = f(_ptr(B), _ptr(gdet), n1, n2, n3, n1s, n2s, float(dx[0]), float(dx[1]), float(dx[2]), _ptr(out),
           C.c_void_p(stream.cuda_stream if stream is not None else 0))
    return _check(rc, "kh_divb_noalloc")


class Mesh:
    """One kh_mesh: statically refined blocks stepped together.

    ``blocks`` is a list of dicts {level, i0, j0, k0, n1, n2, n3} (first
    interior cell and interior size in level-``level`` indices; level l is
    2^l times finer than the base grid of ``cfg``). State lives in three flat
    arenas (U: 8 slots, P: 5, B: 3 per cell of every block); ``views`` gives
    each block's (nvar, n3s, n2s, n1s) window into an arena.
    """

    def __init__(self, cfg: dict, blocks: list, device=None):
        import torch

        if not torch.cuda.is_available():
            raise KHError("no CUDA device: the GB300 path has no CPU fallback")
        self.torch = torch
        self.device = torch.device(device or "cuda:0")
        torch.cuda.set_device(self.device)
        self.cfg = cfg
        self.blocks = blocks
        self._c = coords_from_cfg(cfg)
        arr = (Block * len(blocks))()
        for q, b in enumerate(blocks):
            arr[q] = Block(b["level"], b["i0"], b["j0"], b.get("k0", 0), b["n1"], b["n2"], b.get("n3", 1))
        h = C.c_void_p()
        _check(lib().kh_mesh_init(float(cfg.get("a", 0.0)), C.byref(self._c), float(cfg["gam"]), len(blocks), arr,
                                  C.byref(h)), "kh_mesh_init")
        self._h = h
        self.shapes, self.offsets = [], []
        for q in range(len(blocks)):
            a, b, c, o = C.c_int(), C.c_int(), C.c_int(), C.c_int64()
            _check(lib().kh_mesh_block_shape(h, q, C.byref(a), C.byref(b), C.byref(c), C.byref(o)),
                   "kh_mesh_block_shape")
            self.shapes.append((c.value, b.value, a.value))
            self.offsets.append(o.value)
        self.cells = int(lib().kh_mesh_cells(h))
        self.zones = int(lib().kh_mesh_zones(h))
        self.ghost_cells = int(lib().kh_mesh_ghost_cells(h))

    def close(self):
        if getattr(self, "_h", None):
            lib().kh_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(lib().kh_mesh_set_stream(self._h, C.c_void_p(stream.cuda_stream if stream is not None else 0)),
               "kh_mesh_set_stream")

    # ---- arenas ----
    def empty(self, nvar: int):
        return self.torch.zeros(nvar * self.cells, dtype=self.torch.float64, device=self.device)

    def views(self, arena, nvar: int):
        out = []
        for (n3s, n2s, n1s), off in zip(self.shapes, self.offsets):
            pl = n3s * n2s * n1s
            out.append(arena[nvar * off: nvar * off + nvar * pl].view(nvar, n3s, n2s, n1s))
        return out

    def to_device(self, PBs):
        """List of per-block (8, N3, N2, N1) numpy arrays -> (P arena, B arena)."""
        P, B = self.empty(5), self.empty(3)
        for A, vp, vb in zip(PBs, self.views(P, 5), self.views(B, 3)):
            src = self.torch.from_numpy(np.ascontiguousarray(A))
            vp[:, :, :, : A.shape[3]].copy_(src[:5])
            vb[:, :, :, : A.shape[3]].copy_(src[5:])
        return P, B

    def to_host(self, P, B):
        """(P, B) arenas -> list of per-block (8, N3, N2, N1) numpy arrays."""
        out = []
        for blk, vp, vb in zip(self.blocks, self.views(P, 5), self.views(B, 3)):
            N1 = blk["n1"] + 2 * 3
            out.append(np.concatenate([vp[:, :, :, :N1].cpu().numpy(), vb[:, :, :, :N1].cpu().numpy()]))
        return out

    def cons_to_device(self, Us):
        """List of per-block (8, N3, N2, N1) numpy conserved arrays -> U arena."""
        U = self.empty(8)
        for A, vu in zip(Us, self.views(U, 8)):
            vu[:, :, :, : A.shape[3]].copy_(self.torch.from_numpy(np.ascontiguousarray(A)))
        return U

    def cons_to_host(self, U):
        out = []
        for blk, vu in zip(self.blocks, self.views(U, 8)):
            out.append(vu[:, :, :, : blk["n1"] + 2 * 3].cpu().numpy())
        return out

    # ---- the C ABI ----
    def prim_to_cons(self, P, B, U):
        _check(lib().kh_mesh_prim_to_cons(self._h, _ptr(P), _ptr(B), _ptr(U)), "kh_mesh_prim_to_cons")

    def fill_ghosts(self, P, B):
        _check(lib().kh_mesh_fill_ghosts(self._h, _ptr(P), _ptr(B)), "kh_mesh_fill_ghosts")

    def cfl_dt(self, P, B) -> float:
        d = C.c_double()
        _check(lib().kh_mesh_cfl_dt(self._h, _ptr(P), _ptr(B), C.byref(d)), "kh_mesh_cfl_dt")
        return d.value

    def step(self, U, P, B, dt: float, sync: bool = True):
        if sync:
            d = C.c_double()
            rc = _check(lib().kh_mesh_step(self._h, _ptr(U), _ptr(P), _ptr(B), float(dt), C.byref(d)),
                        "kh_mesh_step")
            return d.value, rc
        _check(lib().kh_mesh_step(self._h, _ptr(U), _ptr(P), _ptr(B), float(dt), None), "kh_mesh_step")
        return None, None

    def divb(self, B):
        mx, l1 = C.c_double(), C.c_double()
        _check(lib().kh_mesh_divb(self._h, _ptr(B), C.byref(mx), C.byref(l1)), "kh_mesh_divb")
        return mx.value, l1.value

    def set_face_field(self, fB):
        """Register the face-field arena (3 planes per block; bfield "face")."""
        self._fB = fB
        _check(lib().kh_mesh_set_face_field(self._h, _ptr(fB)), "kh_mesh_set_face_field")

    def faces_to_device(self, fBs):
        """List of per-block (3, N3, N2, N1) numpy face fields -> face arena."""
        A = self.empty(3)
        for f, v in zip(fBs, self.views(A, 3)):
            v[:, :, :, : f.shape[3]].copy_(self.torch.from_numpy(np.ascontiguousarray(f)))
        return A

    def faces_to_host(self, A):
        out = []
        for blk, v in zip(self.blocks, self.views(A, 3)):
            N1 = blk["n1"] + 2 * 3
            out.append(v[:, :, :, :N1].cpu().numpy())
        return out

    def set_launch(self, tpb_flux: int, tpb_update: int):
        _check(lib().kh_mesh_set_launch(self._h, int(tpb_flux), int(tpb_update)), "kh_mesh_set_launch")

    def get_launch(self):
        a, b = C.c_int(), C.c_int()
        _check(lib().kh_mesh_get_launch(self._h, C.byref(a), C.byref(b)), "kh_mesh_get_launch")
        return a.value, b.value

    def autotune(self, U, P, B, dt: float):
        a, b = C.c_int(), C.c_int()
        _check(lib().kh_mesh_autotune(self._h, _ptr(U), _ptr(P), _ptr(B), float(dt), C.byref(a), C.byref(b)),
               "kh_mesh_autotune")
        return a.value, b.value

    def set_graph(self, enable: bool):
        _check(lib().kh_mesh_set_graph(self._h, 1 if enable else 0), "kh_mesh_set_graph")

    def set_staged_update(self, enable: bool) -> bool:
        """Select the TMA-staged mixed update (kh_mesh_set_staged_update);
        True if it is selected and the mesh qualifies."""
        return _check(lib().kh_mesh_set_staged_update(self._h, 1 if enable else 0), "kh_mesh_set_staged_update") == 1

    def stats(self) -> Stats:
        s = Stats()
        _check(lib().kh_mesh_get_stats(self._h, C.byref(s)), "kh_mesh_get_stats")
        return s

    def launches(self) -> int:
        return int(lib().kh_mesh_launch_count(self._h))
