"""The CUDA library builds, loads and exports every entry point that
include/kharma_gb300.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "kharma_gb300.h")).read()
    return sorted(set(re.findall(r"\b(kh_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_calls():
    names = _declared()
    for must in ("kh_geometry_init", "kh_prim_to_cons", "kh_cons_to_prim", "kh_step", "kh_divb"):
        assert must in names


def test_library_exports_every_symbol():
    from paper_2408_01361_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    from paper_2408_01361_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.kh_strerror.restype = ctypes.c_char_p
    assert lib.kh_strerror(0) == b"success"
    assert lib.kh_strerror(-1) == b"invalid argument"


def test_argument_validation_without_gpu():
    """Unsupported combinations are refused before any device call: the
    flux-correction flag outside {0, 1}, the correction on a multi-block
    mesh, an unknown precision."""
    from paper_2408_01361_gb300 import inputs, kh
    cfg = inputs.linear_mode_cfg(8, ndim=3)

    c = kh.coords_from_cfg(cfg)
    c.fofc = 2
    h = ctypes.c_void_p()
    assert kh.lib().kh_geometry_init(0.0, ctypes.byref(c), float(cfg["gam"]), ctypes.byref(h)) == -1
    c = kh.coords_from_cfg(cfg)
    c.precision = 2
    assert kh.lib().kh_geometry_init(0.0, ctypes.byref(c), float(cfg["gam"]), ctypes.byref(h)) == -1
    blk = kh.Block(0, 0, 0, 0, 8, 8, 8)
    c = kh.coords_from_cfg(cfg)
    c.fofc = 2
    assert kh.lib().kh_mesh_init(0.0, ctypes.byref(c), float(cfg["gam"]), 1, ctypes.byref(blk),
                                 ctypes.byref(h)) == -1
    # the mesh takes the flux correction and the Runge-Kutta integrators with
    # Flux-CT (validation passes; the call then needs a device), not with face CT
    for over in (dict(fofc=True), dict(integrator="rk2"), dict(integrator="ssprk54", fofc=True)):
        c = kh.coords_from_cfg(dict(cfg, **over))
        rc = kh.lib().kh_mesh_init(0.0, ctypes.byref(c), float(cfg["gam"]), 1, ctypes.byref(blk), ctypes.byref(h))
        assert rc != -1, over
        if rc == 0:
            kh.lib().kh_mesh_destroy(h)
        c = kh.coords_from_cfg(dict(cfg, bfield="face", **over))
        assert kh.lib().kh_mesh_init(0.0, ctypes.byref(c), float(cfg["gam"]), 1, ctypes.byref(blk),
                                     ctypes.byref(h)) == -1, over


def test_face_ct_validation_without_gpu():
    """Face-centred CT is refused with the flux correction and with unknown
    scheme values (single grid and mesh)."""
    from paper_2408_01361_gb300 import inputs, kh
    cfg = dict(inputs.linear_mode_cfg(8, ndim=3), bfield="face")
    h = ctypes.c_void_p()
    for over in (dict(fofc=True),):
        c = kh.coords_from_cfg(dict(cfg, **over))
        assert kh.lib().kh_geometry_init(0.0, ctypes.byref(c), float(cfg["gam"]), ctypes.byref(h)) == -1
    for field, value in (("bfield", 2), ("emf", 2)):
        c = kh.coords_from_cfg(cfg)
        setattr(c, field, value)
        assert kh.lib().kh_geometry_init(0.0, ctypes.byref(c), float(cfg["gam"]), ctypes.byref(h)) == -1
    blk = kh.Block(0, 0, 0, 0, 8, 8, 8)
    c = kh.coords_from_cfg(cfg)
    c.emf = 5
    assert kh.lib().kh_mesh_init(0.0, ctypes.byref(c), float(cfg["gam"]), 1, ctypes.byref(blk),
                                 ctypes.byref(h)) == -1


def test_mixed_inversion_and_solver_validation_without_gpu():
    """mixed_inversion outside {df, fp64} and an unknown solver are refused by
    single grids and the refined mesh; the mesh accepts every solver and both
    mixed inversions (validation passes; the call then needs a device:
    KH_ECUDA here, KH_OK on a GPU)."""
    from paper_2408_01361_gb300 import inputs, kh
    cfg = dict(inputs.linear_mode_cfg(8, ndim=3), precision="mixed")
    h = ctypes.c_void_p()
    blk = kh.Block(0, 0, 0, 0, 8, 8, 8)
    for field, bad in (("mixed_inversion", 2), ("inverter", 3)):
        c = kh.coords_from_cfg(cfg)
        setattr(c, field, bad)
        assert kh.lib().kh_geometry_init(0.0, ctypes.byref(c), float(cfg["gam"]), ctypes.byref(h)) == -1
        assert kh.lib().kh_mesh_init(0.0, ctypes.byref(c), float(cfg["gam"]), 1, ctypes.byref(blk),
                                     ctypes.byref(h)) == -1
    for over in (dict(mixed_inversion="fp64"), dict(inverter="1dw"), dict(inverter="kastaun")):
        c = kh.coords_from_cfg(dict(cfg, **over))
        rc = kh.lib().kh_mesh_init(0.0, ctypes.byref(c), float(cfg["gam"]), 1, ctypes.byref(blk), ctypes.byref(h))
        assert rc != -1, over
        if rc == 0:
            kh.lib().kh_mesh_destroy(h)


def test_wait_limit_rejects_a_null_context_without_gpu():
    from paper_2408_01361_gb300 import kh
    assert kh.lib().kh_set_wait_limit(None, 0) == -1
