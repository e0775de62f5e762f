"""Steps of a set of small problems through whichever build of the library
kh.py loads (KH_LIBRARY), writing the final states and the bounds-check
count to an .npz file. Run as a script in a child process by
test_gpu_bounds_check.py, once with the bounds-checked build and once with
the release build; the cases cover the kernels the checks instrument (ghost
fills with periodic, outflow, polar and Dirichlet faces, the FP64 and FP32
face kernels including the TMA tiles on a ragged grid, Flux-CT, both update
kernels, the fixup list, the CFL reduction, the flux correction, face CT and
a Runge-Kutta integrator).

    python tests/bounds_cases.py OUT.npz"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from gpu_helpers import GpuRun  # noqa: E402
from paper_2408_01361_gb300 import inputs, kh  # noqa: E402


def cases():
    tor = inputs.torus_cfg(40, 24, 12, r_out=60.0)
    box = inputs.linear_mode_cfg(8, ndim=3)
    box.update(n1=37, n2=23, n3=11)
    bondi = inputs.bondi_cfg(32, 32)
    return [
        ("torus_fp64", tor, None),
        ("torus_mixed", dict(tor, precision="mixed"), None),
        ("torus_mixed_fofc", dict(tor, precision="mixed", fofc=True), None),
        ("box_mixed_ragged", dict(box, precision="mixed"), None),
        ("box_fp64_ssprk54", dict(box, integrator="ssprk54"), None),
        ("bondi_fp64", bondi, "bondi"),
        ("torus_fp64_face", dict(tor, bfield="face"), "face"),
    ]


def run(out_path):
    res = {}
    for name, cfg, kind in cases():
        dirich = None
        if kind == "bondi":
            P, dirich = inputs.bondi_state(cfg, seed=1)
        elif cfg["coords"] == "minkowski":
            P = inputs.random_prims(cfg, seed=3, rho_range=(0.5, 1.0), u_range=(0.3, 1.0),
                                    ut_scale=(0.3, 0.3, 0.3), b_scale=(0.3, 0.3, 0.3))
        else:
            P = inputs.torus_state(cfg, seed=2)
        ctx = kh.Context(cfg)
        g = GpuRun(ctx, cfg, P, dirichlet=dirich)
        if kind == "face":
            fB = ctx.to_device(inputs.torus_face_field(cfg))
            ctx.set_face_field(fB)
            ctx.face_to_cell(fB, g.B)
            ctx.prim_to_cons(g.P, g.B, g.U)
        dt = 0.5 * ctx.cfl_dt(g.P, g.B)
        for _ in range(2):
            dt, _ = ctx.step(g.U, g.P, g.B, dt)
        U, PB = g.host()
        res[name + "_U"], res[name + "_P"] = U, PB
        res[name + "_nbounds"] = np.array(ctx.stats().nbounds)
        ctx.close()
    np.savez(out_path, **res)


if __name__ == "__main__":
    run(sys.argv[1])
