"""The workload torus (FM torus a = 0.9375, FMKS 192x96x96, WENO5, loop field
at beta = 100) run for 1000 mixed-precision steps (and 100 FP64 steps) on the
GPU: the state stays finite, the CFL step does not collapse, failed
inversions stay a small fraction of the zones, the corner divergence of the
field stays at the FP32 (mixed) / FP64 rounding level of its scale, and the
mass changes only by what the open boundaries let through. The refined
torus (3 static levels, 592 blocks) runs its 200 autotuned mixed steps as a
graph, with the cell-centred and the face-centred field, under the same
bounds on the state, the step and the failures."""
import numpy as np
import pytest

from gpu_helpers import GpuRun, interior
from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


@pytest.mark.parametrize("precision,nsteps,divbar", [("mixed", 1000, 1e-5), ("fp64", 100, 1e-11)])
def test_workload_torus_long_run(kh, orc, precision, nsteps, divbar):
    cfg = dict(inputs.torus_cfg(192, 96, 96), precision=precision)
    P = inputs.torus_state(cfg, seed=2)
    P = orc.apply_bc(cfg, P)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P)
    U0, _ = g.host()
    mass0 = interior(cfg, U0)[0].sum()
    gd = orc.geometry(cfg, 0)[2]
    dx2 = (cfg["x2"][1] - cfg["x2"][0]) / cfg["n2"]
    bscale = np.abs(gd[None, None] * P[5:8]).max() / dx2
    dt0 = ctx.cfl_dt(g.P, g.B)
    dt = 0.5 * dt0
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
    worst_fail = 0
    for s in range(nsteps):
        dtn, nfail = ctx.step(g.U, g.P, g.B, dt)
        worst_fail = max(worst_fail, nfail)
        assert np.isfinite(dtn) and dtn > 0.2 * dt0, (s, dtn, dt0)
        dt = 0.5 * dtn
    Ug, Pg = g.host()
    assert np.isfinite(Ug).all() and np.isfinite(Pg).all()
    assert worst_fail < 1e-3 * nz, worst_fail
    mx, _ = ctx.divb(g.B)
    assert mx < divbar * bscale, (mx, bscale)
    mass1 = interior(cfg, Ug)[0].sum()
    assert abs(mass1 - mass0) < 0.05 * abs(mass0), (mass0, mass1)


@pytest.mark.parametrize("face", [False, True])
def test_refined_torus_long_run(kh, face):
    base, blocks = inputs.smr_torus_layout()
    if face:
        base = dict(base, bfield="face", emf="gs05")
    norms = inputs.torus_norms(base)
    cfgs = [inputs.block_cfg(base, b) for b in blocks]
    Ps = [inputs.torus_state(c, seed=2, norms=norms) for c in cfgs]
    m = kh.Mesh(dict(base, precision="mixed"), blocks)
    if face:
        fs = [inputs.torus_face_field(c, norms=norms) for c in cfgs]
        Ps = [inputs.cell_field_from_faces(c, f, P) for c, f, P in zip(cfgs, fs, Ps)]
        m.set_face_field(m.faces_to_device(fs))
        del fs
    P, B = m.to_device(Ps)
    del Ps
    U = m.empty(8)
    m.prim_to_cons(P, B, U)

    def mass():
        tot = 0.0
        for c, Ub in zip(cfgs, m.cons_to_host(U)):
            dv = np.prod([(c[x][1] - c[x][0]) / c[n] for x, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3"))])
            tot += interior(c, Ub)[0].sum() * dv
        return tot

    mass0 = mass()
    dt0 = m.cfl_dt(P, B)
    m.autotune(U, P, B, 0.5 * dt0)
    m.set_graph(True)
    dt = 0.5 * dt0
    worst_fail = 0
    for s in range(200):
        dtn, nfail = m.step(U, P, B, dt)
        worst_fail = max(worst_fail, nfail)
        assert np.isfinite(dtn) and dtn > 0.2 * dt0, (s, dtn, dt0)
        dt = 0.5 * dtn
    assert worst_fail < 1e-3 * m.zones, worst_fail
    for A in m.to_host(P, B):
        assert np.isfinite(A).all()
    mass1 = mass()
    assert abs(mass1 - mass0) < 0.05 * abs(mass0), (mass0, mass1)
    m.close()
