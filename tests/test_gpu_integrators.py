"""GPU parity of the Runge-Kutta integrators (RK1, RK2, SSPRK(5,4); FP64,
Flux-CT) with the oracle's on a periodic box and on the FMKS torus
(floors, failed inversions and their fixup included), their temporal orders
on a fixed grid, and graph replay equal to eager stepping; the same parity
with face-centred CT (the face field a stage state) and with the first-order
flux correction in every stage, FP64 and mixed."""
import os

import numpy as np
import pytest

from conftest import GOLDEN
from gpu_helpers import GpuRun, TOL, assert_fp64_parity, interior
from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu

INTEGRATORS = ["rk1", "rk2", "ssprk54"]


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


def _case(which):
    if which == "torus":
        cfg = inputs.torus_cfg(48, 32, 16, r_out=60.0)
        return cfg, inputs.torus_state(cfg, seed=2)
    cfg = inputs.linear_mode_cfg(12, ndim=3, recon="weno5")
    cfg["n1"], cfg["n3"] = 16, 10
    rng = np.random.default_rng(3)
    P = np.zeros(inputs.shape(cfg))
    P[0] = 1.0 + 0.1 * rng.random(P[0].shape)
    P[1] = 1.0 + 0.1 * rng.random(P[1].shape)
    P[2:5] = 0.1 * rng.normal(size=P[2:5].shape)
    P[5:] = 0.5 * rng.normal(size=P[5:].shape)
    return cfg, P


def _run(kh, orc, cfg, P, nsteps, graph=False, check_oracle=True):
    Uo = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    ctx = kh.Context(cfg)
    ctx.set_graph(graph)
    g = GpuRun(ctx, cfg, P, U=Uo)
    Uc, Pc, dto = Uo, P, None
    for _ in range(nsteps):
        if check_oracle:
            Uc, Pc, dto, st_o = orc.step(cfg, Uc, Pc, dt)
        dtg, nfail = ctx.step(g.U, g.P, g.B, dt)
        if check_oracle:
            assert nfail == st_o[0]
    Ug, Pg = g.host()
    return Ug, Pg, Uc, Pc, dtg, dto


@pytest.mark.parametrize("integ", INTEGRATORS)
@pytest.mark.parametrize("which", ["box", "torus"])
def test_integrator_step_parity(kh, orc, integ, which):
    cfg, P = _case(which)
    cfg = dict(cfg, integrator=integ)
    Ug, Pg, Uc, Pc, dtg, dto = _run(kh, orc, cfg, P, 3)
    assert_fp64_parity(interior(cfg, Ug), interior(cfg, Uc), "U")
    assert_fp64_parity(interior(cfg, Pg), interior(cfg, Pc), "P")
    assert abs(dtg - dto) <= 1e-10 * dto


def test_temporal_orders_gpu(kh):
    dP, om = inputs.load_eigvec(os.path.join(GOLDEN, "linear_fast_mode.txt"))
    cfg = inputs.linear_mode_cfg(32, ndim=2, recon="weno5")
    # amplitude 1e-2: the fourth-order errors stay well above FP64 rounding
    P = inputs.linear_mode_state(cfg, dP, om, amp=1e-2)
    T = 0.25 * 2 * np.pi / om

    def run(integ, nst):
        c = dict(cfg, integrator=integ)
        ctx = kh.Context(c)
        g = GpuRun(ctx, c, P)
        for _ in range(nst):
            ctx.step(g.U, g.P, g.B, T / nst, sync=False)
        return g.host()[1]

    sl = (slice(None),) + inputs.interior(cfg)
    ref = run("ssprk54", 512)
    n0 = 16
    for integ, p in (("rk1", 1.0), ("rk2", 2.0), ("vl2", 2.0), ("ssprk54", 4.0)):
        e = [np.abs(run(integ, n0 * m)[sl] - ref[sl]).mean() for m in (1, 2, 4)]
        for a, b in ((e[0], e[1]), (e[1], e[2])):
            assert abs(np.log2(a / b) - p) < 0.15, (integ, e)


def test_ssprk54_graph_replay_matches_eager(kh, orc):
    cfg, P = _case("torus")
    cfg = dict(cfg, integrator="ssprk54")
    a = _run(kh, orc, cfg, P, 2, graph=False, check_oracle=False)
    b = _run(kh, orc, cfg, P, 2, graph=True, check_oracle=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("integ", ["rk2", "ssprk54"])
def test_mixed_integrators_vs_oracle(kh, orc, integ):
    """The mixed path's Runge-Kutta stages (FP32 shadow between stages, FP64
    U and final P) against the oracle's FP64 integrator, at the mixed path's
    FP32 level (momenta and velocities against the mass scale near the
    torus's equilibrium, as for the predictor-corrector)."""
    cfg, P = _case("torus")
    cfg = dict(cfg, integrator=integ, precision="mixed")
    Uo = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    Uo2, Po2, _, _ = orc.step(cfg, Uo, P, dt)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P, U=Uo)
    ctx.step(g.U, g.P, g.B, dt)
    Ug, Pg = g.host()
    a, b = interior(cfg, Ug), interior(cfg, Uo2)
    pa, pb = interior(cfg, Pg), interior(cfg, Po2)
    mass = np.abs(b[0]).sum()
    nz = b[0].size
    for v in range(8):
        tol = 2e-3 if v in (2, 3, 4) else 1e-4
        den = max(np.abs(b[v]).sum(), 1e-3 * mass)
        assert np.abs(a[v] - b[v]).sum() / den < tol, ("U", v, np.abs(a[v] - b[v]).sum() / den)
        pden = max(np.abs(pb[v]).sum(), 1e-2 * nz if v in (2, 3, 4) else 0.0)
        assert np.abs(pa[v] - pb[v]).sum() / pden < tol, ("P", v, np.abs(pa[v] - pb[v]).sum() / pden)


# ---- the integrators with face-centred CT and with the flux correction ----

@pytest.mark.parametrize("integ", INTEGRATORS)
@pytest.mark.parametrize("which", ["box3d-gs05", "torus3d-gs05", "torus2d-average"])
def test_face_ct_integrator_parity(kh, orc, integ, which):
    from test_gpu_facect import _case as face_case, _faces_interior, _run as face_run
    cfg, P, fB = face_case(which)
    cfg = dict(cfg, integrator=integ)
    ctx, fBd, Ug, Pg, fg, Uc, Pc, fc, dtg, dto = face_run(kh, orc, cfg, P, fB, 2)
    assert_fp64_parity(interior(cfg, Ug), interior(cfg, Uc), "U")
    assert_fp64_parity(interior(cfg, Pg), interior(cfg, Pc), "P")
    for x, y in zip(_faces_interior(cfg, fg), _faces_interior(cfg, fc)):
        den = np.abs(y).sum()
        if den > 0:
            assert np.abs(x - y).sum() / den < TOL
    assert abs(dtg - dto) <= 1e-10 * dto
    mx, _ = ctx.face_divb(fBd)
    dx = min((cfg[k][1] - cfg[k][0]) / cfg[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3")))
    assert mx < 1e-12 * np.abs(fc).max() / dx


@pytest.mark.parametrize("integ", INTEGRATORS)
@pytest.mark.parametrize("which", ["box_some", "torus3d"])
def test_fofc_integrator_parity(kh, orc, integ, which):
    from test_gpu_fofc import _case as fofc_case, _run as fofc_run
    cfg, P, dirich = fofc_case(which)
    cfg = dict(cfg, integrator=integ)
    cfg, Ug, Pg, Uc, Pc, counts, dtg, dto = fofc_run(kh, orc, cfg, P, dirich, 2)
    for c in counts:
        assert c[0] == c[1] and c[0] > 0 and c[2] == c[3] and c[4] == c[5], counts
    assert_fp64_parity(interior(cfg, Ug), interior(cfg, Uc), "U")
    assert_fp64_parity(interior(cfg, Pg), interior(cfg, Pc), "P")
    assert abs(dtg - dto) <= 1e-10 * dto


def test_ssprk54_face_ct_graph_replay_matches_eager(kh, orc):
    from test_gpu_facect import _case as face_case, _run as face_run
    cfg, P, fB = face_case("torus3d-gs05")
    cfg = dict(cfg, integrator="ssprk54")
    a = face_run(kh, orc, cfg, P, fB, 2, graph=False)
    b = face_run(kh, orc, cfg, P, fB, 2, graph=True)
    for x, y in zip(a[2:5], b[2:5]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("opt", ["face", "fofc"])
def test_mixed_ssprk54_with_options_vs_oracle(kh, orc, opt):
    """The mixed path's SSPRK(5,4) with face CT / the flux correction against
    the oracle's FP64 step at the mixed path's FP32 flux level."""
    if opt == "face":
        from test_gpu_facect import _case as face_case
        cfg, P, fB = face_case("torus3d-gs05")
        dirich = None
    else:
        from test_gpu_fofc import _case as fofc_case
        cfg, P, dirich = fofc_case("torus3d")
        cfg, fB = dict(cfg, fofc=True), None
    cfg = dict(cfg, integrator="ssprk54")
    P = orc.apply_bc(cfg, P, dirich) if dirich is not None else orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    if fB is None:
        Uo, Po, _, _ = orc.step(cfg, U, P, dt)
    else:
        Uo, Po, fo, _, _ = orc.step_face(cfg, U, P, fB, dt)
    c = dict(cfg, precision="mixed")
    ctx = kh.Context(c)
    g = GpuRun(ctx, c, P, U=U)
    if fB is not None:
        fBd = ctx.to_device(fB)
        ctx.set_face_field(fBd)
    ctx.step(g.U, g.P, g.B, dt)
    Ug, Pg = g.host()
    a, b = interior(cfg, Ug), interior(cfg, Uo)
    pa, pb = interior(cfg, Pg), interior(cfg, Po)
    mass = np.abs(b[0]).sum()
    nz = b[0].size
    for v in range(8):
        tol = 2e-3 if v in (2, 3, 4) else 1e-4
        den = max(np.abs(b[v]).sum(), 1e-3 * mass)
        assert np.abs(a[v] - b[v]).sum() / den < tol, ("U", v, np.abs(a[v] - b[v]).sum() / den)
        pden = max(np.abs(pb[v]).sum(), 1e-2 * nz if v in (2, 3, 4) else 0.0)
        assert np.abs(pa[v] - pb[v]).sum() / pden < tol, ("P", v, np.abs(pa[v] - pb[v]).sum() / pden)
    if fB is not None:
        dx = min((cfg[k][1] - cfg[k][0]) / cfg[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3")))
        mx, _ = ctx.face_divb(fBd)
        assert mx < 1e-12 * np.abs(fB).max() / dx
