"""The Minkowski test problems the paper cites, on the GPU path: the
Orszag-Tang vortex and Komissarov's cylindrical explosion step to the
oracle's result (FP64, 1e-10), keep the symmetries of their initial states
over a longer run at 256^2 (FP64 to rounding; the mixed path to its FP32
level), and the periodic vortex conserves its totals."""
import numpy as np
import pytest

from gpu_helpers import ELEM_TOL, TOL, GpuRun, elem_err, interior, rel_l1
from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


def _problem(which, n, precision="fp64", recon="mc"):
    if which == "ot":
        cfg = dict(inputs.orszag_tang_cfg(n, recon=recon), precision=precision)
        return cfg, inputs.orszag_tang_state(cfg)
    cfg = dict(inputs.explosion_cfg(n, recon=recon), precision=precision)
    return cfg, inputs.explosion_state(cfg)


@pytest.mark.parametrize("recon", ["mc", "weno5"])
@pytest.mark.parametrize("which", ["ot", "explosion"])
def test_workload_parity(kh, orc, which, recon):
    cfg, P = _problem(which, 64, recon=recon)
    P = orc.apply_bc(cfg, P)
    Uo = orc.prim_to_cons(cfg, P)
    dt = orc.cfl_dt(cfg, P)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P, U=Uo)
    Uc, Pc = Uo, P
    for _ in range(5):
        Uc, Pc, _, st = orc.step(cfg, Uc, Pc, dt)
        _, nfail = ctx.step(g.U, g.P, g.B, dt)
        assert nfail == st[0] == 0
    Ug, Pg = g.host()
    eu = rel_l1(interior(cfg, Ug), interior(cfg, Uc))
    ep = rel_l1(interior(cfg, Pg), interior(cfg, Pc))
    xu = elem_err(interior(cfg, Ug), interior(cfg, Uc))
    xp = elem_err(interior(cfg, Pg), interior(cfg, Pc))
    for v in range(8):
        if np.abs(interior(cfg, Pc)[v]).max() > 1e-10:
            assert eu[v] < TOL and ep[v] < TOL, (v, eu, ep)
            assert xu[v] < ELEM_TOL and xp[v] < ELEM_TOL, (v, xu, xp)


def _run_to(kh, cfg, P, t_end):
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P)
    t = 0.0
    dt = ctx.cfl_dt(g.P, g.B)
    while t < t_end * (1 - 1e-14):
        h = min(dt, t_end - t)
        dt, _ = ctx.step(g.U, g.P, g.B, h)
        t += h
    return g.host()


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-9), ("mixed", 1e-3)])
def test_orszag_tang_half_turn(kh, orc, precision, bar):
    cfg, P = _problem("ot", 256, precision)
    P = orc.apply_bc(cfg, P)
    U0 = orc.prim_to_cons(cfg, P)
    U, Pg = _run_to(kh, cfg, P, 1.0)
    A = interior(cfg, Pg)
    assert np.isfinite(A).all()
    R = A[:, :, ::-1, ::-1]
    for v in range(8):
        sgn = 1.0 if v < 2 else -1.0
        assert np.abs(A[v] - sgn * R[v]).max() < bar * (np.abs(A[v]).max() + 1.0), v
    s0 = interior(cfg, U0).reshape(8, -1).sum(axis=1)
    s1 = interior(cfg, U).reshape(8, -1).sum(axis=1)
    sc = np.abs(interior(cfg, U0)).reshape(8, -1).sum(axis=1)
    assert np.all(np.abs(s1 - s0) <= (1e-12 if precision == "fp64" else 1e-6) * sc)


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-9), ("mixed", 1e-3)])
def test_explosion_mirror_symmetries(kh, orc, precision, bar):
    cfg, P = _problem("explosion", 256, precision)
    P = orc.apply_bc(cfg, P)
    _, Pg = _run_to(kh, cfg, P, 2.0)
    A = interior(cfg, Pg)
    assert np.isfinite(A).all()
    odd_x, odd_y = {2, 6, 7}, {3, 6}
    for v in range(8):
        sc = np.abs(A[v]).max() + 1e-300
        Rx = A[v][:, :, ::-1] * (-1.0 if v in odd_x else 1.0)
        Ry = A[v][:, ::-1, :] * (-1.0 if v in odd_y else 1.0)
        assert np.abs(A[v] - Rx).max() <= bar * sc, ("x", v)
        assert np.abs(A[v] - Ry).max() <= bar * sc, ("y", v)
