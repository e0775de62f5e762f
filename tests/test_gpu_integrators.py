"""GPU parity of the Runge-Kutta integrators (RK1, RK2, SSPRK(5,4); FP64,
Flux-CT) with the oracle's on a periodic box and on the FMKS torus
(floors, failed inversions and their fixup included), their temporal orders
on a fixed grid, and graph replay equal to eager stepping."""
import os

import numpy as np
import pytest

from conftest import GOLDEN
from gpu_helpers import TOL, GpuRun, interior, rel_l1
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
    eu = rel_l1(interior(cfg, Ug), interior(cfg, Uc))
    ep = rel_l1(interior(cfg, Pg), interior(cfg, Pc))
    assert eu.max() < TOL and ep.max() < TOL, (eu, ep)
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
