"""GPU parity: the FP64 CUDA path (through the C ABI) against the FP64 CPU
oracle on the same seeded inputs. Bar: relative L1 per variable <= 1e-10,
and every cell within 5e-8 of max(|oracle|, 1e-3 x the variable's largest
magnitude) (gpu_helpers.assert_fp64_parity)."""
import os

import numpy as np
import pytest

from conftest import GOLDEN
from gpu_helpers import GpuRun, assert_fp64_parity, interior, rel_l1
from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


def _eig():
    return inputs.load_eigvec(os.path.join(GOLDEN, "linear_slow_mode.txt"))


def _torus_small(n1=48, n2=32, n3=16):
    cfg = inputs.torus_cfg(n1, n2, n3, r_out=60.0)
    return cfg, inputs.torus_state(cfg, seed=2)


def _random_cases():
    mink = inputs.linear_mode_cfg(20, ndim=3)
    Pm = inputs.random_prims(mink, seed=7, ut_scale=(6.0, 6.0, 6.0), b_scale=(4.0, 4.0, 4.0))
    fm = inputs.torus_cfg(40, 24, 1)
    fm["x1"] = (np.log(1.2), np.log(50.0))
    Pf = inputs.random_prims(fm, seed=8, ut_scale=(6.0, 6.0, 6.0), b_scale=(4.0, 4.0, 4.0))
    return [(mink, Pm), (fm, Pf)]


@pytest.mark.parametrize("case", [0, 1])
def test_prim_to_cons(kh, orc, case):
    cfg, P = _random_cases()[case]
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P)
    U, _ = g.host()
    Uo = orc.prim_to_cons(cfg, P)
    assert rel_l1(U, Uo).max() < 1e-13


@pytest.mark.parametrize("case", [0, 1])
def test_cons_to_prim(kh, orc, case):
    cfg, P = _random_cases()[case]
    Uo = orc.prim_to_cons(cfg, P)
    guess = P * (1 + 0.05 * (inputs.uniform01(99, np.arange(P.size)).reshape(P.shape) - 0.5))
    Po, pflag_o, nfail_o = orc.cons_to_prim(cfg, Uo, guess)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, guess, U=Uo)
    pflag = ctx.torch.zeros(ctx.shape(1)[1:], dtype=ctx.torch.int8, device=ctx.device)
    nfail = ctx.cons_to_prim(g.U, g.P, g.B, pflag)
    _, Pg = g.host()
    assert nfail == nfail_o == 0
    assert_fp64_parity(Pg, Po, "c2p")
    assert int(pflag.abs().sum()) == 0


@pytest.mark.parametrize("which", ["mode3d", "bondi", "torus"])
def test_fluxes(kh, orc, which):
    if which == "mode3d":
        cfg = inputs.linear_mode_cfg(16, ndim=3)
        dP, om = _eig()
        P = inputs.linear_mode_state(cfg, dP, om, amp=0.05)
        dirich = None
    elif which == "bondi":
        cfg = inputs.bondi_cfg(32, 32)
        P, dirich = inputs.bondi_state(cfg, seed=1)
    else:
        cfg, P = _torus_small()
        dirich = None
    P = orc.apply_bc(cfg, P, dirich)
    Fo, cto = orc.fluxes(cfg, P)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P)
    F = [ctx.empty(8) for _ in range(3)]
    ctx.fluxes(g.P, g.B, F[0], F[1], F[2] if cfg["n3"] > 1 else None)
    nd = 3 if cfg["n3"] > 1 else 2
    for d in range(nd):
        Fg = ctx.to_host(F[d], P.shape[3])
        # compare every entry the oracle computed (others are zero there)
        mask = np.abs(Fo[d]).sum(axis=0) > 0
        a = Fg[:, mask]
        b = Fo[d][:, mask]
        assert_fp64_parity(a, b, ("flux", d))


def _step_case(which):
    if which == "mode3d":
        cfg = inputs.linear_mode_cfg(32, ndim=3)
        dP, om = _eig()
        return cfg, inputs.linear_mode_state(cfg, dP, om), None
    if which == "bondi":
        cfg = inputs.bondi_cfg(64, 64)
        P, dirich = inputs.bondi_state(cfg, seed=1)
        return cfg, P, dirich
    if which == "torus_mc":
        cfg, P = _torus_small()
        cfg["recon"] = "mc"
        return cfg, P, None
    cfg, P = _torus_small()
    return cfg, P, None


@pytest.mark.parametrize("which", ["mode3d", "bondi", "torus_mc", "torus_weno5"])
@pytest.mark.parametrize("nsteps", [1, 10])
def test_step_parity(kh, orc, which, nsteps):
    cfg, P, dirich = _step_case(which)
    Uo = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P, dirich)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P, U=Uo, dirichlet=dirich)
    dt_gpu = ctx.cfl_dt(g.P, g.B)
    assert abs(dt_gpu - 2 * dt) <= 1e-12 * 2 * dt
    Uc, Pc = Uo, P
    for _ in range(nsteps):
        Uc, Pc, dtn_o, st_o = orc.step(cfg, Uc, Pc, dt, dirich)
        dtn_g, nfail = ctx.step(g.U, g.P, g.B, dt)
        assert nfail == st_o[0]
    Ug, Pg = g.host()
    assert_fp64_parity(interior(cfg, Ug), interior(cfg, Uc), "U")
    assert_fp64_parity(interior(cfg, Pg), interior(cfg, Pc), "P")
    assert abs(dtn_g - dtn_o) <= 1e-10 * dtn_o


@pytest.mark.parametrize("which", ["mode3d", "torus_weno5"])
def test_divb_parity_and_invariance(kh, orc, which):
    cfg, P, dirich = _step_case(which)
    P = orc.apply_bc(cfg, P, dirich)
    mo, lo = orc.divb(cfg, P)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P)
    mg, lg = ctx.divb(g.B)
    # the corner divergence is a sum of terms of size |sqrt(-g) B| / dx that
    # cancel: compare at that scale (both values are round-off when B comes
    # from a vector potential)
    gdet = orc.geometry(cfg, 0)[2]
    scale = np.abs(gdet[None, None] * P[5:8]).max() / min(
        (cfg["x1"][1] - cfg["x1"][0]) / cfg["n1"], (cfg["x2"][1] - cfg["x2"][0]) / cfg["n2"])
    assert abs(mg - mo) <= 1e-10 * mo + 1e-13 * scale and abs(lg - lo) <= 1e-10 * lo + 1e-13 * scale
    dt = 0.5 * ctx.cfl_dt(g.P, g.B)
    for _ in range(3):
        ctx.step(g.U, g.P, g.B, dt)
    ctx.fill_ghosts(g.P, g.B)
    m2, _ = ctx.divb(g.B)
    assert abs(m2 - mg) < 1e-12 * scale + 1e-12 * mg


def test_determinism(kh):
    cfg, P, _ = _step_case("torus_weno5")
    outs = []
    for _ in range(2):
        ctx = kh.Context(cfg)
        g = GpuRun(ctx, cfg, P)
        dt = 0.5 * ctx.cfl_dt(g.P, g.B)
        for _ in range(3):
            ctx.step(g.U, g.P, g.B, dt)
        outs.append(g.host())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_linear_mode_one_period_gpu(kh, orc):
    """The paper's regression problem run to one wave period on the GPU path:
    pointwise parity with the oracle over the whole (smooth) run, and the
    error against the analytic mode equal to the oracle's."""
    cfg = inputs.linear_mode_cfg(32, ndim=3)
    dP, om = _eig()
    P = inputs.linear_mode_state(cfg, dP, om)
    T = 2 * np.pi / om
    dt0 = orc.cfl_dt(cfg, P)
    Uo = orc.prim_to_cons(cfg, P)
    Uo2, Po2, to, st = orc.evolve(cfg, Uo, P, 0, -dt0, T)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P, U=Uo)
    t = 0.0
    dt = dt0
    while t < T * (1 - 1e-14):
        h = min(dt, T - t)
        dt, nfail = ctx.step(g.U, g.P, g.B, h)
        assert nfail == 0
        t += h
    assert abs(t - to) < 1e-12
    _, Pg = g.host()
    assert_fp64_parity(interior(cfg, Pg), interior(cfg, Po2), "P")
    Pex = inputs.linear_mode_state(cfg, dP, om, t=T)
    sl = inputs.interior(cfg)
    eg = np.array([np.abs(Pg[v][sl] - Pex[v][sl]).mean() for v in range(8)])
    eo = np.array([np.abs(Po2[v][sl] - Pex[v][sl]).mean() for v in range(8)])
    assert np.all(np.abs(eg - eo) <= 1e-6 * eo + 1e-18), (eg, eo)


def test_full_size_torus_one_step(kh, orc):
    """The benchmark workload (192x96x96 FMKS torus, WENO5) at full size, in the
    launch configuration the benchmark times: one step vs the oracle."""
    cfg = inputs.torus_cfg(192, 96, 96)
    P = inputs.torus_state(cfg, seed=2)
    Uo = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    Uo2, Po2, dto, st = orc.step(cfg, Uo, P, dt)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P, U=Uo)
    dtg, nfail = ctx.step(g.U, g.P, g.B, dt)
    assert nfail == st[0]
    Ug, Pg = g.host()
    assert_fp64_parity(interior(cfg, Ug), interior(cfg, Uo2), "U")
    assert_fp64_parity(interior(cfg, Pg), interior(cfg, Po2), "P")
    assert abs(dtg - dto) <= 1e-10 * dto


def test_full_size_bondi_10_steps(kh, orc):
    """The 128x128 MKS Bondi problem at full size, 10 steps (smooth flow)."""
    cfg = inputs.bondi_cfg(128, 128)
    P, dirich = inputs.bondi_state(cfg, seed=1)
    Uo = orc.prim_to_cons(cfg, P)
    dt = orc.cfl_dt(cfg, P, dirich)
    Uc, Pc = Uo, P
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P, U=Uo, dirichlet=dirich)
    dtg = dt
    for _ in range(10):
        Uc, Pc, dt, st = orc.step(cfg, Uc, Pc, dt, dirich)
        dtg2, nfail = ctx.step(g.U, g.P, g.B, dtg)
        dtg = dtg2
    Ug, Pg = g.host()
    assert_fp64_parity(interior(cfg, Ug), interior(cfg, Uc), "U")
    assert_fp64_parity(interior(cfg, Pg), interior(cfg, Pc), "P")


def test_ragged_and_minimum_sizes(kh, orc):
    """Row length not a multiple of the 16-element padding, odd sizes, and the
    minimum grid (4 zones per direction)."""
    for n1, n2, n3 in ((37, 23, 11), (4, 4, 4), (5, 7, 1)):
        cfg = inputs.linear_mode_cfg(8, ndim=3)
        cfg.update(n1=n1, n2=n2, n3=n3)
        P = inputs.random_prims(cfg, seed=3, rho_range=(0.5, 1.0), u_range=(0.3, 1.0), ut_scale=(0.3, 0.3, 0.3),
                                b_scale=(0.3, 0.3, 0.3))
        P = orc.apply_bc(cfg, P)
        Uo = orc.prim_to_cons(cfg, P)
        dt = 0.3 * orc.cfl_dt(cfg, P)
        Uo2, Po2, _, st = orc.step(cfg, Uo, P, dt)
        ctx = kh.Context(cfg)
        g = GpuRun(ctx, cfg, P, U=Uo)
        _, nfail = ctx.step(g.U, g.P, g.B, dt)
        assert nfail == st[0]
        Ug, Pg = g.host()
        assert_fp64_parity(interior(cfg, Ug), interior(cfg, Uo2), ("U", n1, n2, n3))
        assert_fp64_parity(interior(cfg, Pg), interior(cfg, Po2), ("P", n1, n2, n3))


def test_failed_inversion_fixup_parity(kh, orc):
    """Zones whose conserved state has no physical inversion (momentum beyond
    what the energy allows) fail in both stages; the neighbour-average fixup
    and the re-synchronised U must match the oracle's."""
    cfg = inputs.linear_mode_cfg(12, ndim=3)
    P = inputs.random_prims(cfg, seed=5, rho_range=(0.5, 1.0), u_range=(0.3, 1.0), ut_scale=(0.2, 0.2, 0.2),
                            b_scale=(0.2, 0.2, 0.2))
    P = orc.apply_bc(cfg, P)
    Uo = orc.prim_to_cons(cfg, P)
    for (k, j, i) in ((5, 5, 5), (6, 9, 4), (10, 3, 12)):
        Uo[2, k, j, i] = 40.0 * abs(Uo[1, k, j, i]) + 40.0
    dt = 0.2 * orc.cfl_dt(cfg, P)
    Uo2, Po2, _, st = orc.step(cfg, Uo, P, dt)
    assert st[0] >= 6
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P, U=Uo)
    _, nfail = ctx.step(g.U, g.P, g.B, dt)
    assert nfail == st[0]
    Ug, Pg = g.host()
    assert_fp64_parity(interior(cfg, Ug), interior(cfg, Uo2), "U")
    assert_fp64_parity(interior(cfg, Pg), interior(cfg, Po2), "P")


def test_inversion_failure_codes_match(kh, orc):
    """Crafted unphysical U: both inverters report failure at the same cells."""
    cfg = inputs.linear_mode_cfg(8, ndim=2)
    P = inputs.random_prims(cfg, seed=9, ut_scale=(1.0, 1.0, 1.0), b_scale=(1.0, 1.0, 1.0))
    Uo = orc.prim_to_cons(cfg, P)
    bad = np.zeros(Uo.shape[1:], dtype=bool)
    bad[0, 2:5, 3:9] = True
    Uo[2][bad] = 100.0 * np.abs(Uo[1][bad]) + 100.0
    Po, pflag_o, nfail_o = orc.cons_to_prim(cfg, Uo, P)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P, U=Uo)
    pflag = ctx.torch.zeros(ctx.shape(1)[1:], dtype=ctx.torch.int8, device=ctx.device)
    nfail = ctx.cons_to_prim(g.U, g.P, g.B, pflag)
    pf = pflag.cpu().numpy()[:, :, :P.shape[3]]
    assert nfail == nfail_o == int(bad.sum())
    assert np.array_equal(pf != 0, pflag_o != 0)
