"""GPU parity of the first-order flux correction (FP64 path, through the C
ABI) against the oracle's, on the same seeded inputs: periodic boxes where
some or all zones are flagged, 2-D and 3-D tori whose atmosphere sits at its
floors, and a Bondi flow with Dirichlet x1 ghosts. Bar: relative L1 per
variable <= 1e-10, flagged-zone counts equal."""
import numpy as np
import pytest

from gpu_helpers import GpuRun, assert_fp64_parity, interior, rel_l1
from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


def _box(rho_min, n=(20, 12, 10), seed=3):
    cfg = inputs.linear_mode_cfg(8, ndim=3, recon="weno5")
    cfg["n1"], cfg["n2"], cfg["n3"] = n
    cfg = dict(cfg, floors=dict(rho_min=rho_min, u_min=1e-20))
    rng = np.random.default_rng(seed)
    P = np.zeros(inputs.shape(cfg))
    P[0] = 1.0 + 0.1 * rng.random(P[0].shape)
    P[1] = 1.0 + 0.1 * rng.random(P[1].shape)
    P[2:5] = 0.1 * rng.normal(size=P[2:5].shape)
    P[5:] = 0.5 * rng.normal(size=P[5:].shape)
    return cfg, P, None


def _case(which):
    if which == "box_none":
        return _box(1e-20)
    if which == "box_some":
        return _box(1.05)
    if which == "box_all":
        return _box(10.0)
    if which == "torus3d":
        return _rough_torus(16, "weno5")
    if which == "torus2d_mc":
        return _rough_torus(1, "mc")
    cfg = inputs.bondi_cfg(64, 64)
    cfg["floors"] = dict(cfg["floors"], rho_min=0.1)  # the outer third floors
    P, dirich = inputs.bondi_state(cfg, seed=1)
    return cfg, P, dirich


def _rough_torus(n3, recon):
    """FM torus with seeded roughness on every zone and component (rho, u: 1%
    relative; u~: 1e-3 of the largest; B: 1e-3 sqrt(rho)). The plain torus's
    atmosphere sits exactly at its floors, where whether a floor acts is
    decided by round-off; a flag decided that way may differ between two
    correct implementations and then selects different face fluxes. Here
    every zone's decision has a margin far above round-off."""
    cfg = inputs.torus_cfg(48, 32, n3, r_out=60.0, recon=recon)
    P = inputs.torus_state(cfg, seed=2)
    xi = inputs.uniform01(13, np.arange(P.size)).reshape(P.shape) - 0.5
    sc = np.maximum(np.abs(P).reshape(8, -1).max(axis=1), 1e-2)[:, None, None, None]
    Pr = P + 1e-3 * sc * xi
    Pr[0:2] = P[0:2] * (1 + 1e-2 * xi[0:2])
    Pr[5:] = P[5:] + 1e-3 * np.sqrt(P[0:1]) * xi[5:]
    return cfg, Pr, None


def _run(kh, orc, cfg, P, dirich, nsteps, graph=False):
    cfg = dict(cfg, fofc=True)
    Uo = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P, dirich)
    ctx = kh.Context(cfg)
    ctx.set_graph(graph)
    g = GpuRun(ctx, cfg, P, U=Uo, dirichlet=dirich)
    Uc, Pc = Uo, P
    counts = []
    for _ in range(nsteps):
        Uc, Pc, dtn_o, st_o = orc.step(cfg, Uc, Pc, dt, dirich)
        n_o = orc.last_nfofc
        ctx.step(g.U, g.P, g.B, dt, sync=False)
        st = ctx.stats()
        counts.append((st.nfofc, n_o, st.nfail, st_o[0], st.nfloor, st_o[1]))
    Ug, Pg = g.host()
    return cfg, Ug, Pg, Uc, Pc, counts, st.dt_cfl, dtn_o


@pytest.mark.parametrize("which,nsteps", [("box_none", 1), ("box_some", 1), ("box_some", 3), ("box_all", 1),
                                          ("torus3d", 1), ("torus3d", 3), ("torus2d_mc", 5), ("bondi", 1),
                                          ("bondi", 3)])
def test_fofc_step_parity(kh, orc, which, nsteps):
    cfg, P, dirich = _case(which)
    cfg, Ug, Pg, Uc, Pc, counts, dtg, dto = _run(kh, orc, cfg, P, dirich, nsteps)
    for c in counts:
        assert c[0] == c[1] and c[2] == c[3] and c[4] == c[5], counts
    if which == "box_none":
        assert all(c[0] == 0 for c in counts)
    else:
        assert all(c[0] > 0 for c in counts)
    assert_fp64_parity(interior(cfg, Ug), interior(cfg, Uc), "U")
    assert_fp64_parity(interior(cfg, Pg), interior(cfg, Pc), "P")
    assert abs(dtg - dto) <= 1e-10 * dto


def test_fofc_without_flags_is_the_plain_step(kh, orc):
    cfg, P, _ = _box(1e-20)
    outs = []
    for fofc in (False, True):
        c = dict(cfg, fofc=fofc)
        ctx = kh.Context(c)
        g = GpuRun(ctx, c, P)
        for _ in range(2):
            ctx.step(g.U, g.P, g.B, 1e-3)
        outs.append(g.host())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_fofc_graph_replay_matches_eager(kh, orc):
    cfg, P, dirich = _case("torus3d")
    a = _run(kh, orc, cfg, P, dirich, 3, graph=False)
    b = _run(kh, orc, cfg, P, dirich, 3, graph=True)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert a[5] == b[5]


def test_fofc_adjoint_refused(kh):
    cfg, P, _ = _box(1.05)
    ctx = kh.Context(dict(cfg, fofc=True))
    g = GpuRun(ctx, dict(cfg, fofc=True), P)
    gU = [ctx.empty(8) for _ in range(2)]
    with pytest.raises(kh.KHError):
        ctx.step_adjoint(g.U, g.P, g.B, 1e-3, gU=gU[0])


# ---- mixed precision: FP32 trial decisions and FP32 donor-cell fluxes ----

def test_mixed_fofc_all_and_none_flagged(kh, orc):
    for rho_min, expect in ((1e-20, 0), (10.0, 2 * 20 * 12 * 10)):
        cfg, P, _ = _box(rho_min)
        outs = []
        for fofc in (False, True):
            c = dict(cfg, fofc=fofc, precision="mixed")
            ctx = kh.Context(c)
            g = GpuRun(ctx, c, P)
            ctx.step(g.U, g.P, g.B, 1e-3)
            assert ctx.stats().nfofc == (expect if fofc else 0)
            outs.append(g.host())
        same = np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
        assert same == (expect == 0)
    # every zone flagged: the mixed step is first order; against the oracle's
    # donor-cell step at the mixed path's FP32 level
    c = dict(cfg, recon="donor")
    U = orc.prim_to_cons(c, P)
    Uo, Po, _, _ = orc.step(c, U, P, 1e-3)
    ep = rel_l1(interior(cfg, outs[1][1]), interior(cfg, Po))
    eu = rel_l1(interior(cfg, outs[1][0]), interior(cfg, Uo))
    assert ep.max() < 1e-5 and eu.max() < 1e-5, (ep, eu)


@pytest.mark.parametrize("which", ["box_some", "torus3d"])
def test_mixed_fofc_vs_oracle(kh, orc, which):
    cfg, P, dirich = _case(which)
    cfg = dict(cfg, fofc=True)
    Uo = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P, dirich)
    Uo2, Po2, _, st_o = orc.step(cfg, Uo, P, dt, dirich)
    n_o = orc.last_nfofc
    c = dict(cfg, precision="mixed")
    ctx = kh.Context(c)
    g = GpuRun(ctx, c, P, U=Uo)
    ctx.step(g.U, g.P, g.B, dt)
    n_g = ctx.stats().nfofc
    # FP32 decisions: a zone within FP32 rounding of a threshold may go
    # either way (the rough states keep such zones rare)
    assert abs(n_g - n_o) <= 2 + n_o // 200, (n_g, n_o)
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
