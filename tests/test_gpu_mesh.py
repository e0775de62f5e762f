"""Refined mesh on the GPU (one launch per kernel over all blocks, one ghost
gather) against the oracle's mesh: FP64 within 1e-10 relative L1 per
variable and block, mixed precision within the bounds of the single-grid
mixed path, the graph replay bit-identical to direct launches, and a mesh of
uneven blocks at one level equal to the single-grid CUDA step."""
import numpy as np
import pytest

from gpu_helpers import ELEM_TOL, TOL, GpuRun, assert_fp64_parity, elem_err, interior, rel_l1
from mesh_cases import (block_interior, blk, box_two_level, mode_states, slice_blocks, torus_base, torus_states,
                        torus_three_level, torus_two_level, uneven_split)
from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


@pytest.fixture(scope="module")
def OM():
    from oracle.mesh import OracleMesh
    return OracleMesh


def _case(which):
    if which == "torus2_mc":
        base, blocks = torus_two_level("mc")
        return base, blocks, torus_states(base, blocks)
    if which == "torus2_weno5":
        base, blocks = torus_two_level("weno5")
        return base, blocks, torus_states(base, blocks)
    if which == "torus3_weno5":
        base, blocks = torus_three_level("weno5")
        return base, blocks, torus_states(base, blocks)
    base, blocks = box_two_level(16, "weno5" if which == "box_weno5" else "mc")
    return base, blocks, mode_states(base, blocks)


def _oracle_run(orc, OM, base, blocks, Ps, nsteps, dt=None):
    M = OM(base, blocks, inputs.block_cfg)
    Us = [orc.prim_to_cons(inputs.block_cfg(base, b), P) for b, P in zip(blocks, Ps)]
    if dt is None:
        dt = 0.5 * _mesh_cfl(orc, M, base, blocks, Ps)
    U0 = [u.copy() for u in Us]
    out = []
    Uc, Pc = Us, Ps
    for _ in range(nsteps):
        Uc, Pc, dtn, st = M.step(Uc, Pc, dt)
        out.append((dtn, st))
    return U0, dt, Uc, Pc, out


def _mesh_cfl(orc, M, base, blocks, Ps):
    """CFL dt of the mesh state from the oracle's per-block fluxes."""
    Pf = [P.copy() for P in Ps]
    M.fill_ghosts(Pf)
    cts = [orc.fluxes(inputs.block_cfg(base, b), P)[1] for b, P in zip(blocks, Pf)]
    return M.cfl_dt(cts)


def _flat(base, blocks, arrays):
    """(8, zones of all blocks): every block's interior, concatenated."""
    return np.concatenate([block_interior(base, B, A).reshape(8, -1) for B, A in zip(blocks, arrays)], axis=1)


def _compare(base, blocks, got, ref, tol):
    """Relative L1 per variable over the whole mesh (blocks at the poles hold
    only atmosphere, where momenta are round-off: a per-block norm would
    measure round-off against round-off); at the FP64 parity bar also the
    element-wise bound of gpu_helpers.elem_err, over the whole mesh."""
    a, b = _flat(base, blocks, got), _flat(base, blocks, ref)
    e = rel_l1(a, b)
    assert e.max() < tol, e
    if tol == TOL:
        x = elem_err(a, b)
        assert x.max() < ELEM_TOL, x


def test_mesh_prim_to_cons(kh, orc):
    base, blocks, Ps = _case("torus2_mc")
    m = kh.Mesh(base, blocks)
    P, B = m.to_device(Ps)
    U = m.empty(8)
    m.prim_to_cons(P, B, U)
    Uo = [orc.prim_to_cons(inputs.block_cfg(base, b), Pb) for b, Pb in zip(blocks, Ps)]
    # the theta momentum of the equilibrium torus is itself metric round-off
    _compare(base, blocks, m.cons_to_host(U), Uo, 1e-11)


@pytest.mark.parametrize("which", ["torus2_mc", "torus2_weno5", "torus3_weno5", "box_mc", "box_weno5"])
def test_mesh_ghost_fill_matches_oracle(kh, OM, which):
    base, blocks, Ps = _case(which)
    m = kh.Mesh(base, blocks)
    P, B = m.to_device(Ps)
    m.fill_ghosts(P, B)
    got = m.to_host(P, B)
    M = OM(base, blocks, inputs.block_cfg)
    ref = [p.copy() for p in Ps]
    M.fill_ghosts(ref)
    for b in range(len(blocks)):
        N1 = blocks[b]["n1"] + 6
        scale = np.abs(ref[b][:, :, :, :N1]).reshape(8, -1).max(axis=1) + 1e-300
        err = (np.abs(got[b] - ref[b][:, :, :, :N1]).reshape(8, -1).max(axis=1) / scale).max()
        assert err < 1e-14, (b, err)


@pytest.mark.parametrize("which,nsteps", [("torus2_mc", 2), ("torus2_weno5", 2), ("torus3_weno5", 1),
                                          ("box_mc", 1), ("box_weno5", 1)])
def test_mesh_step_parity(kh, orc, OM, which, nsteps):
    base, blocks, Ps = _case(which)
    U0, dt, Uo, Po, hist = _oracle_run(orc, OM, base, blocks, Ps, nsteps)
    m = kh.Mesh(base, blocks)
    P, B = m.to_device(Ps)
    U = m.cons_to_device(U0)
    assert abs(m.cfl_dt(P, B) - 2 * dt) <= 1e-10 * 2 * dt
    for q in range(nsteps):
        dtn, nfail = m.step(U, P, B, dt)
        assert nfail == hist[q][1][0]
        assert abs(dtn - hist[q][0]) <= 1e-10 * hist[q][0]
    _compare(base, blocks, m.cons_to_host(U), Uo, TOL)
    _compare(base, blocks, m.to_host(P, B), Po, TOL)


@pytest.mark.parametrize("which", ["torus_mc", "mode3d_weno5"])
def test_single_level_mesh_equals_single_grid_gpu(kh, orc, which):
    if which == "torus_mc":
        cfg = torus_base(32, 24, "mc")
        Pfull = inputs.torus_state(cfg, seed=2)
        blocks = uneven_split(cfg, [10, 28], [10, 14])
    else:
        cfg = inputs.linear_mode_cfg(16, ndim=3, recon="weno5")
        Pfull = mode_states(cfg, [blk(0, 0, 0, 0, 16, 16, 16)])[0]
        blocks = uneven_split(cfg, [6], [10], [5])
    Pfull = orc.apply_bc(cfg, Pfull)
    Ufull = orc.prim_to_cons(cfg, Pfull)
    dt = 0.5 * orc.cfl_dt(cfg, Pfull)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, Pfull, U=Ufull)
    m = kh.Mesh(cfg, blocks)
    P, B = m.to_device(slice_blocks(cfg, Pfull, blocks))
    U = m.cons_to_device(slice_blocks(cfg, Ufull, blocks))
    # the torus runs one step: later failed inversions fall next to block
    # edges, where a fixup averages over its own block only
    for _ in range(1 if which == "torus_mc" else 3):
        dts, nf_s = ctx.step(g.U, g.P, g.B, dt)
        dtm, nf_m = m.step(U, P, B, dt)
        assert nf_s == nf_m
        assert abs(dts - dtm) <= 1e-12 * dts
    Ug, PBg = g.host()
    refU, refP = slice_blocks(cfg, Ug, blocks), slice_blocks(cfg, PBg, blocks)
    _compare(cfg, blocks, m.cons_to_host(U), refU, 1e-12)
    _compare(cfg, blocks, m.to_host(P, B), refP, 1e-12)


def test_mesh_mixed_error_vs_oracle(kh, orc, OM):
    base, blocks, Ps = _case("torus2_weno5")
    U0, dt, Uo, Po, hist = _oracle_run(orc, OM, base, blocks, Ps, 1)
    mb = dict(base, precision="mixed")
    m = kh.Mesh(mb, blocks)
    P, B = m.to_device(Ps)
    U = m.cons_to_device(U0)
    dtn, _ = m.step(U, P, B, dt)
    assert abs(dtn - hist[0][0]) < 1e-5 * hist[0][0]
    a, r = _flat(base, blocks, m.cons_to_host(U)), _flat(base, blocks, Uo)
    pa, pr = _flat(base, blocks, m.to_host(P, B)), _flat(base, blocks, Po)
    mass, nz = np.abs(r[0]).sum(), r[0].size
    # the near-equilibrium norm of the single-grid mixed-path test (momenta
    # and velocities against the mass scale / 1e-2 per zone; the rest
    # relative) and the element-wise error, each within 5x of the error
    # measured on GB300 when the bounds were set (floor 1e-9)
    meas = dict(
        U=[3.6e-10, 9.6e-9, 7.4e-9, 1.7e-6, 7.3e-9, 2.7e-11, 8.2e-12, 2.3e-10],
        P=[4.0e-10, 2.9e-8, 1.9e-6, 4.1e-8, 2.2e-6, 4.8e-10, 2.1e-10, 2.2e-6],
        eU=[1.3e-6, 2.6e-5, 1.7e-4, 2.5e-4, 2.3e-4, 2.1e-7, 1.7e-7, 3.4e-3],
        eP=[5.7e-7, 1.7e-6, 2.6e-2, 1.7e-3, 6.0e-2, 6.8e-7, 1.6e-7, 2.7e-3])
    bound = {key: np.maximum(5.0 * np.array(val), 1e-9) for key, val in meas.items()}
    xu, xp = elem_err(a, r), elem_err(pa, pr)
    for v in range(8):
        den = max(np.abs(r[v]).sum(), 1e-3 * mass)
        assert np.abs(a[v] - r[v]).sum() / den < bound["U"][v], ("U", v)
        pden = max(np.abs(pr[v]).sum(), 1e-2 * nz if v in (2, 3, 4) else 0.0)
        assert np.abs(pa[v] - pr[v]).sum() / pden < bound["P"][v], ("P", v)
        assert xu[v] < bound["eU"][v] and xp[v] < bound["eP"][v], (v, xu, xp)


def _mesh_run(kh, base, blocks, Ps, U0, dt, nsteps, **over):
    m = kh.Mesh(dict(base, **over), blocks)
    P, B = m.to_device(Ps)
    U = m.cons_to_device(U0)
    nf = []
    for _ in range(nsteps):
        _, nfail = m.step(U, P, B, dt)
        nf.append(nfail)
    return m.cons_to_host(U), m.to_host(P, B), nf


@pytest.mark.parametrize("inverter", ["1dw", "kastaun"])
def test_mesh_other_solvers(kh, orc, OM, inverter):
    """The refined mesh with the one-unknown (1D_W) and bracketed (Kastaun)
    solvers, its update kernels instantiated per solver. On the two-level 3-D
    box (no inversion fails) the FP64 mesh equals the oracle's mesh step
    (its own bracketed 1D_w inversion: every solver finds the same root)
    within the FP64 bar; the mixed mesh (these solvers invert in FP64 there)
    equals the double-float Noble-2D mixed mesh within 1e-5 element-wise
    (the same FP32 stencil; the inversions agree far below FP32)."""
    base, blocks, Ps = _case("box_weno5")
    U0, dt, Uo, Po, hist = _oracle_run(orc, OM, base, blocks, Ps, 2)
    assert all(h[1][0] == 0 for h in hist)
    Ug, Pg, nf = _mesh_run(kh, base, blocks, Ps, U0, dt, 2, inverter=inverter)
    assert nf == [0, 0]
    assert_fp64_parity(_flat(base, blocks, Ug), _flat(base, blocks, Uo), "U")
    assert_fp64_parity(_flat(base, blocks, Pg), _flat(base, blocks, Po), "P")
    Um, Pm, _ = _mesh_run(kh, base, blocks, Ps, U0, dt, 2, precision="mixed", inverter=inverter)
    Ud, Pd, _ = _mesh_run(kh, base, blocks, Ps, U0, dt, 2, precision="mixed")
    assert elem_err(_flat(base, blocks, Um), _flat(base, blocks, Ud)).max() < 1e-5
    assert elem_err(_flat(base, blocks, Pm), _flat(base, blocks, Pd)).max() < 1e-5


def test_mesh_mixed_fp64_inversion(kh, orc, OM):
    """The mixed mesh with the whole inversion and the floors in FP64 for
    every zone: the same failed zones as the oracle's mesh, and its state
    within 1e-4 element-wise of the double-float mixed mesh (as on single
    grids: the FP32 floor decisions and P* rounding remain)."""
    base, blocks, Ps = _case("torus2_weno5")
    U0, dt, Uo, Po, hist = _oracle_run(orc, OM, base, blocks, Ps, 1)
    Uf, Pf, nf = _mesh_run(kh, base, blocks, Ps, U0, dt, 1, precision="mixed", mixed_inversion="fp64")
    assert nf[0] == hist[0][1][0]
    Ud, Pd, _ = _mesh_run(kh, base, blocks, Ps, U0, dt, 1, precision="mixed")
    assert elem_err(_flat(base, blocks, Uf), _flat(base, blocks, Ud)).max() < 1e-4
    assert elem_err(_flat(base, blocks, Pf), _flat(base, blocks, Pd)).max() < 1e-4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mesh_graph_replay_bitwise(kh, precision):
    base, blocks, Ps = _case("torus3_weno5")
    base = dict(base, precision=precision)
    res = []
    for graph in (False, True):
        m = kh.Mesh(base, blocks)
        P, B = m.to_device(Ps)
        U = m.empty(8)
        m.prim_to_cons(P, B, U)
        m.set_graph(graph)
        dt = 0.5 * m.cfl_dt(P, B)
        for _ in range(3):
            dt_next, _ = m.step(U, P, B, dt)
        res.append((U.cpu().numpy(), P.cpu().numpy(), B.cpu().numpy(), dt_next))
    for a, b in zip(res[0][:3], res[1][:3]):
        assert np.array_equal(a, b)
    assert res[0][3] == res[1][3]


@pytest.mark.parametrize("bad", ["overlap", "hole", "odd", "jump"])
def test_mesh_rejects_invalid_layouts(kh, bad):
    base = torus_base(32, 24, "mc")
    if bad == "overlap":
        blocks = [blk(0, 0, 0, 0, 32, 24, 1), blk(0, 0, 0, 0, 8, 8, 1)]
    elif bad == "hole":
        blocks = [blk(0, 0, 0, 0, 32, 20, 1)]
    elif bad == "odd":
        blocks = [blk(0, 0, 0, 0, 32, 6, 1), blk(0, 0, 18, 0, 32, 6, 1), blk(1, 1, 12, 0, 63, 24, 1)]
    else:  # a level-2 block touching level-0 blocks
        blocks = [blk(0, 0, 0, 0, 32, 6, 1), blk(0, 0, 18, 0, 32, 6, 1), blk(2, 0, 24, 0, 128, 48, 1)]
    with pytest.raises(kh.KHError):
        kh.Mesh(base, blocks)


@pytest.mark.parametrize("which", ["torus2_weno5", "box_mc"])
def test_mesh_divb_parity_and_invariance(kh, orc, which):
    """Corner divB inside every block: equal to the oracle's per-block value
    at the start, held by Flux-CT through steps (level interfaces excluded)."""
    base, blocks, Ps = _case(which)
    m = kh.Mesh(base, blocks)
    P, B = m.to_device(Ps)
    mg, lg = m.divb(B)
    mx, tot, cnt, scale = 0.0, 0.0, 0, 0.0
    for b, Pb in zip(blocks, Ps):
        c = inputs.block_cfg(base, b)
        mo, lo = orc.divb(c, Pb)
        nc = (b["n1"] - 1) * (b["n2"] - 1) * (b["n3"] - 1 if base["n3"] > 1 else 1)
        mx, tot, cnt = max(mx, mo), tot + lo * nc, cnt + nc
        gdet = orc.geometry(c, 0)[2]
        dxm = min((c["x1"][1] - c["x1"][0]) / c["n1"], (c["x2"][1] - c["x2"][0]) / c["n2"])
        scale = max(scale, np.abs(gdet[None, None] * Pb[5:8]).max() / dxm)
    assert abs(mg - mx) <= 1e-10 * mx + 1e-13 * scale
    assert abs(lg - tot / cnt) <= 1e-10 * (tot / cnt) + 1e-13 * scale
    U = m.empty(8)
    m.prim_to_cons(P, B, U)
    dt = 0.5 * m.cfl_dt(P, B)
    for _ in range(3):
        m.step(U, P, B, dt)
    m2, _ = m.divb(B)
    assert abs(m2 - mg) < 1e-12 * scale + 1e-12 * mg


def test_mesh_launch_settings_and_autotune_bitwise(kh):
    """Threads per block change nothing in the result; the autotuner picks
    one of its candidates and caches it."""
    base, blocks, Ps = _case("torus2_weno5")
    res = []
    for cfg in ((64, 256), (256, 64), None):
        m = kh.Mesh(base, blocks)
        P, B = m.to_device(Ps)
        U = m.empty(8)
        m.prim_to_cons(P, B, U)
        dt = 0.5 * m.cfl_dt(P, B)
        if cfg is None:
            got = m.autotune(U, P, B, dt)
            assert got[0] in (64, 128, 256) and got[1] in (64, 128, 256)
            assert m.get_launch() == got
            assert m.autotune(U, P, B, dt) == got  # cached
        else:
            m.set_launch(*cfg)
            assert m.get_launch() == cfg
        for _ in range(2):
            m.step(U, P, B, dt)
        res.append((U.cpu().numpy(), P.cpu().numpy(), B.cpu().numpy()))
    for r in res[1:]:
        for a, b in zip(res[0], r):
            assert np.array_equal(a, b)
    with pytest.raises(kh.KHError):
        m.set_launch(48, 128)
