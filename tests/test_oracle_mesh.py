"""The oracle's refined mesh pinned to things other than itself: a mesh of
uneven blocks at one level reproduces the single-grid oracle step (whose
boundary rules are independent code), and the refined ghost fill reproduces
linear data exactly (MC prolongation and volume-average restriction are exact
for linear functions), including across periodic wraps."""
import numpy as np
import pytest

from mesh_cases import blk, box_two_level, mode_states, slice_blocks, torus_base, uneven_split, block_interior
from oracle.mesh import OracleMesh
from paper_2408_01361_gb300 import inputs


def _single_case(which):
    """Cases whose failed inversions (if any) lie away from the block edges: a
    failed zone is refilled from neighbours inside its own block, so a fixup
    next to a block edge legitimately differs from the single grid's."""
    if which == "torus_mc":
        cfg = torus_base(32, 24, "mc")
        P = inputs.torus_state(cfg, seed=2)
        blocks = uneven_split(cfg, [10, 28], [10, 14])
    else:
        cfg = inputs.linear_mode_cfg(16, ndim=3, recon="weno5" if which == "mode3d_weno5" else "mc")
        P = mode_states(cfg, [blk(0, 0, 0, 0, 16, 16, 16)])[0]
        blocks = uneven_split(cfg, [6], [10], [5])
    return cfg, P, blocks


@pytest.mark.parametrize("which", ["torus_mc", "mode3d", "mode3d_weno5"])
def test_single_level_mesh_equals_single_grid(orc, which):
    cfg, P, blocks = _single_case(which)
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    U1, P1, dt1, st1 = orc.step(cfg, U, P, dt)
    M = OracleMesh(cfg, blocks, inputs.block_cfg)
    Um, Pm, dtm, stm = M.step(slice_blocks(cfg, U, blocks), slice_blocks(cfg, P, blocks), dt)
    assert list(stm) == list(st1)
    ref_U = slice_blocks(cfg, U1, blocks)
    ref_P = slice_blocks(cfg, P1, blocks)
    for b, B in enumerate(blocks):
        for got, ref in ((Um[b], ref_U[b]), (Pm[b], ref_P[b])):
            g, r = block_interior(cfg, B, got), block_interior(cfg, B, ref)
            scale = np.abs(r).reshape(8, -1).max(axis=1)[:, None] + 1e-300
            err = (np.abs(g - r).reshape(8, -1) / scale).max()
            # the blocks' geometry is computed from their own origins: rounding only
            assert err < 1e-10, (b, err)
    assert abs(dtm - dt1) <= 1e-12 * dt1


@pytest.mark.parametrize("integrator", ["rk2", "ssprk54"])
def test_single_level_mesh_rk_equals_single_grid(orc, integrator):
    """The mesh's Runge-Kutta step (stage inputs ghost-filled across blocks)
    on uneven blocks at one level reproduces the single-grid oracle's
    Runge-Kutta step, whose stages fill ghosts by its own boundary rules."""
    cfg, P, blocks = _single_case("mode3d")
    cfg = dict(cfg, integrator=integrator)
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    U1, P1, dt1, st1 = orc.step(cfg, U, P, dt)
    M = OracleMesh(cfg, blocks, inputs.block_cfg)
    Um, Pm, dtm, stm = M.step_rk(slice_blocks(cfg, U, blocks), slice_blocks(cfg, P, blocks), dt, integrator)
    assert list(stm) == list(st1)
    ref_U, ref_P = slice_blocks(cfg, U1, blocks), slice_blocks(cfg, P1, blocks)
    for b, B in enumerate(blocks):
        for got, ref in ((Um[b], ref_U[b]), (Pm[b], ref_P[b])):
            g, r = block_interior(cfg, B, got), block_interior(cfg, B, ref)
            scale = np.abs(r).reshape(8, -1).max(axis=1)[:, None] + 1e-300
            assert (np.abs(g - r).reshape(8, -1) / scale).max() < 1e-10, b
    assert abs(dtm - dt1) <= 1e-12 * dt1
    # the stages differ from the predictor-corrector's
    Uv, _, _, _ = M.step(slice_blocks(cfg, U, blocks), slice_blocks(cfg, P, blocks), dt)
    assert max(np.abs(block_interior(cfg, B, a) - block_interior(cfg, B, c)).max()
               for B, a, c in zip(blocks, Um, Uv)) > 1e-12


def test_single_level_mesh_fofc_equals_single_grid(orc):
    """With the first-order flux correction the mesh runs every block's trial,
    fills the flags' ghost cells across blocks and corrects from them; on
    uneven blocks at one level this reproduces the single grid's correction,
    whose ghost flags follow its own boundary rules. The torus flags ~1,000
    zones (floors acting in the trial) and 30 inversions fail; the cuts lie
    away from those zones, whose fixup would otherwise draw on neighbours
    inside their own block only."""
    cfg = dict(torus_base(32, 24, "mc"), fofc=True)
    P = orc.apply_bc(cfg, inputs.torus_state(cfg, seed=2))
    blocks = uneven_split(cfg, [16], [10, 14])
    U = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    U1, P1, dt1, st1 = orc.step(cfg, U, P, dt)
    assert orc.last_nfofc > 500
    M = OracleMesh(cfg, blocks, inputs.block_cfg)
    Um, Pm, dtm, stm = M.step(slice_blocks(cfg, U, blocks), slice_blocks(cfg, P, blocks), dt)
    assert list(stm) == list(st1)
    ref_U, ref_P = slice_blocks(cfg, U1, blocks), slice_blocks(cfg, P1, blocks)
    for b, B in enumerate(blocks):
        for got, ref in ((Um[b], ref_U[b]), (Pm[b], ref_P[b])):
            g, r = block_interior(cfg, B, got), block_interior(cfg, B, ref)
            scale = np.abs(r).reshape(8, -1).max(axis=1)[:, None] + 1e-300
            assert (np.abs(g - r).reshape(8, -1) / scale).max() < 1e-10, b
    assert abs(dtm - dt1) <= 1e-12 * dt1
    # the correction changed the step
    Mp = OracleMesh(dict(cfg, fofc=False), blocks, inputs.block_cfg)
    Up, _, _, _ = Mp.step(slice_blocks(cfg, U, blocks), slice_blocks(cfg, P, blocks), dt)
    assert max(np.abs(block_interior(cfg, B, a) - block_interior(cfg, B, c)).max()
               for B, a, c in zip(blocks, Um, Up)) > 1e-8


def _linear_fill(base, blocks, coef):
    M = OracleMesh(base, blocks, inputs.block_cfg)
    Ps, centres = [], []
    for b, B in enumerate(blocks):
        c = inputs.block_cfg(base, B)
        X = [inputs.centers(c, d) for d in range(3)]
        Z, Y, Xx = np.meshgrid(X[2], X[1], X[0], indexing="ij")
        grid = (Xx, Y, Z)
        F = np.array([coef[v, 0] + sum(coef[v, d + 1] * grid[d] for d in range(3)) for v in range(8)])
        P = np.full(F.shape, np.nan)
        sl = (slice(None),) + inputs.interior(c)
        P[sl] = F[sl]
        Ps.append(P)
        centres.append((grid, F))
    M.fill_ghosts(Ps)
    return M, Ps, centres


@pytest.mark.parametrize("dim", [2, 3])
def test_refined_ghost_fill_exact_for_linear_data(dim):
    if dim == 2:
        base = inputs.linear_mode_cfg(16, ndim=2)
        base["bc"] = ["outflow", "outflow", "outflow", "outflow", "periodic", "periodic"]
        blocks = [blk(0, 0, 0, 0, 4, 16, 1), blk(0, 12, 0, 0, 4, 16, 1), blk(0, 4, 0, 0, 8, 4, 1),
                  blk(0, 4, 12, 0, 8, 4, 1), blk(1, 8, 8, 0, 10, 16, 1), blk(1, 18, 8, 0, 6, 16, 1)]
    else:
        base, blocks = box_two_level(16)
        base["bc"] = ["outflow"] * 6
    rng = np.random.default_rng(5)
    coef = rng.uniform(-1.0, 1.0, size=(8, 4))
    M, Ps, centres = _linear_fill(base, blocks, coef)
    dx0 = [(base[k][1] - base[k][0]) / base[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3"))]
    checked = {0: 0, 1: 0, -1: 0}
    for b, (P, (grid, F)) in enumerate(zip(Ps, centres)):
        assert np.isfinite(P).all(), b
        away = np.ones(P.shape[1:], dtype=bool)
        for d in range(dim):
            lo, hi = base[("x1", "x2", "x3")[d]]
            away &= (grid[d] > lo + 2 * dx0[d]) & (grid[d] < hi - 2 * dx0[d])
        ghost = np.ones(P.shape[1:], dtype=bool)
        ghost[inputs.interior(inputs.block_cfg(base, blocks[b]))] = False
        sel = away & ghost
        err = np.abs(P[:, sel] - F[:, sel]).max()
        assert err < 1e-12, (b, err)
        # which kinds of fill were exercised: the owner level of each checked ghost
        for idx in zip(*np.nonzero(sel)):
            x = [grid[d][idx] for d in range(3)]
            if dim == 2:
                x[2] = 0.5
            checked[blocks[M._owner(x)]["level"] - blocks[b]["level"]] += 1
    assert checked[0] > 0 and checked[1] > 0 and checked[-1] > 0, checked


def test_periodic_prolongation_wraps():
    """A refined block touching a periodic edge prolongs with a slope whose
    neighbour value comes from across the wrap: exact for data periodic and
    linear across the refined block's neighbourhood (a constant in x1 plus a
    linear function of x2)."""
    base = inputs.linear_mode_cfg(16, ndim=2)
    base["bc"] = ["periodic", "periodic", "outflow", "outflow", "periodic", "periodic"]
    blocks = [blk(1, 0, 0, 0, 8, 32, 1), blk(0, 4, 0, 0, 8, 16, 1), blk(1, 24, 0, 0, 8, 32, 1)]
    coef = np.zeros((8, 4))
    coef[:, 0] = np.arange(1, 9)
    coef[:, 2] = np.linspace(-1, 1, 8)
    M, Ps, centres = _linear_fill(base, blocks, coef)
    for P, (grid, F) in zip(Ps, centres):
        inside = (grid[1] > 2.0 / 16) & (grid[1] < 1 - 2.0 / 16)
        assert np.abs(P[:, inside] - F[:, inside]).max() < 1e-12
