"""Face-centred CT on the oracle's refined mesh: a mesh of uneven blocks at
one level reproduces the single-grid face-CT step; on two-level meshes (the
2-D torus, the 3-D box with a refined centre) the face divergence of every
cell of every block stays at rounding, and each coarse face on a level
interface moves exactly as the mean of the fine faces covering it (the
edge-EMF matching), so their difference is constant in time -- zero for the
torus field, whose coarse faces start as the fine means."""
import numpy as np
import pytest

from mesh_cases import blk, box_two_level, slice_blocks, torus_base, torus_two_level, uneven_split, block_interior
from oracle.mesh import OracleMesh
from paper_2408_01361_gb300 import inputs


def _pad8(A):
    return np.concatenate([A, np.zeros((8 - A.shape[0],) + A.shape[1:])])


def _face_blocks(cfg, fB, blocks):
    return [f[:3] for f in slice_blocks(cfg, _pad8(fB), blocks)]


@pytest.mark.parametrize("which", ["torus_mc", "mode3d_weno5"])
def test_single_level_face_mesh_equals_single_grid(orc, which):
    if which == "torus_mc":
        cfg = dict(torus_base(32, 24, "mc"), bfield="face", emf="gs05")
        P = inputs.torus_state(cfg, seed=2)
        fB = inputs.torus_face_field(cfg)
        blocks = uneven_split(cfg, [10, 28], [10, 14])
    else:
        import os
        from conftest import GOLDEN
        cfg = dict(inputs.linear_mode_cfg(16, ndim=3, recon="weno5"), bfield="face", emf="gs05")
        dP, om = inputs.load_eigvec(os.path.join(GOLDEN, "linear_slow_mode.txt"))
        P = inputs.linear_mode_state(cfg, dP, om, amp=0.05)
        fB = inputs.linear_mode_face_field(cfg, dP, om, amp=0.05)
        blocks = uneven_split(cfg, [6], [10], [5])
    P = orc.apply_bc(cfg, inputs.cell_field_from_faces(cfg, fB, P))
    U = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    U1, P1, f1, dt1, st1 = orc.step_face(cfg, U, P, fB, dt)
    M = OracleMesh(cfg, blocks, inputs.block_cfg)
    Um, Pm, fm, dtm, stm = M.step_face(slice_blocks(cfg, U, blocks), slice_blocks(cfg, P, blocks),
                                       _face_blocks(cfg, fB, blocks), dt)
    assert list(stm) == list(st1)
    refs = (slice_blocks(cfg, U1, blocks), slice_blocks(cfg, P1, blocks))
    for b, B in enumerate(blocks):
        for got, ref in ((Um[b], refs[0][b]), (Pm[b], refs[1][b])):
            g, r = block_interior(cfg, B, got), block_interior(cfg, B, ref)
            scale = np.abs(r).reshape(8, -1).max(axis=1)[:, None] + 1e-300
            assert (np.abs(g - r).reshape(8, -1) / scale).max() < 1e-10, b
    assert abs(dtm - dt1) <= 1e-12 * dt1


def _interface_mismatch(M, fs):
    """Per coarse face on a level interface: coarse value - mean of the fine
    faces covering it."""
    out = []
    ng = M.ng
    for b, bb in enumerate(M.blocks):
        for f, fb in enumerate(M.blocks):
            if fb["level"] != bb["level"] + 1:
                continue
            cb, cf = M.cfgs[b], M.cfgs[f]
            nb = (cb["n1"], cb["n2"], cb["n3"])
            nf = (cf["n1"], cf["n2"], cf["n3"])
            for a in range(M.ndim):
                rng = [range(ng, ng + nb[q] + (1 if q == a else 0)) if q < M.ndim else range(0, 1) for q in range(3)]
                for k in rng[2]:
                    for j in rng[1]:
                        for i in rng[0]:
                            loc = (i, j, k)
                            cand = []
                            ok = True
                            for q in range(3):
                                if q >= M.ndim:
                                    cand.append([0])
                                    continue
                                G = M._global(b, q, loc[q])
                                xs = [M._local(f, q, 2 * G)] if q == a else [M._local(f, q, 2 * G),
                                                                              M._local(f, q, 2 * G + 1)]
                                hi = ng + nf[q] if q == a else ng + nf[q] - 1
                                ok &= all(ng <= x <= hi for x in xs)
                                cand.append(xs)
                            if not ok:
                                continue
                            fine = [fs[f][a][kk, jj, ii] for kk in cand[2] for jj in cand[1] for ii in cand[0]]
                            out.append(fs[b][a][k, j, i] - np.mean(fine))
    return np.array(out)


def _two_level(which):
    if which == "torus":
        base, blocks = torus_two_level("mc")
        base = dict(base, bfield="face", emf="gs05")
        norms = inputs.torus_norms(base)
        M = OracleMesh(base, blocks, inputs.block_cfg)
        Ps = [inputs.torus_state(c, seed=2, norms=norms) for c in M.cfgs]
        fs = [inputs.torus_face_field(c, norms=norms) for c in M.cfgs]
    else:
        import os
        from conftest import GOLDEN
        base, blocks = box_two_level(16, "mc")
        base = dict(base, bfield="face", emf="gs05")
        M = OracleMesh(base, blocks, inputs.block_cfg)
        dP, om = inputs.load_eigvec(os.path.join(GOLDEN, "linear_fast_mode.txt"))
        Ps = [inputs.linear_mode_state(c, dP, om, amp=0.05) for c in M.cfgs]
        fs = [inputs.linear_mode_face_field(c, dP, om, amp=0.05) for c in M.cfgs]
    Ps = [inputs.cell_field_from_faces(c, f, P) for c, f, P in zip(M.cfgs, fs, Ps)]
    M.fill_ghosts(Ps)
    return M, Ps, fs


@pytest.mark.parametrize("which", ["torus", "box3d"])
def test_two_level_face_divergence_and_interfaces(orc, which):
    M, Ps, fs = _two_level(which)
    Us = [orc.prim_to_cons(c, P) for c, P in zip(M.cfgs, Ps)]
    d0 = [orc.face_divb(c, f, field=True)[2] for c, f in zip(M.cfgs, fs)]
    m0 = _interface_mismatch(M, fs)
    assert m0.size > 0
    if which == "torus":
        assert np.abs(m0).max() < 1e-13 * max(np.abs(f).max() for f in fs)
    dt = 0.5 * min(orc.cfl_dt(c, P) for c, P in zip(M.cfgs, Ps))
    for _ in range(3):
        Us, Ps, fs, dtn, st = M.step_face(Us, Ps, fs, dt)
    scale = max(np.abs(f).max() for f in fs)
    for b, (c, f) in enumerate(zip(M.cfgs, fs)):
        dx = min((c[k][1] - c[k][0]) / c[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3")))
        d1 = orc.face_divb(c, f, field=True)[2]
        assert np.abs(d1 - d0[b]).max() < 1e-12 * scale / dx, b
    m1 = _interface_mismatch(M, fs)
    assert np.abs(m1 - m0).max() < 1e-13 * scale
    assert all(np.isfinite(P).all() for P in Ps)
