"""Face-centred CT on the GPU's refined mesh against the oracle's (interface
EMFs matched from the finer blocks): FP64 steps within 1e-10 for U, P and
the face fields on two- and three-level tori and the two-level 3-D box; the
face divergence of every block at rounding and each coarse interface face
equal to the mean of its fine faces up to a constant (FP64 and mixed); graph
replay bit-identical to direct launches."""
import os

import numpy as np
import pytest

from conftest import GOLDEN
from gpu_helpers import TOL, rel_l1
from mesh_cases import block_interior, box_two_level, torus_three_level, torus_two_level
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


def _case(which, precision="fp64"):
    if which.startswith("torus"):
        base, blocks = (torus_three_level if which == "torus3" else torus_two_level)(
            "weno5" if which != "torus2_mc" else "mc")
        base = dict(base, bfield="face", emf="gs05", precision=precision)
        norms = inputs.torus_norms(base)
        cfgs = [inputs.block_cfg(base, b) for b in blocks]
        Ps = [inputs.torus_state(c, seed=2, norms=norms) for c in cfgs]
        fs = [inputs.torus_face_field(c, norms=norms) for c in cfgs]
    else:
        base, blocks = box_two_level(16, "mc")
        base = dict(base, bfield="face", emf="gs05", precision=precision)
        dP, om = inputs.load_eigvec(os.path.join(GOLDEN, "linear_fast_mode.txt"))
        cfgs = [inputs.block_cfg(base, b) for b in blocks]
        Ps = [inputs.linear_mode_state(c, dP, om, amp=0.05) for c in cfgs]
        fs = [inputs.linear_mode_face_field(c, dP, om, amp=0.05) for c in cfgs]
    Ps = [inputs.cell_field_from_faces(c, f, P) for c, f, P in zip(cfgs, fs, Ps)]
    return base, blocks, cfgs, Ps, fs


def _flat(base, blocks, arrays, n=8):
    return np.concatenate([block_interior(base, B, A)[:n].reshape(n, -1) for B, A in zip(blocks, arrays)], axis=1)


def _gpu(kh, base, blocks, Ps, Us, fs, nsteps, dt, graph=False):
    m = kh.Mesh(base, blocks)
    m.set_graph(graph)
    P, B = m.to_device(Ps)
    U = m.cons_to_device(Us)
    fB = m.faces_to_device(fs)
    m.set_face_field(fB)
    hist = []
    for _ in range(nsteps):
        hist.append(m.step(U, P, B, dt))
    return m, m.cons_to_host(U), m.to_host(P, B), m.faces_to_host(fB), hist


@pytest.mark.parametrize("which,nsteps", [("torus2_mc", 2), ("torus2_weno5", 2), ("torus3", 1), ("box", 1)])
def test_mesh_face_ct_parity(kh, orc, OM, which, nsteps):
    base, blocks, cfgs, Ps, fs = _case(which)
    M = OM(base, blocks, inputs.block_cfg)
    Pf = [P.copy() for P in Ps]
    M.fill_ghosts(Pf)
    Us = [orc.prim_to_cons(c, P) for c, P in zip(cfgs, Pf)]
    dt = 0.5 * min(orc.cfl_dt(c, P) for c, P in zip(cfgs, Pf))
    Uo, Po, fo = Us, Pf, fs
    hist_o = []
    for _ in range(nsteps):
        Uo, Po, fo, dtn, st = M.step_face(Uo, Po, fo, dt)
        hist_o.append((dtn, st))
    m, Ug, Pg, fg, hist = _gpu(kh, base, blocks, Ps, Us, fs, nsteps, dt)
    for (dtg, nf), (dto, st) in zip(hist, hist_o):
        assert nf == st[0]
        assert abs(dtg - dto) <= 1e-10 * dto
    for got, ref in ((Ug, Uo), (Pg, Po)):
        fr, fg_ = _flat(base, blocks, ref), _flat(base, blocks, got)
        # per slot relative L1; field slots against the whole field's scale and
        # momentum slots against at least 1e-3 of the mass scale (the box's
        # level interfaces generate u~3 and B^3 ~ 1e-5 by cancellation of O(1)
        # terms: their own scale would measure rounding against cancellation)
        den = np.abs(fr).sum(axis=1)
        den[5:] = np.abs(fr[5:]).sum()
        den[2:5] = np.maximum(den[2:5], 1e-3 * np.abs(fr[0]).sum())
        e = np.abs(fg_ - fr).sum(axis=1) / den
        assert e.max() < TOL, e
    N1s = [b["n1"] + 6 for b in blocks]
    g = np.concatenate([f[:, :, :, :n].reshape(3, -1) for f, n in zip(fg, N1s)], axis=1)
    r = np.concatenate([f[:, :, :, :n].reshape(3, -1) for f, n in zip(fo, N1s)], axis=1)
    # the face field against its own scale (its x3 component of the box is
    # generated at level interfaces by cancellation, as B^3 above)
    assert np.abs(g - r).sum(axis=1).max() / np.abs(r).sum() < TOL


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-13), ("mixed", 1e-6)])
@pytest.mark.parametrize("which", ["torus2_weno5", "box"])
def test_mesh_face_divergence_and_interfaces(kh, orc, OM, which, precision, bar):
    import test_oracle_mesh_facect as T
    base, blocks, cfgs, Ps, fs = _case(which, precision)
    M = OM(base, blocks, inputs.block_cfg)
    Pf = [P.copy() for P in Ps]
    M.fill_ghosts(Pf)
    Us = [orc.prim_to_cons(c, P) for c, P in zip(cfgs, Pf)]
    dt = 0.5 * min(orc.cfl_dt(c, P) for c, P in zip(cfgs, Pf))
    m0 = T._interface_mismatch(M, fs)
    d0 = [orc.face_divb(c, f, field=True)[2] for c, f in zip(cfgs, fs)]
    _, _, _, fg, _ = _gpu(kh, base, blocks, Ps, Us, fs, 3, dt)
    fg = [np.ascontiguousarray(f) for f in fg]
    scale = max(np.abs(f).max() for f in fs)
    for b, (c, f) in enumerate(zip(cfgs, fg)):
        dx = min((c[k][1] - c[k][0]) / c[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3")))
        d1 = orc.face_divb(c, f, field=True)[2]
        assert np.abs(d1 - d0[b]).max() < 1e-12 * scale / dx, b
    m1 = T._interface_mismatch(M, fg)
    assert np.abs(m1 - m0).max() < bar * scale


def test_mesh_face_ct_graph_replay_bitwise(kh, orc, OM):
    base, blocks, cfgs, Ps, fs = _case("torus2_weno5")
    M = OM(base, blocks, inputs.block_cfg)
    Pf = [P.copy() for P in Ps]
    M.fill_ghosts(Pf)
    Us = [orc.prim_to_cons(c, P) for c, P in zip(cfgs, Pf)]
    dt = 0.5 * min(orc.cfl_dt(c, P) for c, P in zip(cfgs, Pf))
    a = _gpu(kh, base, blocks, Ps, Us, fs, 2, dt, graph=False)
    b = _gpu(kh, base, blocks, Ps, Us, fs, 2, dt, graph=True)
    for x, y in zip(a[1] + a[2] + a[3], b[1] + b[2] + b[3]):
        assert np.array_equal(x, y)
