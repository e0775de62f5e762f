"""First-order flux correction on the refined mesh: each stage runs every
block's trial, fills the flags' ghost cells across blocks by the state's
ghost map and corrects the faces of the flagged zones of every block. FP64
against the oracle mesh's correction (its own trial, flag map and stage
routine) at the FP64 bars, with the predictor-corrector and with SSPRK(5,4);
mixed with the staged update bitwise equal to the own-loads update and
within the single-grid mixed bars of the oracle."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_fp64_parity
from mesh_cases import torus_states
from paper_2408_01361_gb300 import inputs
from test_gpu_mesh import _case, _flat, _mesh_cfl
from test_gpu_mesh_staged import _layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


@pytest.fixture(scope="module")
def OM():
    from oracle.mesh import OracleMesh
    return OracleMesh


def _oracle(orc, OM, base, blocks, Ps, nsteps, integrator="vl2"):
    M = OM(base, blocks, inputs.block_cfg)
    Us = [orc.prim_to_cons(inputs.block_cfg(base, b), P) for b, P in zip(blocks, Ps)]
    dt = 0.5 * _mesh_cfl(orc, M, base, blocks, Ps)
    U0 = [u.copy() for u in Us]
    Uc, Pc, hist = Us, Ps, []
    for _ in range(nsteps):
        if integrator == "vl2":
            Uc, Pc, dtn, st = M.step(Uc, Pc, dt)
        else:
            Uc, Pc, dtn, st = M.step_rk(Uc, Pc, dt, integrator)
        hist.append((dtn, st))
    return U0, dt, Uc, Pc, hist


def _gpu(kh, base, blocks, Ps, U0, dt, nsteps, staged=True):
    m = kh.Mesh(base, blocks)
    m.set_staged_update(staged)
    P, B = m.to_device(Ps)
    U = m.cons_to_device(U0)
    out, nfofc = [], 0
    for _ in range(nsteps):
        out.append(m.step(U, P, B, dt))
        nfofc += m.stats().nfofc
    torch.cuda.synchronize()
    return m.cons_to_host(U), m.to_host(P, B), out, nfofc


@pytest.mark.parametrize("integrator", ["vl2", "ssprk54"])
@pytest.mark.parametrize("which", ["torus2_mc", "torus3d"])
def test_mesh_fofc_fp64_parity(kh, orc, OM, which, integrator):
    if which == "torus3d":
        base, blocks = _layout()
        Ps = torus_states(base, blocks)
    else:
        base, blocks, Ps = _case(which)
    base = dict(base, fofc=True, integrator=integrator)
    U0, dt, Uo, Po, hist = _oracle(orc, OM, base, blocks, Ps, 2, integrator)
    Ug, Pg, out, nfofc = _gpu(kh, base, blocks, Ps, U0, dt, 2)
    assert nfofc > 0
    assert [o[1] for o in out] == [h[1][0] for h in hist]
    assert_fp64_parity(_flat(base, blocks, Ug), _flat(base, blocks, Uo), "U")
    assert_fp64_parity(_flat(base, blocks, Pg), _flat(base, blocks, Po), "P")
    assert abs(out[-1][0] - hist[-1][0]) < 1e-10 * hist[-1][0]


def test_mesh_fofc_mixed(kh, orc, OM):
    base, blocks = _layout()
    base = dict(base, fofc=True)
    Ps = torus_states(base, blocks)
    U0, dt, Uo, Po, _ = _oracle(orc, OM, base, blocks, Ps, 1)
    mb = dict(base, precision="mixed")
    Us, Pss, _, nf = _gpu(kh, mb, blocks, Ps, U0, dt, 2, True)
    Ul, Pl, _, _ = _gpu(kh, mb, blocks, Ps, U0, dt, 2, False)
    assert nf > 0
    for a, b in zip(Us + Pss, Ul + Pl):
        assert np.array_equal(a, b)
    Ug, Pg, _, _ = _gpu(kh, mb, blocks, Ps, U0, dt, 1)
    a, r = _flat(base, blocks, Ug), _flat(base, blocks, Uo)
    pa, pr = _flat(base, blocks, Pg), _flat(base, blocks, Po)
    mass, nz = np.abs(r[0]).sum(), r[0].size
    for v in range(8):  # the single-grid mixed bars
        tol = 2e-3 if v in (2, 3, 4) else 1e-4
        ue = np.abs(a[v] - r[v]).sum() / max(np.abs(r[v]).sum(), 1e-3 * mass)
        pe = np.abs(pa[v] - pr[v]).sum() / max(np.abs(pr[v]).sum(), 1e-2 * nz if v in (2, 3, 4) else 0.0)
        print("mixed mesh fofc vs oracle", v, ue, pe)
        assert ue < tol and pe < tol, v
