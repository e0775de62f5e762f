"""Runge-Kutta integrators (RK1, RK2, SSPRK(5,4)) on the refined mesh: every
stage's input ghost-filled across blocks, stage bases formed over the whole
arena. FP64 against the oracle mesh's Runge-Kutta step (the oracle's own
table and stage routine) at the FP64 bars; mixed with the staged (TMA)
update bitwise equal to the update that loads its inputs itself -- the
later stages read the stage base through their own tensor maps -- and
within 5x of its measured error against the oracle."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_fp64_parity, elem_err
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


def _oracle_rk(orc, OM, base, blocks, Ps, integrator, nsteps):
    M = OM(base, blocks, inputs.block_cfg)
    Us = [orc.prim_to_cons(inputs.block_cfg(base, b), P) for b, P in zip(blocks, Ps)]
    dt = 0.5 * _mesh_cfl(orc, M, base, blocks, Ps)
    U0 = [u.copy() for u in Us]
    Uc, Pc, hist = Us, Ps, []
    for _ in range(nsteps):
        Uc, Pc, dtn, st = M.step_rk(Uc, Pc, dt, integrator)
        hist.append((dtn, st))
    return U0, dt, Uc, Pc, hist


def _gpu_rk(kh, base, blocks, Ps, U0, dt, nsteps, staged=True, **over):
    m = kh.Mesh(dict(base, **over), blocks)
    m.set_staged_update(staged)
    P, B = m.to_device(Ps)
    U = m.cons_to_device(U0)
    out = []
    for _ in range(nsteps):
        out.append(m.step(U, P, B, dt))
    torch.cuda.synchronize()
    return m.cons_to_host(U), m.to_host(P, B), out


@pytest.mark.parametrize("integrator", ["rk1", "rk2", "ssprk54"])
@pytest.mark.parametrize("which", ["box_weno5", "torus2_weno5"])
def test_mesh_rk_fp64_parity(kh, orc, OM, which, integrator):
    base, blocks, Ps = _case(which)
    base = dict(base, integrator=integrator)
    U0, dt, Uo, Po, hist = _oracle_rk(orc, OM, base, blocks, Ps, integrator, 2)
    Ug, Pg, out = _gpu_rk(kh, base, blocks, Ps, U0, dt, 2)
    assert_fp64_parity(_flat(base, blocks, Ug), _flat(base, blocks, Uo), "U")
    assert_fp64_parity(_flat(base, blocks, Pg), _flat(base, blocks, Po), "P")
    assert abs(out[-1][0] - hist[-1][0]) < 1e-10 * hist[-1][0]
    assert [o[1] for o in out] == [h[1][0] for h in hist]


# element-wise error of one mixed step against the oracle, measured on GB300
MIXED_MEAS = {
    "ssprk54": dict(eU=[2.3e-7, 2.8e-6, 2.0e-6, 2.2e-4, 2.2e-6, 1.1e-7, 1.4e-7, 3.9e-4],
                    eP=[1.4e-7, 5.5e-7, 2.4e-2, 1.3e-4, 5.7e-2, 6.1e-7, 1.8e-7, 9.8e-5]),
}


@pytest.mark.parametrize("integrator", ["rk2", "ssprk54"])
def test_mesh_rk_mixed_staged(kh, orc, OM, integrator):
    base, blocks = _layout()
    base = dict(base, integrator=integrator)
    Ps = torus_states(base, blocks)
    U0, dt, Uo, Po, _ = _oracle_rk(orc, OM, base, blocks, Ps, integrator, 1)
    Us, Pss, _ = _gpu_rk(kh, base, blocks, Ps, U0, dt, 2, True, precision="mixed")
    Ul, Pl, _ = _gpu_rk(kh, base, blocks, Ps, U0, dt, 2, False, precision="mixed")
    for a, b in zip(Us + Pss, Ul + Pl):
        assert np.array_equal(a, b)
    Ug, Pg, _ = _gpu_rk(kh, base, blocks, Ps, U0, dt, 1, True, precision="mixed")
    a, r = _flat(base, blocks, Ug), _flat(base, blocks, Uo)
    pa, pr = _flat(base, blocks, Pg), _flat(base, blocks, Po)
    mass, nz = np.abs(r[0]).sum(), r[0].size
    # the single-grid mixed integrators' bars: relative L1 per variable,
    # momenta and velocities against the mass scale near the equilibrium
    for v in range(8):
        tol = 2e-3 if v in (2, 3, 4) else 1e-4
        assert np.abs(a[v] - r[v]).sum() / max(np.abs(r[v]).sum(), 1e-3 * mass) < tol, ("U", v)
        assert np.abs(pa[v] - pr[v]).sum() / max(np.abs(pr[v]).sum(), 1e-2 * nz if v in (2, 3, 4) else 0.0) < tol, v
    eu, ep = elem_err(a, r), elem_err(pa, pr)
    print(integrator, "mixed RK mesh vs oracle: eU", eu, "eP", ep)
    if integrator in MIXED_MEAS:
        meas = MIXED_MEAS[integrator]
        for v in range(8):  # within 5x of the measured error (floor 1e-9)
            assert eu[v] < max(5.0 * meas["eU"][v], 1e-9) and ep[v] < max(5.0 * meas["eP"][v], 1e-9), v
    else:
        # RK2's first stage is a full forward-Euler step: at the polar cap one
        # zone more fails its inversion than in FP64 (242 against 241), and
        # the zones its fixup and the second stage touch differ by O(1) of
        # their small components; measured 19 zones of 27,648 above 1e-3
        eb = np.abs(a - r) / np.maximum(np.abs(r), 1e-3 * np.abs(r).max(axis=1, keepdims=True))
        assert int((eb.max(axis=0) > 1e-3).sum()) <= 5 * 19
