"""The refined mesh's mixed update with TMA-staged tiles (3-D, Flux-CT,
Noble-2D, every block 16 or 32 zones wide): a 3-D two-level torus whose
blocks have both widths and rows that are not a multiple of the tile's (16
rows per tile on the 16-wide blocks, 8 on the 32-wide ones). The staged update
must give the same bits as the update that loads its inputs itself (the same
per-zone arithmetic, its roundings fixed where a compiler could fuse them
differently), with and without graph replay and when the step is handed
another U array (its tensor maps rebuilt), and stay within the mixed path's
error of the oracle's mesh."""
import numpy as np
import pytest
import torch

from gpu_helpers import elem_err
from mesh_cases import blk, torus_states
from paper_2408_01361_gb300 import inputs
from test_gpu_mesh import _flat, _oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


@pytest.fixture(scope="module")
def OM():
    from oracle.mesh import OracleMesh
    return OracleMesh


def _layout():
    """Level-0 polar caps (32 wide, 6 rows: one ragged tile of 8 rows) and a
    level-1 band (two 16-wide blocks of 24 rows: a full and a ragged tile of
    16; two 32-wide blocks of 24 rows: three tiles of 8)."""
    base = inputs.torus_cfg(32, 24, 8, r_out=60.0, recon="weno5")
    blocks = [blk(0, 0, 0, 0, 32, 6, 8), blk(0, 0, 18, 0, 32, 6, 8),
              blk(1, 0, 12, 0, 16, 24, 16), blk(1, 16, 12, 0, 16, 24, 16),
              blk(1, 32, 12, 0, 32, 24, 8), blk(1, 32, 12, 8, 32, 24, 8)]
    return base, blocks


@pytest.fixture(scope="module")
def case():
    base, blocks = _layout()
    return base, blocks, torus_states(base, blocks)


def _run(kh, base, blocks, Ps, U0, dt, nsteps, staged, graph=False, swap_u=False):
    m = kh.Mesh(dict(base, precision="mixed"), blocks)
    assert m.set_staged_update(staged) == staged
    m.set_graph(graph)
    P, B = m.to_device(Ps)
    U = m.cons_to_device(U0)
    n0 = m.launches()
    for s in range(nsteps):
        if swap_u and s == nsteps // 2:
            U = U.clone()  # another array: the staged update's U^n maps are rebuilt
        m.step(U, P, B, dt)
    torch.cuda.synchronize()
    return m.cons_to_host(U), m.to_host(P, B), m.launches() - n0


def test_staged_update_selection(kh, case):
    base, blocks, Ps = case
    assert kh.Mesh(dict(base, precision="mixed"), blocks).set_staged_update(True)
    # does not qualify: FP64, face-centred CT, a 2-D mesh, a block of another width
    assert not kh.Mesh(base, blocks).set_staged_update(True)
    assert not kh.Mesh(dict(base, precision="mixed", bfield="face"), blocks).set_staged_update(True)
    odd = [dict(b) for b in blocks[:2]] + [blk(1, 0, 12, 0, 24, 24, 16), blk(1, 24, 12, 0, 8, 24, 16)] + blocks[4:]
    assert not kh.Mesh(dict(base, precision="mixed"), odd).set_staged_update(True)


def test_staged_update_bitwise(kh, orc, OM, case):
    base, blocks, Ps = case
    U0, dt, _, _, _ = _oracle_run(orc, OM, base, blocks, Ps, 0)
    Us, Ps_, ns = _run(kh, base, blocks, Ps, U0, dt, 4, True)
    Uo, Po, no = _run(kh, base, blocks, Ps, U0, dt, 4, False)
    # one launch per block width and stage instead of one per stage
    assert ns - no == 4 * 2
    for a, b in zip(Us + Ps_, Uo + Po):
        assert np.array_equal(a, b)
    Ug, Pg, _ = _run(kh, base, blocks, Ps, U0, dt, 4, True, graph=True)
    Uw, Pw, _ = _run(kh, base, blocks, Ps, U0, dt, 4, True, swap_u=True)
    for a, b, c in zip(Us + Ps_, Ug + Pg, Uw + Pw):
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_staged_update_vs_oracle(kh, orc, OM, case):
    base, blocks, Ps = case
    U0, dt, Uo, Po, hist = _oracle_run(orc, OM, base, blocks, Ps, 1)
    Ug, Pg, _ = _run(kh, base, blocks, Ps, U0, dt, 1, True)
    a, r = _flat(base, blocks, Ug), _flat(base, blocks, Uo)
    pa, pr = _flat(base, blocks, Pg), _flat(base, blocks, Po)
    mass, nz = np.abs(r[0]).sum(), r[0].size
    eu, ep = elem_err(a, r), elem_err(pa, pr)
    l1u = [np.abs(a[v] - r[v]).sum() / max(np.abs(r[v]).sum(), 1e-3 * mass) for v in range(8)]
    l1p = [np.abs(pa[v] - pr[v]).sum() / max(np.abs(pr[v]).sum(), 1e-2 * nz if v in (2, 3, 4) else 0.0)
           for v in range(8)]
    print("staged mesh vs oracle: U l1", np.array(l1u), "P l1", np.array(l1p), "eU", eu, "eP", ep)
    # within 5x of the error measured on GB300 when the bounds were set (floor 1e-9)
    meas = dict(
        U=[3.0e-10, 8.5e-9, 3.7e-9, 1.1e-6, 3.7e-9, 3.1e-11, 9.5e-12, 1.4e-10],
        P=[4.2e-10, 3.3e-8, 1.9e-6, 4.4e-8, 1.7e-6, 5.2e-10, 2.5e-10, 1.1e-6],
        eU=[1.3e-6, 2.5e-5, 1.7e-4, 2.7e-4, 2.2e-4, 2.5e-7, 2.7e-7, 2.5e-3],
        eP=[7.0e-7, 2.0e-6, 2.5e-2, 2.3e-3, 5.9e-2, 1.3e-6, 3.6e-7, 6.3e-4])
    bound = {key: np.maximum(5.0 * np.array(val), 1e-9) for key, val in meas.items()}
    for v in range(8):
        assert l1u[v] < bound["U"][v] and l1p[v] < bound["P"][v], v
        assert eu[v] < bound["eU"][v] and ep[v] < bound["eP"][v], v
