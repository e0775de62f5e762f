"""Restart: N + M steps in one run equal N steps, the state (U, P, B) saved
to the host with torch.save, loaded into a fresh context, and M more steps --
bit for bit. The arrays the caller holds are the whole state of a run:
nothing the library keeps between steps (the FP32 shadow of the mixed path,
captured graphs, autotuned launch settings, the staged update's tensor maps)
changes what the next step computes. Single grid (FP64 and mixed, the torus
with WENO5) and the refined mesh (mixed, the staged update; FP64)."""
import io

import numpy as np
import pytest
import torch

from mesh_cases import blk, torus_states
from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu

N, M = 3, 2


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


def _through_host(tensors):
    """Device tensors -> bytes (torch.save) -> new device tensors."""
    buf = io.BytesIO()
    torch.save([t.detach().cpu() for t in tensors], buf)
    buf.seek(0)
    dev = tensors[0].device
    return [t.to(dev) for t in torch.load(buf)]


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("graph", [False, True])
def test_restart_single_grid(kh, precision, graph):
    cfg = dict(inputs.torus_cfg(48, 32, 16, r_out=60.0), precision=precision)
    P0 = inputs.torus_state(cfg, seed=2)

    def start():
        ctx = kh.Context(cfg)
        ctx.set_graph(graph)
        PB = ctx.to_device(P0)
        P, B = ctx.split(PB)
        U = ctx.empty(8)
        ctx.prim_to_cons(P, B, U)
        return ctx, U, PB

    ctx, U, PB = start()
    P, B = ctx.split(PB)
    dt = 0.5 * ctx.cfl_dt(P, B)
    for _ in range(N + M):
        ctx.step(U, P, B, dt)
    whole = [U.clone(), PB.clone()]

    ctx, U, PB = start()
    P, B = ctx.split(PB)
    for _ in range(N):
        ctx.step(U, P, B, dt)
    U2, PB2 = _through_host([U, PB])
    del ctx, U, PB, P, B
    ctx2 = kh.Context(cfg)
    ctx2.set_graph(graph)
    P2, B2 = ctx2.split(PB2)
    for _ in range(M):
        ctx2.step(U2, P2, B2, dt)
    torch.cuda.synchronize()
    assert _same(whole, [U2, PB2])


def _mesh_layout():
    """3-D two-level torus with 16- and 32-wide blocks (the staged update)."""
    base = inputs.torus_cfg(32, 24, 8, r_out=60.0, recon="weno5")
    blocks = [blk(0, 0, 0, 0, 32, 6, 8), blk(0, 0, 18, 0, 32, 6, 8),
              blk(1, 0, 12, 0, 16, 24, 16), blk(1, 16, 12, 0, 16, 24, 16),
              blk(1, 32, 12, 0, 32, 24, 8), blk(1, 32, 12, 8, 32, 24, 8)]
    return base, blocks


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_restart_mesh(kh, precision):
    base, blocks = _mesh_layout()
    cfg = dict(base, precision=precision)
    Ps = torus_states(base, blocks)

    def start():
        m = kh.Mesh(cfg, blocks)
        P, B = m.to_device(Ps)
        U = m.empty(8)
        m.prim_to_cons(P, B, U)
        return m, U, P, B

    m, U, P, B = start()
    dt = 0.5 * m.cfl_dt(P, B)
    for _ in range(N + M):
        m.step(U, P, B, dt)
    whole = [U.clone(), P.clone(), B.clone()]
    m.close()

    m, U, P, B = start()
    for _ in range(N):
        m.step(U, P, B, dt)
    U2, P2, B2 = _through_host([U, P, B])
    m.close()
    m2 = kh.Mesh(cfg, blocks)
    for _ in range(M):
        m2.step(U2, P2, B2, dt)
    torch.cuda.synchronize()
    assert _same(whole, [U2, P2, B2])
    m2.close()
    assert np.isfinite(whole[0].cpu().numpy()).all()
