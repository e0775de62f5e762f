"""The bounded device wait of the mixed path's face kernels (the paper's
"Algorithm" section detects and repairs failures instead of stopping; here a
TMA tile that does not arrive in time is reported, not waited for forever).

Each face CTA stages its tile by one TMA tensor copy and polls the copy's
mbarrier a bounded number of times (kh_set_wait_limit). With the limit at 0
every CTA gives up before its first poll: it counts a timeout, keeps waiting
until its copy has landed, and leaves; kh_step then returns KH_ETIMEOUT. The
wait that runs out is a real wait on a real copy; nothing faults or hangs.
With the limit restored, the same context steps again and matches a context
that never timed out bit for bit."""
import numpy as np
import pytest

from gpu_helpers import GpuRun
from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu

KH_ETIMEOUT = -4


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


@pytest.mark.parametrize("graph", [False, True])
def test_tma_wait_timeout_is_reported_and_the_context_recovers(kh, orc, graph):
    cfg = inputs.torus_cfg(48, 32, 16, r_out=60.0)
    cfg["precision"] = "mixed"
    P = inputs.torus_state(cfg, seed=2)
    U = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    _, _, _, st = orc.step(cfg, U, P, dt)

    ctx = kh.Context(cfg)
    ctx.set_graph(graph)
    g = GpuRun(ctx, cfg, P, U=U)
    ctx.set_wait_limit(0)
    assert ctx.step_rc(g.U, g.P, g.B, dt) == KH_ETIMEOUT
    ctx.set_wait_limit()  # the default bound
    g = GpuRun(ctx, cfg, P, U=U)
    dtg, nfail = ctx.step(g.U, g.P, g.B, dt)
    assert nfail == st[0]
    Ug, Pg = g.host()

    ref = kh.Context(cfg)
    r = GpuRun(ref, cfg, P, U=U)
    dtr, _ = ref.step(r.U, r.P, r.B, dt)
    Ur, Pr = r.host()
    assert dtg == dtr
    assert np.array_equal(Ug, Ur) and np.array_equal(Pg, Pr)
