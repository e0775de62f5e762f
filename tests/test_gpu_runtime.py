"""Runtime features of the step: CUDA-graph replay, launch configuration and
the autotuner leave the arithmetic unchanged (bitwise), on both precisions."""
import numpy as np
import pytest

from gpu_helpers import GpuRun
from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


def _run(kh, cfg, P, nsteps, graph=False, launch=None, autotune=False):
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P)
    dt = 0.5 * ctx.cfl_dt(g.P, g.B)
    if launch:
        ctx.set_launch(*launch)
    if autotune:
        tf, tu = ctx.autotune(g.U, g.P, g.B, dt)
        assert tf in (64, 128, 256) and tu in (64, 128, 256)
        assert ctx.get_launch() == (tf, tu)
    ctx.set_graph(graph)
    dts = []
    for _ in range(nsteps):
        d, _ = ctx.step(g.U, g.P, g.B, dt)
        dts.append(d)
        dt = 0.5 * d
    return g.host(), dts


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_is_bitwise(kh, precision):
    cfg = inputs.torus_cfg(40, 24, 12, r_out=60.0)
    cfg["precision"] = precision
    P = inputs.torus_state(cfg, seed=2)
    (U0, P0), d0 = _run(kh, cfg, P, 4)
    (U1, P1), d1 = _run(kh, cfg, P, 4, graph=True)
    assert np.array_equal(U0, U1) and np.array_equal(P0, P1) and d0 == d1


def test_launch_config_and_autotune_are_bitwise(kh):
    cfg = inputs.torus_cfg(40, 24, 12, r_out=60.0)
    cfg["precision"] = "mixed"
    P = inputs.torus_state(cfg, seed=2)
    (U0, P0), _ = _run(kh, cfg, P, 2)
    (U1, P1), _ = _run(kh, cfg, P, 2, launch=(64, 256))
    (U2, P2), _ = _run(kh, cfg, P, 2, autotune=True, graph=True)
    for A, B in ((U0, U1), (P0, P1), (U0, U2), (P0, P2)):
        assert np.array_equal(A, B)


def test_graph_follows_new_pointers(kh):
    """Two states (different tensors) stepped alternately with graph replay
    match the same sequence without graphs: a new pointer triple re-captures
    instead of replaying stale pointers."""
    cfg = inputs.linear_mode_cfg(12, ndim=3)
    P = inputs.random_prims(cfg, seed=3, rho_range=(0.5, 1), u_range=(0.3, 1), ut_scale=(0.2, 0.2, 0.2),
                            b_scale=(0.2, 0.2, 0.2))
    out = []
    for graph in (True, False):
        ctx = kh.Context(cfg)
        ctx.set_graph(graph)
        a = GpuRun(ctx, cfg, P)
        b = GpuRun(ctx, cfg, P)
        ctx.step(a.U, a.P, a.B, 1e-3)
        ctx.step(b.U, b.P, b.B, 1e-3)
        ctx.step(b.U, b.P, b.B, 2e-3)
        ctx.step(a.U, a.P, a.B, 1e-3)
        out.append((a.host(), b.host()))
    (ga, gb), (na, nb) = out
    assert np.array_equal(ga[0], na[0]) and np.array_equal(gb[0], nb[0])
    assert np.array_equal(ga[1], na[1]) and np.array_equal(gb[1], nb[1])
    assert not np.array_equal(ga[0], gb[0])


def test_pack_unpack_state_round_trip(kh):
    """kh_pack_state writes the interior of U, P, B in the compact order
    [16][n3][n2][n1]; kh_unpack_state puts it back (interior cells only);
    a step from the unpacked state equals a step from the original."""
    cfg = inputs.torus_cfg(40, 24, 10, r_out=60.0)
    P = inputs.torus_state(cfg, seed=2)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P)
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
    buf = ctx.torch.empty(16 * nz, dtype=ctx.torch.float64, device=ctx.device)
    ctx.pack_state(g.U, g.P, g.B, buf)
    Uh, Ph = g.host()
    sl = (slice(None),) + inputs.interior(cfg)
    packed = buf.cpu().numpy().reshape(16, cfg["n3"], cfg["n2"], cfg["n1"])
    assert np.array_equal(packed[:8], Uh[sl]) and np.array_equal(packed[8:], Ph[sl])
    U2 = ctx.empty(8)
    PB2 = ctx.empty(8)
    P2, B2 = ctx.split(PB2)
    ctx.unpack_state(buf, U2, P2, B2)
    dt = 0.5 * ctx.cfl_dt(g.P, g.B)
    ctx.step(g.U, g.P, g.B, dt)
    ctx.step(U2, P2, B2, dt)
    N1 = P.shape[3]
    assert np.array_equal(ctx.to_host(U2, N1)[sl], ctx.to_host(g.U, N1)[sl])
    assert np.array_equal(ctx.to_host(PB2, N1)[sl], ctx.to_host(g.PB, N1)[sl])


def test_pack_unpack_state_through_pinned_host_memory(kh):
    """The compact state read and written straight from page-locked host
    memory (the kernels address it over the host link; no separate copy):
    identical to the device-buffer path."""
    cfg = inputs.torus_cfg(40, 24, 10, r_out=60.0)
    P = inputs.torus_state(cfg, seed=2)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P)
    torch = ctx.torch
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
    dev = torch.empty(16 * nz, dtype=torch.float64, device=ctx.device)
    host = torch.full((16 * nz,), -1.0, dtype=torch.float64, pin_memory=True)
    ctx.pack_state(g.U, g.P, g.B, dev)
    ctx.pack_state(g.U, g.P, g.B, host)
    torch.cuda.synchronize()
    assert np.array_equal(host.numpy(), dev.cpu().numpy())
    host.mul_(1.0 + 1e-3)  # a different state, written by the host
    U2, PB2 = ctx.empty(8), ctx.empty(8)
    P2, B2 = ctx.split(PB2)
    ctx.unpack_state(host, U2, P2, B2)
    U3, PB3 = ctx.empty(8), ctx.empty(8)
    P3, B3 = ctx.split(PB3)
    ctx.unpack_state(host.to(ctx.device), U3, P3, B3)
    torch.cuda.synchronize()
    assert torch.equal(U2, U3) and torch.equal(PB2, PB3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_profiled_graph_replay(kh, precision):
    """kh_profile with kh_set_graph: the captured step holds the group events,
    so every replay times every group of both stages; the arithmetic is the
    unprofiled step's, bit for bit, and switching profiling off again
    re-captures a step without the events."""
    cfg = inputs.torus_cfg(40, 24, 12, r_out=60.0)
    cfg["precision"] = precision
    P = inputs.torus_state(cfg, seed=2)
    (U0, P0), d0 = _run(kh, cfg, P, 4)
    ctx = kh.Context(cfg)
    g = GpuRun(ctx, cfg, P)
    dt = 0.5 * ctx.cfl_dt(g.P, g.B)
    ctx.set_graph(True)
    ctx.profile(True)
    dts = []
    for q in range(4):
        if q == 2:
            ctx.profile(False)  # the events go, the graph is captured again
        d, _ = ctx.step(g.U, g.P, g.B, dt)
        if q == 1:
            prof = ctx.profile_read()
        dts.append(d)
        dt = 0.5 * d
    U1, P1 = g.host()
    assert np.array_equal(U0, U1) and np.array_equal(P0, P1) and d0 == dts
    for name in ("flux_x1", "flux_x2", "flux_x3", "update", "cfl"):
        ms, n = prof[name]
        assert n == (2 if name == "cfl" else 4) and ms > 0.0, (name, prof[name])
