"""kh_divb_noalloc: the divB reduction for callers that cannot call cudaMalloc
(and so cannot create a context). Its result must equal the context-based
kh_divb on the same field, call after call, with its scratch living in a
static device array shared by all calls. Collected last on purpose: a
failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _case(kind):
    if kind == "minkowski3d":
        cfg = inputs.linear_mode_cfg(8, ndim=3)
        cfg.update(n1=20, n2=16, n3=12)
        P = inputs.random_prims(cfg, seed=21, b_scale=(1.0, 1.0, 1.0))
    else:
        cfg = inputs.torus_cfg(40, 24, 1, r_out=60.0)
        P = inputs.random_prims(cfg, seed=22, b_scale=(1.0, 1.0, 1.0))
    return cfg, P


def _gdet(cfg, ctx):
    """sqrt(-g) at cell centres in the [n2s][n1s] layout (1 in Minkowski; the
    Kerr-Schild closed form of the input generator otherwise)."""
    torch = ctx.torch
    g = np.ones((ctx.n2s, ctx.n1s))
    if cfg["coords"] != "minkowski":
        x1 = inputs.centers(cfg, 0)
        x2 = inputs.centers(cfg, 1)
        X2, X1 = np.meshgrid(x2, x1, indexing="ij")
        g[:, : x1.size] = inputs.gdet_native(cfg, X1, X2)
    return torch.from_numpy(g).to(ctx.device)


def _both(kind):
    from paper_2408_01361_gb300 import kh

    cfg, P = _case(kind)
    ctx = kh.Context(cfg)
    PB = ctx.to_device(P)
    _, B = ctx.split(PB)
    ref_max, ref_l1 = ctx.divb(B)
    gdet = _gdet(cfg, ctx)
    out = ctx.torch.full((2,), -1.0, dtype=ctx.torch.float64, device=ctx.device)
    dx = [(cfg[a][1] - cfg[a][0]) / cfg[n] for a, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3"))]
    kh.divb_noalloc(B, gdet, cfg["n1"], cfg["n2"], cfg["n3"], ctx.n1s, ctx.n2s, dx, out)
    ctx.torch.cuda.synchronize()
    got = out.cpu().numpy()
    return (ref_max, ref_l1), got, (ctx, B, gdet, out, cfg, dx)


@pytest.mark.parametrize("order", [("minkowski3d", "fmks2d", "minkowski3d")])
def test_noalloc_matches_context_divb(order):
    for kind in order:
        (ref_max, ref_l1), got, _ = _both(kind)
        assert ref_max > 0 and ref_l1 > 0
        # the 3-D Minkowski field uses gdet = 1 exactly; the FMKS one uses the
        # generator's closed-form sqrt(-g), equal to the library's to ~1e-15
        assert abs(got[0] - ref_max) <= TOL * ref_max, (kind, got, ref_max)
        assert abs(got[1] - ref_l1) <= TOL * ref_l1, (kind, got, ref_l1)


def test_noalloc_repeat_call_allocates_nothing():
    import torch

    (ref_max, ref_l1), got, (ctx, B, gdet, out, cfg, dx) = _both("minkowski3d")
    from paper_2408_01361_gb300 import kh

    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        out.fill_(-1.0)
        kh.divb_noalloc(B, gdet, cfg["n1"], cfg["n2"], cfg["n3"], ctx.n1s, ctx.n2s, dx, out)
        torch.cuda.synchronize()
        v = out.cpu().numpy()
        assert abs(v[0] - ref_max) <= TOL * ref_max and abs(v[1] - ref_l1) <= TOL * ref_l1
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_oversize_grid():
    from paper_2408_01361_gb300 import kh

    import torch

    t = torch.zeros(16, dtype=torch.float64, device="cuda:0")
    with pytest.raises(kh.KHError, match="KH_EINVAL"):
        # (n2 - 1) * (n3 - 1) = 300 * 300 rows > KH_DIVB_NOALLOC_MAX_ROWS; rejected before any launch
        kh.divb_noalloc(t, t, 8, 301, 301, 16, 307, (1.0, 1.0, 1.0), t)


def test_noalloc_accepts_the_largest_grid():
    """(n2 - 1) (n3 - 1) = 256 x 256 = KH_DIVB_NOALLOC_MAX_ROWS rows: the last
    scratch slot is used, and the result still equals kh_divb's."""
    from paper_2408_01361_gb300 import kh

    cfg = inputs.linear_mode_cfg(8, ndim=3)
    cfg.update(n1=4, n2=257, n3=257)
    P = inputs.random_prims(cfg, seed=23, b_scale=(1.0, 1.0, 1.0))
    ctx = kh.Context(cfg)
    PB = ctx.to_device(P)
    _, B = ctx.split(PB)
    ref_max, ref_l1 = ctx.divb(B)
    gdet = _gdet(cfg, ctx)
    out = ctx.torch.full((2,), -1.0, dtype=ctx.torch.float64, device=ctx.device)
    dx = [(cfg[a][1] - cfg[a][0]) / cfg[n] for a, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3"))]
    assert (cfg["n2"] - 1) * (cfg["n3"] - 1) == 65536
    kh.divb_noalloc(B, gdet, cfg["n1"], cfg["n2"], cfg["n3"], ctx.n1s, ctx.n2s, dx, out)
    ctx.torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert abs(got[0] - ref_max) <= TOL * ref_max and abs(got[1] - ref_l1) <= TOL * ref_l1, (got, ref_max, ref_l1)


def test_noalloc_rejects_host_memory():
    """The arrays must be memory of the current device (the scratch address is
    that device's): a host array is refused before any launch."""
    from paper_2408_01361_gb300 import kh

    import torch

    d = torch.zeros(16, dtype=torch.float64, device="cuda:0")
    h = torch.zeros(4096, dtype=torch.float64)
    with pytest.raises(kh.KHError, match="KH_EINVAL"):
        kh.divb_noalloc(h, d, 4, 4, 1, 16, 10, (1.0, 1.0, 1.0), d)
