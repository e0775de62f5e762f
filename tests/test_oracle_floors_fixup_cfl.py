"""Pins for the oracle's floors, fixup and CFL time step (the paper's
"Algorithm" section: floors after every inversion, failed zones repaired from
their neighbours, the step size from the fastest signal speed; the floor
values and the neighbour rule are the readings of the floors and fixup
paragraphs listed with the other readings of the paper).

Every expected value below is a closed form fixed by the definitions (the
floor formulas on a state whose b^2 and Lorentz factor are known in closed
form; the neighbour mean of quadratic data; the sound and magnetosonic speeds
of a uniform state at rest or boosted), or a brute-force mean taken from the
inputs, never from the oracle's own output."""
import itertools

import numpy as np
import pytest

from paper_2408_01361_gb300 import inputs

GAM = 13.0 / 9.0


def _cfg(coords="ks", a=0.0, **floors):
    fl = dict(rho_min=1e-20, u_min=1e-20, bsq_rho_max=1e300, bsq_u_max=1e300, u_rho_max=1e300, gamma_max=1e300)
    fl.update(floors)
    return dict(coords=coords, n1=8, n2=8, n3=1, recon="mc", bc=["outflow"] * 6, a=a, gam=GAM,
                x1=(1.0, 20.0), x2=(0.1, 3.0), x3=(0.0, 6.283185307179586), cfl=0.9, floors=fl)


# Schwarzschild in Kerr-Schild coordinates (x1 = r, x2 = theta): the spatial
# metric is diag(1 + 2/r, r^2, r^2 sin^2 theta) and the lapse (1 + 2/r)^-1/2.
R0, TH0 = 10.0, np.pi / 3


def _ks_gij(r, th):
    return np.diag([1.0 + 2.0 / r, r * r, (r * np.sin(th)) ** 2])


def _ks_alpha2(r):
    return 1.0 / (1.0 + 2.0 / r)


def _state(rho, u, ut=(0.0, 0.0, 0.0), B=(0.0, 0.0, 0.0)):
    return np.array([rho, u, *ut, *B], dtype=np.float64)


def test_floors_leave_a_state_above_them_unchanged(orc):
    cfg = _cfg(rho_min=1e-4, u_min=1e-6, bsq_rho_max=100.0, bsq_u_max=5000.0, u_rho_max=100.0, gamma_max=50.0)
    P = _state(0.3, 0.02, (0.1, 0.01, -0.02), (0.01, 0.001, 0.002))
    Q, flag = orc.point_floors(cfg, R0, TH0, P)
    assert flag == 0 and np.array_equal(Q, P)


def test_density_floor_scales_as_r_to_minus_three_halves(orc):
    cfg = _cfg(rho_min=1e-4)
    Q, flag = orc.point_floors(cfg, R0, TH0, _state(1e-12, 1e-3))
    assert flag == 1
    assert Q[0] == pytest.approx(1e-4 * R0 ** -1.5, rel=1e-15)
    assert Q[1] == 1e-3 and np.array_equal(Q[2:], np.zeros(6))


def test_energy_floor_scales_as_r_to_minus_five_halves(orc):
    cfg = _cfg(u_min=1e-6)
    Q, flag = orc.point_floors(cfg, R0, TH0, _state(1.0, 1e-15))
    assert flag == 1
    assert Q[1] == pytest.approx(1e-6 * R0 ** -2.5, rel=1e-15)
    assert Q[0] == 1.0


def test_floors_take_the_radius_not_the_native_coordinate(orc):
    """MKS: r = exp(x1), so the floor at x1 = ln 10 is rho_min 10^-3/2."""
    cfg = _cfg(coords="mks", rho_min=1e-4, u_min=1e-6)
    cfg["x1"] = (0.0, 3.0)
    Q, flag = orc.point_floors(cfg, np.log(R0), 0.37, _state(1e-14, 1e-16))
    assert flag == 1
    assert Q[0] == pytest.approx(1e-4 * R0 ** -1.5, rel=1e-14)
    assert Q[1] == pytest.approx(1e-6 * R0 ** -2.5, rel=1e-14)


def test_minkowski_floors_are_constants(orc):
    cfg = _cfg(coords="minkowski", rho_min=3e-5, u_min=2e-7)
    cfg["x1"], cfg["x2"] = (0.0, 1.0), (0.0, 1.0)
    Q, flag = orc.point_floors(cfg, 0.7, 0.2, _state(1e-9, 1e-12))
    assert flag == 1 and Q[0] == 3e-5 and Q[1] == 2e-7


def test_magnetic_ceilings_hit_exactly_and_are_not_swapped(orc):
    """A fluid at rest in the normal frame has u_i = 0, so b^t = 0 and
    b^i = alpha B^i: b^2 = alpha^2 g_ij B^i B^j. rho and u are raised to
    b^2/100 and b^2/5000 (different limits, so a swap shows)."""
    cfg = _cfg(rho_min=1e-10, u_min=1e-12, bsq_rho_max=100.0, bsq_u_max=5000.0)
    B = np.array([0.07, 0.004, -0.003])
    bsq = _ks_alpha2(R0) * B @ _ks_gij(R0, TH0) @ B
    Q, flag = orc.point_floors(cfg, R0, TH0, _state(1e-7, 1e-9, (0, 0, 0), B))
    assert flag == 1
    assert Q[0] == pytest.approx(bsq / 100.0, rel=1e-14)
    assert Q[1] == pytest.approx(bsq / 5000.0, rel=1e-14)
    assert np.array_equal(Q[5:], B)


def test_temperature_ceiling(orc):
    cfg = _cfg(u_rho_max=100.0)
    Q, flag = orc.point_floors(cfg, R0, TH0, _state(1e-3, 1.0))
    assert flag == 2
    assert Q[1] == pytest.approx(0.1, rel=1e-15) and Q[0] == 1e-3


@pytest.mark.parametrize("spin", [0.0, 0.9375])
def test_lorentz_factor_ceiling_rescales_to_gamma_max_along_u(orc, spin):
    """gamma = sqrt(1 + g_ij u~^i u~^j) is brought to exactly gamma_max by a
    positive rescale of u~ (direction kept); rho, u and B are untouched."""
    cfg = _cfg(a=spin, gamma_max=50.0)
    if spin == 0.0:
        gij = _ks_gij(R0, TH0)
    else:
        gcov, _, _, _ = orc.metric_points(cfg, [R0], [TH0])
        gij = gcov[0, 1:, 1:]
    d = np.array([3.0, 0.05, 0.08])
    s = np.sqrt((200.0 ** 2 - 1.0) / (d @ gij @ d))
    P = _state(0.2, 0.01, tuple(s * d), (0.01, 0.0, 0.002))
    Q, flag = orc.point_floors(cfg, R0, TH0, P)
    assert flag == 4
    ut = Q[2:5]
    assert np.sqrt(1.0 + ut @ gij @ ut) == pytest.approx(50.0, rel=1e-13)
    ratio = ut / P[2:5]
    assert np.all(ratio > 0) and np.ptp(ratio) < 1e-15
    assert np.array_equal(Q[[0, 1, 5, 6, 7]], P[[0, 1, 5, 6, 7]])


# ---------------------------------------------------------------------------
# Fixup: a zone whose inversion fails takes the equal-weight mean of the
# non-failed interior zones of its 3x3x3 (3x3 in 2-D) neighbourhood.
# ---------------------------------------------------------------------------
COEF = np.array([[1.0, 0.01, 0.02],     # rho: a + b R^2 + c (i - i_f)
                 [0.5, 0.005, -0.01],   # u
                 [0.1, 0.002, 0.003],   # u~1
                 [-0.05, 0.001, 0.0],   # u~2
                 [0.02, -0.001, 0.001]])  # u~3


def _quad_state(cfg, centre):
    shp = inputs.shape(cfg)
    K, J, I = np.meshgrid(*[np.arange(n) for n in shp[1:]], indexing="ij")
    kf, jf, i_f = centre
    R2 = (I - i_f) ** 2 + (J - jf) ** 2 + ((K - kf) ** 2 if shp[1] > 1 else 0)
    P = np.zeros(shp)
    for v in range(5):
        P[v] = COEF[v, 0] + COEF[v, 1] * R2 + COEF[v, 2] * (I - i_f)
    P[5], P[6], P[7] = 0.3, -0.2, 0.1
    return P


def _fixup_run(orc, cfg, P0, failed):
    """One stage with cdt = 0 (U = U0 exactly) whose U0 is made unphysical
    (momenta x 50) at the `failed` cells."""
    P0 = orc.apply_bc(cfg, P0)
    U0 = orc.prim_to_cons(cfg, P0)
    for c in failed:
        U0[(slice(2, 5),) + c] *= 50.0
    _, pflag, _ = orc.cons_to_prim(cfg, U0, P0)
    for c in failed:
        assert pflag[c] != 0, c
    Uout, Pout = U0.copy(), P0.copy()
    _, st = orc.stage(cfg, U0, P0, 0.0, Uout, Pout)
    return P0, Uout, Pout, st


def _brute_mean(cfg, P0, c, failed):
    sl = inputs.interior(cfg)
    lo = [s.start for s in sl]
    hi = [s.stop for s in sl]
    offs = [(-1, 0, 1) if P0.shape[1] > 1 else (0,), (-1, 0, 1), (-1, 0, 1)]
    acc, n = np.zeros(5), 0
    for d in itertools.product(*offs):
        q = tuple(c[a] + d[a] for a in range(3))
        if q == c or q in failed or any(q[a] < lo[a] or q[a] >= hi[a] for a in range(3)):
            continue
        acc += P0[(slice(0, 5),) + q]
        n += 1
    return acc / n, n


def test_fixup_lone_zone_takes_the_26_neighbour_mean(orc):
    """Quadratic data a + b R^2 + c di: over the 26 neighbours R^2 averages
    54/26 and di cancels, so the repaired value is a + (27/13) b (6 face
    neighbours would give a + b, 27 cells a + 2b)."""
    cfg = inputs.linear_mode_cfg(8, ndim=3)
    c = (6, 6, 6)
    P0, Uout, Pout, st = _fixup_run(orc, cfg, _quad_state(cfg, c), [c])
    assert st == [1, 0, 0]
    want = COEF[:, 0] + COEF[:, 1] * 27.0 / 13.0
    np.testing.assert_allclose(Pout[(slice(0, 5),) + c], want, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Pout[(slice(5, 8),) + c], P0[(slice(5, 8),) + c], rtol=1e-14)
    # U is recomputed from the repaired primitives
    Ufix = orc.prim_to_cons(cfg, Pout)
    np.testing.assert_allclose(Uout[(slice(None),) + c], Ufix[(slice(None),) + c], rtol=1e-14, atol=1e-15)
    # every other zone keeps its inversion of U0 (= P0 to round-off)
    sl = (slice(None),) + inputs.interior(cfg)
    mask = np.ones(P0.shape[1:], bool)
    mask[c] = False
    d = np.abs(Pout[sl] - P0[sl])[:, mask[sl[1:]]]
    assert d.max() < 1e-13


def test_fixup_2d_lone_zone_takes_the_8_neighbour_mean(orc):
    cfg = inputs.linear_mode_cfg(8, ndim=2)
    c = (0, 6, 6)
    _, _, Pout, st = _fixup_run(orc, cfg, _quad_state(cfg, c), [c])
    assert st == [1, 0, 0]
    want = COEF[:, 0] + COEF[:, 1] * 12.0 / 8.0
    np.testing.assert_allclose(Pout[(slice(0, 5),) + c], want, rtol=1e-12, atol=1e-14)


def test_fixup_skips_failed_and_non_interior_neighbours(orc):
    """Two adjacent failed zones and one at the interior corner: each takes the
    brute-force mean of its good interior neighbours (25, 25 and 7 of them;
    the corner's ghost neighbours hold valid periodic images but are not
    used). Closed form for the pair: a + (53/25) b - c/25."""
    cfg = inputs.linear_mode_cfg(8, ndim=3)
    c0, c1, corner = (6, 6, 6), (6, 6, 7), (3, 3, 3)
    failed = [c0, c1, corner]
    P0, _, Pout, st = _fixup_run(orc, cfg, _quad_state(cfg, c0), failed)
    assert st == [3, 0, 0]
    np.testing.assert_allclose(Pout[(slice(0, 5),) + c0], COEF[:, 0] + COEF[:, 1] * 53 / 25 - COEF[:, 2] / 25,
                               rtol=1e-12, atol=1e-14)
    for c, n_want in ((c0, 25), (c1, 25), (corner, 7)):
        want, n = _brute_mean(cfg, P0, c, failed)
        assert n == n_want
        np.testing.assert_allclose(Pout[(slice(0, 5),) + c], want, rtol=1e-12, atol=1e-14)


def test_fixup_with_no_good_neighbour_keeps_the_input(orc):
    cfg = inputs.linear_mode_cfg(4, ndim=3)
    P0 = _quad_state(cfg, (5, 5, 5))
    sl = inputs.interior(cfg)
    cells = [tuple(x) for x in np.argwhere(np.ones(P0.shape[1:], bool)[sl]) + np.array([s.start for s in sl])]
    P0b, _, Pout, st = _fixup_run(orc, cfg, P0, cells)
    assert st == [64, 0, 64]
    assert np.array_equal(Pout[(slice(0, 5),) + sl], P0b[(slice(0, 5),) + sl])


# ---------------------------------------------------------------------------
# CFL time step: dt = cfl / sum_d (ctop_d / dx_d), minimised over zones.
# ---------------------------------------------------------------------------
def _box(n=(8, 6, 4), ext=(1.0, 1.8, 2.8), gam=4.0 / 3.0):
    cfg = inputs.linear_mode_cfg(8, ndim=3 if n[2] > 1 else 2)
    cfg.update(n1=n[0], n2=n[1], n3=n[2], x1=(0.0, ext[0]), x2=(0.0, ext[1]), x3=(0.0, ext[2]), gam=gam)
    dx = [ext[a] / n[a] for a in range(3 if n[2] > 1 else 2)]
    return cfg, np.array(dx)


def _uniform(cfg, prims):
    P = np.zeros(inputs.shape(cfg))
    P[:] = np.asarray(prims, dtype=np.float64)[:, None, None, None]
    return P


def _cs2(gam, rho, u):
    p = (gam - 1.0) * u
    return gam * p / (rho + u + p), rho + u + p


@pytest.mark.parametrize("ndim", [2, 3])
def test_cfl_dt_at_rest_is_sound_crossing(orc, ndim):
    cfg, dx = _box(n=(8, 6, 4 if ndim == 3 else 1))
    rho, u = 1.3, 0.7
    cs = np.sqrt(_cs2(cfg["gam"], rho, u)[0])
    dt = orc.cfl_dt(cfg, _uniform(cfg, [rho, u, 0, 0, 0, 0, 0, 0]))
    assert dt == pytest.approx(0.9 / (cs * np.sum(1.0 / dx)), rel=1e-13)


def test_cfl_dt_magnetised_rest_state_uses_the_fast_speed(orc):
    """c_ms^2 = v_A^2 + c_s^2 - v_A^2 c_s^2, v_A^2 = b^2/(b^2 + w), b^2 = |B|^2 at rest."""
    cfg, dx = _box()
    rho, u, B = 0.9, 0.4, np.array([0.4, -0.3, 0.2])
    cs2, w = _cs2(cfg["gam"], rho, u)
    va2 = B @ B / (B @ B + w)
    cms = np.sqrt(va2 + cs2 - va2 * cs2)
    dt = orc.cfl_dt(cfg, _uniform(cfg, [rho, u, 0, 0, 0, *B]))
    assert dt == pytest.approx(0.9 / (cms * np.sum(1.0 / dx)), rel=1e-13)


def test_cfl_dt_boosted_state(orc):
    """Fluid moving at v along x1: the x1 speed is (v + c)/(1 + v c) (velocity
    addition), the transverse ones c sqrt((1 - v^2)/(1 - c^2 v^2)) (a
    Lorentz-transformed isotropic front); each divides its own dx."""
    cfg, dx = _box()
    rho, u, v = 1.1, 0.6, 0.6
    c = np.sqrt(_cs2(cfg["gam"], rho, u)[0])
    ut1 = v / np.sqrt(1 - v * v)
    par = (v + c) / (1 + v * c)
    perp = c * np.sqrt((1 - v * v) / (1 - c * c * v * v))
    dt = orc.cfl_dt(cfg, _uniform(cfg, [rho, u, ut1, 0, 0, 0, 0, 0]))
    assert dt == pytest.approx(0.9 / (par / dx[0] + perp / dx[1] + perp / dx[2]), rel=1e-12)


def test_cfl_dt_is_the_minimum_over_zones(orc):
    """One hot zone in a cold uniform box (MC keeps the extremum flat, so every
    face touching it carries the hot speed): dt is the hot zone's."""
    cfg, dx = _box()
    P = _uniform(cfg, [1.0, 0.01, 0, 0, 0, 0, 0, 0])
    P[1, 5, 5, 6] = 3.0
    cs_hot = np.sqrt(_cs2(cfg["gam"], 1.0, 3.0)[0])
    dt = orc.cfl_dt(cfg, P)
    assert dt == pytest.approx(0.9 / (cs_hot * np.sum(1.0 / dx)), rel=1e-13)
