"""Pins for the Minkowski test problems the paper cites (the Orszag-Tang
vortex, Komissarov's cylindrical explosion) on the oracle: the symmetries
of their initial states survive the evolution to rounding (the half-turn of
the vortex; both mirror symmetries of the explosion), and the periodic
vortex conserves its totals exactly."""
import numpy as np

from paper_2408_01361_gb300 import inputs


def _evolve(orc, cfg, P, t_end):
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    U2, P2, t, st = orc.evolve(cfg, U, P, 0, -orc.cfl_dt(cfg, P), t_end)
    assert abs(t - t_end) < 1e-12 and st == [0, 0, 0]
    return U, U2, P2


def test_orszag_tang_half_turn_and_conservation(orc):
    cfg = inputs.orszag_tang_cfg(32)
    U, U2, P2 = _evolve(orc, cfg, inputs.orszag_tang_state(cfg), 0.5)
    sl = inputs.interior(cfg)
    A = P2[(slice(None),) + sl]
    R = A[:, :, ::-1, ::-1]
    for v in range(8):
        sgn = 1.0 if v < 2 else -1.0
        assert np.abs(A[v] - sgn * R[v]).max() < 1e-12 * (np.abs(A[v]).max() + 1.0), v
    s0 = U[(slice(None),) + sl].reshape(8, -1).sum(axis=1)
    s1 = U2[(slice(None),) + sl].reshape(8, -1).sum(axis=1)
    sc = np.abs(U[(slice(None),) + sl]).reshape(8, -1).sum(axis=1)
    assert np.all(np.abs(s1 - s0) <= 1e-13 * sc)


def test_explosion_mirror_symmetries(orc):
    cfg = inputs.explosion_cfg(48)
    _, _, P2 = _evolve(orc, cfg, inputs.explosion_state(cfg), 0.5)
    sl = inputs.interior(cfg)
    A = P2[(slice(None),) + sl]
    odd_x = {2, 6, 7}  # x -> -x: u~1, B2, B3 change sign
    odd_y = {3, 6}     # y -> -y: u~2, B2 change sign
    for v in range(8):
        sc = np.abs(A[v]).max() + 1e-300
        Rx = A[v][:, :, ::-1] * (-1.0 if v in odd_x else 1.0)
        Ry = A[v][:, ::-1, :] * (-1.0 if v in odd_y else 1.0)
        assert np.abs(A[v] - Rx).max() <= 1e-12 * sc, ("x", v)
        assert np.abs(A[v] - Ry).max() <= 1e-12 * sc, ("y", v)
    assert A[0].max() < 1e-2 and A[0].min() > 0  # the blast has expanded
