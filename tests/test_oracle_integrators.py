"""Pins for the oracle's Runge-Kutta integrators (the paper's "Algorithm"
section: RK1, RK2 and SSPRK(5)4 beside the predictor-corrector), by what
their definitions fix: on a fixed grid the temporal error against a
reference run with a much smaller step falls as dt^1 (RK1), dt^2 (RK2 and
the predictor-corrector) and dt^4 (SSPRK(5,4)); a wrong coefficient in any
stage breaks the order. Every integrator conserves the totals of a periodic
box exactly and keeps a uniform state."""
import os

import numpy as np
import pytest

from conftest import GOLDEN
from paper_2408_01361_gb300 import inputs

ORDERS = {"rk1": 1.0, "rk2": 2.0, "vl2": 2.0, "ssprk54": 4.0}


def test_temporal_orders(orc):
    dP, om = inputs.load_eigvec(os.path.join(GOLDEN, "linear_fast_mode.txt"))
    cfg = inputs.linear_mode_cfg(16, ndim=2, recon="weno5")
    P = orc.apply_bc(cfg, inputs.linear_mode_state(cfg, dP, om))
    U = orc.prim_to_cons(cfg, P)
    T = 0.25 * 2 * np.pi / om
    n0 = int(np.ceil(T / orc.cfl_dt(cfg, P)))

    def run(integ, nst):
        c = dict(cfg, integrator=integ)
        Uc, Pc = U, P
        for _ in range(nst):
            Uc, Pc, _, st = orc.step(c, Uc, Pc, T / nst)
            assert st == [0, 0, 0]
        return Pc

    sl = (slice(None),) + inputs.interior(cfg)
    ref = run("ssprk54", 256)
    for integ, p in ORDERS.items():
        e = [np.abs(run(integ, n0 * m)[sl] - ref[sl]).mean() for m in (1, 2, 4)]
        for a, b in ((e[0], e[1]), (e[1], e[2])):
            assert abs(np.log2(a / b) - p) < 0.1, (integ, e)


@pytest.mark.parametrize("integ", ["rk1", "rk2", "ssprk54"])
def test_conservation_and_uniform_state(orc, integ):
    cfg = dict(inputs.linear_mode_cfg(8, ndim=3, recon="weno5"), integrator=integ)
    rng = np.random.default_rng(4)
    P = np.zeros(inputs.shape(cfg))
    P[0] = 1.0 + 0.1 * rng.random(P[0].shape)
    P[1] = 1.0 + 0.1 * rng.random(P[1].shape)
    P[2:5] = 0.1 * rng.normal(size=P[2:5].shape)
    P[5:] = 0.3 * rng.normal(size=P[5:].shape)
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    U2, P2, _, st = orc.step(cfg, U, P, 0.01)
    assert st == [0, 0, 0]
    sl = (slice(None),) + inputs.interior(cfg)
    tot0 = U[sl].reshape(8, -1).sum(axis=1)
    tot1 = U2[sl].reshape(8, -1).sum(axis=1)
    scale = np.abs(U[sl]).reshape(8, -1).sum(axis=1)
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale), (tot1 - tot0) / scale
    Pu = np.zeros(inputs.shape(cfg))
    Pu[:] = np.array([0.8, 0.5, 0.3, -0.2, 0.1, 0.4, 0.7, -0.3])[:, None, None, None]
    Uu = orc.prim_to_cons(cfg, Pu)
    Uu2, Pu2, _, _ = orc.step(cfg, Uu, Pu, 0.01)
    assert np.abs(Uu2[sl] - Uu[sl]).max() < 1e-14
    assert np.abs(Pu2[sl] - Pu[sl]).max() < 1e-13
