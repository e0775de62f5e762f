"""Pins for the oracle's Runge-Kutta integrators (the paper's "Algorithm"
section: RK1, RK2 and SSPRK(5)4 beside the predictor-corrector), by what
their definitions fix: on a fixed grid the temporal error against a
reference run with a much smaller step falls as dt^1 (RK1), dt^2 (RK2 and
the predictor-corrector) and dt^4 (SSPRK(5,4)); a wrong coefficient in any
stage breaks the order. Every integrator conserves the totals of a periodic
box exactly and keeps a uniform state. Combined with face-centred CT (the
face field a stage state like U) every integrator keeps each cell's face
divergence, and with averaged edge EMFs it is the Flux-CT integrator (a
separate code path) to rounding; combined with the first-order flux
correction it is the plain integrator where no zone is flagged and the
donor-cell integrator where every zone is."""
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


def _box(n=8, ndim=3, recon="weno5", seed=3):
    cfg = inputs.linear_mode_cfg(n, ndim=ndim, recon=recon)
    rng = np.random.default_rng(seed)
    P = np.zeros(inputs.shape(cfg))
    P[0] = 1.0 + 0.1 * rng.random(P[0].shape)
    P[1] = 1.0 + 0.1 * rng.random(P[1].shape)
    P[2:5] = 0.1 * rng.normal(size=P[2:5].shape)
    fB = inputs.random_face_field(cfg, seed + 2, 0.5)
    return cfg, inputs.cell_field_from_faces(cfg, fB, P), fB


@pytest.mark.parametrize("integ", ["rk1", "rk2", "ssprk54"])
def test_face_ct_integrators(orc, integ):
    cfg, P, fB = _box()
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    dx = min((cfg[k][1] - cfg[k][0]) / cfg[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3")))
    scale = np.abs(fB).max() / dx
    # the face divergence is kept (upwinded EMFs)
    cf = dict(cfg, bfield="face", emf="gs05", integrator=integ)
    _, _, d0 = orc.face_divb(cf, fB, field=True)
    Uf, Pf, f = U, P, fB
    for _ in range(2):
        Uf, Pf, f, _, _ = orc.step_face(cf, Uf, Pf, f, dt)
    _, _, d1 = orc.face_divb(cf, f, field=True)
    assert np.abs(d1 - d0).max() < 1e-13 * scale
    # a stage that ignored the face field's stage states would not move it
    # as the Flux-CT integrator moves B: averaged EMFs = Flux-CT, to rounding
    ca = dict(cf, emf="average")
    c = dict(cfg, integrator=integ)
    Ua, Pa, Uf, Pf, f = U, P, U, P, fB
    for _ in range(2):
        Ua, Pa, _, _ = orc.step(c, Ua, Pa, dt)
        Uf, Pf, f, _, _ = orc.step_face(ca, Uf, Pf, f, dt)
    sl = inputs.interior(cfg)
    for v in range(8):
        sc = np.abs(Ua[v][sl]).max() + 1e-300
        assert np.abs(Ua[v][sl] - Uf[v][sl]).max() < 1e-13 * sc, (v, integ)
        sc = np.abs(Pa[v][sl]).max() + 1e-300
        assert np.abs(Pa[v][sl] - Pf[v][sl]).max() < 1e-13 * sc, (v, integ)
    # and differs from the predictor-corrector's face step
    Uv, _, _, _, _ = orc.step_face(dict(ca, integrator="vl2"), U, P, fB, dt)
    U1, _, _, _, _ = orc.step_face(ca, U, P, fB, dt)
    assert integ == "rk2" or not np.allclose(U1[(slice(None),) + sl], Uv[(slice(None),) + sl], rtol=1e-10, atol=0)


@pytest.mark.parametrize("integ", ["rk1", "rk2", "ssprk54"])
def test_fofc_integrators(orc, integ):
    """rho_min = 10 floors every zone of every RK1 / RK2 stage (each stage's
    base has rho < 10); SSPRK(5,4)'s later bases combine floored states, so
    there only some zones are flagged."""
    cfg = inputs.linear_mode_cfg(8, ndim=3, recon="weno5")
    cfg["n1"], cfg["n2"], cfg["n3"] = 10, 8, 6
    rng = np.random.default_rng(3)
    P = np.zeros(inputs.shape(cfg))
    P[0] = 1.0 + 0.1 * rng.random(P[0].shape)
    P[1] = 1.0 + 0.1 * rng.random(P[1].shape)
    P[2:5] = 0.1 * rng.normal(size=P[2:5].shape)
    P[5:] = 0.5 * rng.normal(size=P[5:].shape)
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    dt = 1e-3
    sl = (slice(None),) + inputs.interior(cfg)
    for rho_min, ref_recon in ((1e-20, "weno5"), (10.0, "donor")):
        c = dict(cfg, integrator=integ, floors=dict(rho_min=rho_min, u_min=1e-20))
        Uo, Po, _, _ = orc.step(dict(c, fofc=True), U, P, dt)
        nflag = orc.last_nfofc
        Ur, Pr, _, _ = orc.step(dict(c, recon=ref_recon), U, P, dt)
        if rho_min > 1 and integ == "ssprk54":
            assert 2 * 10 * 8 * 6 <= nflag < 5 * 10 * 8 * 6
            assert np.isfinite(Uo).all() and np.isfinite(Po).all()
        elif rho_min > 1:
            assert nflag == (2 if integ == "rk2" else 1) * 10 * 8 * 6
            # every zone flagged in every stage: the donor-cell integrator
            assert np.allclose(Uo[sl], Ur[sl], rtol=1e-13, atol=0)
            assert np.allclose(Po[sl], Pr[sl], rtol=1e-13, atol=0)
        else:
            assert nflag == 0
            assert np.array_equal(Uo[sl], Ur[sl]) and np.array_equal(Po[sl], Pr[sl])
