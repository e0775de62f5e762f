"""Pins for the oracle's tangent step (or_step_jvp: the step templated on
forward-mode dual numbers, with the implicit-function derivative of the
inversion): its values are the plain FP64 step's bit for bit; its
directional derivatives equal central differences of the plain FP64 step
(an independent evaluation) on rough states, including the derivative in
the adiabatic index; and conservation in a periodic box fixes the tangent
of the totals exactly (sum U^{n+1} = sum U^n for every input, so the same
holds for every direction)."""
import numpy as np
import pytest
from scipy.ndimage import maximum_filter

from paper_2408_01361_gb300 import inputs


def _random_box(recon, n=6, seed=3):
    cfg = inputs.linear_mode_cfg(n, ndim=3, recon=recon)
    rng = np.random.default_rng(seed)
    P = np.zeros(inputs.shape(cfg))
    P[0] = 1.0 + 0.1 * rng.random(P[0].shape)
    P[1] = 1.0 + 0.1 * rng.random(P[1].shape)
    P[2:5] = 0.1 * rng.normal(size=P[2:5].shape)
    P[5:] = 0.5 * rng.normal(size=P[5:].shape)
    return cfg, P


def _rough_torus(orc, recon):
    """2-D FM torus in FMKS with seeded roughness on the body (no component
    uniform there, so the reconstruction is away from its kinks)."""
    cfg = inputs.torus_cfg(48, 32, 1, r_out=60.0, recon=recon)
    P = inputs.torus_state(cfg, seed=2)
    body = (P[0:1] > 1e-2).astype(float)
    xi = inputs.uniform01(13, np.arange(P.size)).reshape(P.shape) - 0.5
    sc = np.maximum(np.abs(P).reshape(8, -1).max(axis=1), 1e-2)[:, None, None, None]
    Pr = P + 1e-3 * sc * xi * body
    Pr[0:2] = P[0:2]
    return cfg, orc.apply_bc(cfg, Pr)


def _fd(orc, cfg, U, P, vU, vP, dt, h):
    a = orc.step(cfg, U + h * vU, P + h * vP, dt)
    b = orc.step(cfg, U - h * vU, P - h * vP, dt)
    return (a[0] - b[0]) / (2 * h), (a[1] - b[1]) / (2 * h)


def _check_against_fd(orc, cfg, U, P, vU, vP, dt, tol):
    sl = (slice(None),) + inputs.interior(cfg)
    J = orc.step_jvp(cfg, U, P, vU, vP, 0.0, dt)
    f1 = _fd(orc, cfg, U, P, vU, vP, dt, 1e-6)
    f2 = _fd(orc, cfg, U, P, vU, vP, dt, 5e-7)
    for q in (0, 1):
        jv = J[2 + q][sl]
        sc = np.abs(jv).reshape(8, -1).max(axis=1)[:, None, None, None] + 1e-300
        noise = (np.abs(f1[q][sl] - f2[q][sl]) / sc).max()
        err = (np.abs(jv - f2[q][sl]) / sc).max()
        assert noise < tol, ("difference quotients not converged", noise)
        assert err < tol, (q, err, noise)


def test_jvp_values_are_the_plain_step(orc):
    for cfg, P in (_random_box("mc"), _rough_torus(orc, "weno5")):
        P = orc.apply_bc(cfg, P)
        U = orc.prim_to_cons(cfg, P)
        dt = 0.5 * orc.cfl_dt(cfg, P)
        rng = np.random.default_rng(4)
        vU, vP = rng.normal(size=P.shape), rng.normal(size=P.shape)
        U1, P1, dtn, st = orc.step(cfg, U, P, dt)
        J = orc.step_jvp(cfg, U, P, vU, vP, 0.7, dt)
        assert np.array_equal(J[0], U1) and np.array_equal(J[1], P1)
        assert J[4] == dtn and J[5] == st


@pytest.mark.parametrize("recon", ["mc", "weno5"])
def test_jvp_matches_central_differences_box(orc, recon):
    """Rough Minkowski box: directions on two zones (one in P, one in U);
    the tangent matches the quotients within 1e-7 of each component's
    largest derivative (they agree with each other to ~1e-9)."""
    cfg, P = _random_box(recon)
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    dt = 0.3 / 6
    rng = np.random.default_rng(5)
    for _ in range(3):
        vU = np.zeros_like(P)
        vP = np.zeros_like(P)
        vP[(slice(None),) + tuple(rng.integers(3, 9, size=3))] = rng.normal(size=8)
        vU[(slice(None),) + tuple(rng.integers(3, 9, size=3))] = rng.normal(size=8)
        _check_against_fd(orc, cfg, U, P, vU, vP, dt, 1e-7)


@pytest.mark.parametrize("recon", ["mc", "weno5"])
def test_jvp_gamma_derivative_box(orc, recon):
    cfg, P = _random_box(recon)
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    dt = 0.3 / 6
    sl = (slice(None),) + inputs.interior(cfg)
    z = np.zeros_like(P)
    J = orc.step_jvp(cfg, U, P, z, z, 1.0, dt)
    h = 1e-6
    a = orc.step(dict(cfg, gam=cfg["gam"] + h), U, P, dt)
    b = orc.step(dict(cfg, gam=cfg["gam"] - h), U, P, dt)
    for q in (0, 1):
        fd = (a[q] - b[q]) / (2 * h)
        assert np.abs(J[2 + q][sl] - fd[sl]).max() < 1e-7 * np.abs(fd[sl]).max()


@pytest.mark.parametrize("recon", ["mc", "weno5"])
def test_jvp_conserves_totals_in_periodic_box(orc, recon):
    cfg, P = _random_box(recon)
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    sl = (slice(None),) + inputs.interior(cfg)
    rng = np.random.default_rng(6)
    vU = np.zeros_like(P)
    vP = np.zeros_like(P)
    vU[sl] = rng.normal(size=vU[sl].shape)
    vP[sl] = rng.normal(size=vP[sl].shape)
    J = orc.step_jvp(cfg, U, P, vU, vP, 0.3, 0.3 / 6)
    tot_out = J[2][sl].sum(axis=(1, 2, 3))
    tot_in = vU[sl].sum(axis=(1, 2, 3))
    assert np.all(np.abs(tot_out - tot_in) <= 1e-13 * np.abs(J[2][sl]).sum(axis=(1, 2, 3)))


def test_jvp_matches_central_differences_torus(orc):
    """FMKS torus (metric, connection sources, polar and outflow ghosts),
    WENO5: directions on body zones with no failed or floored zone within 7
    zones (there the frozen-floor and frozen-fixup rules differ from the
    derivative of the plain step by design)."""
    cfg, P = _rough_torus(orc, "weno5")
    U = orc.prim_to_cons(cfg, P)
    dt = 0.5 * orc.cfl_dt(cfg, P)
    z = np.zeros_like(P)
    zf = orc.step_jvp(cfg, U, P, z, z, 0.0, dt)[6]
    near = maximum_filter(zf[0], size=15, mode="constant") > 0
    ok = np.argwhere(~near & (P[0, 0] > 0.01))
    assert len(ok) >= 6
    rng = np.random.default_rng(5)
    for _ in range(3):
        j, i = ok[rng.integers(len(ok))]
        vU = np.zeros_like(P)
        vP = np.zeros_like(P)
        vP[:, 0, j, i] = rng.normal(size=8) * np.abs(P[:, 0, j, i]).clip(1e-3)
        vU[:, 0, j, i] = rng.normal(size=8) * np.abs(U[:, 0, j, i]).clip(1e-3)
        _check_against_fd(orc, cfg, U, P, vU, vP, dt, 2e-5)
