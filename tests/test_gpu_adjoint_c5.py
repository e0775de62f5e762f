"""The adjoint at the adjoint workload's sizes: gradients of the final total
energy E = -sum (U_energy - U_rho) dV and of a mass flux through an x1 face
plane on the last step's second stage (at the torus's horizon: the accretion
rate) through 20 steps of the 64^3 linear-mode box and of the 128x64 FMKS
torus (a = 0.9375, the workload's torus parameters), with respect to the
initial conserved and primitive variables and the adiabatic index.

Checks, per objective and direction v (on every interior zone, and on gamma):
  * the CUDA adjoint (torch.autograd wrappers, per-step checkpoints) against
    the oracle's dual-number tangent chained over the same 20 steps
    (independent code, the same derivative rules: branches as taken, the
    inversion by the implicit-function theorem, floored components and
    fixed-up zones frozen): within 1e-6 of the sum of the terms' magnitudes;
  * against central differences of the CUDA forward for the flux objective
    on the box. The step is piecewise smooth (MC's branches, the max in the
    LLF speed): a perturbation of size h flips every branch decided within h
    of a tie, and over 20 steps the perturbation reaches every zone, so a
    difference quotient carries an error of its own that does not vanish
    with h at a useful rate -- measured on the oracle alone (16^3 and 32^3
    boxes, 20 steps), quotients of a direction on every zone stay 0.2-0.6%
    from the exact (dual-number) derivative for h from 1e-5 to 1e-7; for a
    direction on three zones the 16^3 box reaches 3e-8 at h = 1e-7, the 32^3
    box (whole box reached) still 0.2%. The check therefore takes a direction
    on three zones, h = 1e-7 relative and h/2, and a bound of 5e-3 of the
    quotient (or twice the quotients' difference, if larger).
    On the torus the adjoint's rules themselves differ from the function:
    floored components and fixed-up zones are frozen (zero derivative), while
    the floors there include the magnetisation ceilings rho >= b^2/100 that
    do depend on the state -- near the horizon the accretion rate's
    derivative through them is tens of percent. There the dual-number tangent
    (the same rules) is the check, and central differences are not used.
  * the mixed-precision forward: the gradient of the FP64 step taken along
    the mixed trajectory (adj_ctx) against the FP64 trajectory's, within the
    distance of the two trajectories."""
import os

import numpy as np
import pytest

from conftest import GOLDEN
from paper_2408_01361_gb300 import inputs

pytestmark = pytest.mark.gpu

NSTEPS = 20


@pytest.fixture(scope="module")
def kh():
    from paper_2408_01361_gb300 import kh as _kh
    return _kh


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    return _t


def _rough(P, seed, amp):
    xi = inputs.uniform01(seed, np.arange(P.size)).reshape(P.shape) - 0.5
    sc = np.maximum(np.abs(P).reshape(P.shape[0], -1).max(axis=1), 1e-2)[:, None, None, None]
    return P + amp * sc * xi


def _box(orc):
    """The 64^3 slow-mode box (MC) with seeded roughness on every component
    (no limiter branch decided by a tie)."""
    cfg = inputs.linear_mode_cfg(64, ndim=3)
    dP, om = inputs.load_eigvec(os.path.join(GOLDEN, "linear_slow_mode.txt"))
    P = _rough(inputs.linear_mode_state(cfg, dP, om, amp=1e-4), 31, 0.02)
    P = orc.apply_bc(cfg, P)
    return cfg, P, 0.5 * orc.cfl_dt(cfg, P), inputs.shape(cfg)[3] // 2


def _torus(orc, recon="mc"):
    """The 128x64 FMKS torus (2-D) with seeded roughness on every zone and
    component, so that no branch is decided by round-off."""
    cfg = inputs.torus_cfg(128, 64, 1, recon=recon)
    P = inputs.torus_state(cfg, seed=3)
    xi = inputs.uniform01(33, np.arange(P.size)).reshape(P.shape) - 0.5
    sc = np.maximum(np.abs(P).reshape(8, -1).max(axis=1), 1e-2)[:, None, None, None]
    Pr = P + 1e-3 * sc * xi
    Pr[0:2] = P[0:2] * (1 + 1e-2 * xi[0:2])
    Pr[5:] = P[5:] + 1e-3 * np.sqrt(P[0:1]) * xi[5:]
    Pr = orc.apply_bc(cfg, Pr)
    # the x1 face nearest the horizon r_h = 1 + sqrt(1 - a^2) (x1 = ln r)
    rh = 1.0 + np.sqrt(1.0 - cfg["a"] ** 2)
    dx1 = (cfg["x1"][1] - cfg["x1"][0]) / cfg["n1"]
    k = int(np.floor((np.log(rh) - cfg["x1"][0]) / dx1 + 0.5))
    return cfg, Pr, 0.5 * orc.cfl_dt(cfg, Pr), 3 + k


def _dV(cfg):
    return np.prod([(cfg[k][1] - cfg[k][0]) / cfg[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3"))])


def _dA1(cfg):
    return np.prod([(cfg[k][1] - cfg[k][0]) / cfg[n] for k, n in (("x2", "n2"), ("x3", "n3"))])


def _rollout(kh, torch, cfg, U0, P0, dt, i_face, precision=None):
    """Adjoint gradients of E and of the face-plane mass flux through NSTEPS
    steps: dict objective -> (J, gU0, gPB0, g_gamma)."""
    from paper_2408_01361_gb300 import autograd as kga
    c = dict(cfg, precision=precision) if precision else cfg
    ctx = kh.Context(c)
    adj = kh.Context(cfg) if precision == "mixed" else None
    N1 = P0.shape[3]
    ksl, jsl, isl = inputs.interior(cfg)
    out = {}
    for name in ("energy", "mdot"):
        Ut = ctx.to_device(U0).requires_grad_(True)
        PB = ctx.to_device(P0)
        Pt = PB[:5].clone().requires_grad_(True)
        Bt = PB[5:].clone().requires_grad_(True)
        gam = torch.tensor(cfg["gam"], dtype=torch.float64, device=ctx.device, requires_grad=True)
        U, P, B = Ut, Pt, Bt
        for q in range(NSTEPS):
            if q == NSTEPS - 1:
                U, P, B, F1 = kga.step(ctx, U, P, B, gam, dt, adj_ctx=adj, with_flux=True)
            else:
                U, P, B = kga.step(ctx, U, P, B, gam, dt, adj_ctx=adj)
        if name == "energy":
            J = -(U[1, ksl, jsl, isl] - U[0, ksl, jsl, isl]).sum() * _dV(cfg)
        else:
            J = -F1[0, ksl, jsl, i_face].sum() * _dA1(cfg)
        J.backward()
        out[name] = (float(J.detach()), ctx.to_host(Ut.grad, N1),
                     np.concatenate([ctx.to_host(Pt.grad, N1), ctx.to_host(Bt.grad, N1)]), float(gam.grad))
    return out


def _dual(orc, cfg, U0, P0, dt, vU, vP, dgam, i_face):
    """The oracle's tangents of E and of the face-plane mass flux along (vU,
    vP, dgam), chained over NSTEPS steps."""
    Uo, Po, dU, dP = U0, P0, vU, vP
    for q in range(NSTEPS):
        T = orc.step_jvp(cfg, Uo, Po, dU, dP, dgam, dt, flux=(q == NSTEPS - 1))
        Uo, Po, dU, dP = T[0], T[1], T[2], T[3]
    ksl, jsl, isl = inputs.interior(cfg)
    dE = -(dU[1][ksl, jsl, isl] - dU[0][ksl, jsl, isl]).sum() * _dV(cfg)
    dM = -T[7][0, ksl, jsl, i_face].sum() * _dA1(cfg)
    return {"energy": dE, "mdot": dM}


def _direction(cfg, U0, P0, seed, zones=None):
    """A random direction on every interior zone (zones=None) or on `zones`
    random interior zones, each variable scaled by its largest magnitude,
    and a random gamma component."""
    rng = np.random.default_rng(seed)
    sl = (slice(None),) + inputs.interior(cfg)
    vU = np.zeros(P0.shape)
    vP = np.zeros(P0.shape)
    if zones is None:
        vU[sl] = rng.normal(size=vU[sl].shape)
        vP[sl] = rng.normal(size=vP[sl].shape)
    else:
        lo = [s.start for s in inputs.interior(cfg)]
        hi = [s.stop for s in inputs.interior(cfg)]
        for _ in range(zones):
            z = tuple(int(rng.integers(lo[a], hi[a])) for a in range(3))
            vU[(slice(None),) + z] = rng.normal(size=8)
            vP[(slice(None),) + z] = rng.normal(size=8)
    vU *= np.abs(U0).reshape(8, -1).max(axis=1)[:, None, None, None]
    vP *= np.abs(P0).reshape(8, -1).max(axis=1)[:, None, None, None]
    return vU, vP, float(rng.normal())


def _pair(g, vU, vP, dgam):
    """<gradient, direction> and the sum of its terms' magnitudes."""
    _, gU, gPB, gg = g
    terms = np.concatenate([(gU * vU).ravel(), (gPB * vP).ravel(), [gg * dgam]])
    return terms.sum(), np.abs(terms).sum()


def _cuda_mdot(kh, cfg, U0, P0, dt, gam, i_face):
    from gpu_helpers import GpuRun
    c = dict(cfg, gam=gam)
    ctx = kh.Context(c)
    g = GpuRun(ctx, c, P0, U=U0)
    for _ in range(NSTEPS):
        ctx.step(g.U, g.P, g.B, dt)
    F1 = ctx.stage_flux(1).cpu().numpy()
    ksl, jsl, _ = inputs.interior(cfg)
    return -F1[0, ksl, jsl, i_face].sum() * _dA1(cfg)


def _fd(f, U0, P0, gam, vU, vP, dgam, rel=1e-7):
    """Central differences of f(U, P, gam) along the direction at steps h and
    h/2 (h = rel, the direction already carries each variable's scale)."""
    out = []
    for h in (rel, 0.5 * rel):
        out.append((f(U0 + h * vU, P0 + h * vP, gam + h * dgam * gam)
                    - f(U0 - h * vU, P0 - h * vP, gam - h * dgam * gam)) / (2 * h))
    return out


def _check_case(kh, torch, orc, cfg, P0, dt, i_face, seeds, fd):
    """Adjoint vs the oracle's dual tangent for a direction on every zone
    (both objectives), and (fd) vs central differences of the CUDA forward
    for the flux objective along a direction on three zones."""
    U0 = orc.prim_to_cons(cfg, P0)
    grads = _rollout(kh, torch, cfg, U0, P0, dt, i_face)
    checked = 0
    for seed in seeds:
        vU, vP, dgam_unit = _direction(cfg, U0, P0, seed)
        dgam = dgam_unit * cfg["gam"]
        tan = _dual(orc, cfg, U0, P0, dt, vU, vP, dgam, i_face)
        for name in ("energy", "mdot"):
            adj, scale = _pair(grads[name], vU, vP, dgam)
            assert abs(adj - tan[name]) <= 1e-6 * scale, (name, seed, adj, tan[name], scale)
        if not fd:
            continue
        vU, vP, dgam_unit = _direction(cfg, U0, P0, seed + 100, zones=3)
        dgam = dgam_unit * cfg["gam"]
        fds = _fd(lambda U, P, g: _cuda_mdot(kh, cfg, U, P, dt, g, i_face), U0, P0, cfg["gam"], vU, vP, dgam_unit)
        adj, _ = _pair(grads["mdot"], vU, vP, dgam)
        band = abs(fds[0] - fds[1])
        assert abs(adj - fds[1]) <= max(2.0 * band, 5e-3 * abs(fds[1])), (seed, adj, fds)
        checked += 1
    return grads, checked


def test_c5_box_64cubed_20_steps(kh, torch, orc):
    """The periodic box: E is conserved exactly, so dE/dP0 = 0 and dE/dU0 =
    -dV (e_energy - e_rho) at every interior zone; the face-plane mass flux
    is a generic objective."""
    cfg, P0, dt, i_face = _box(orc)
    grads, checked = _check_case(kh, torch, orc, cfg, P0, dt, i_face, seeds=(40, 41), fd=True)
    _, gU, gPB, gg = grads["energy"]
    sl = (slice(None),) + inputs.interior(cfg)
    want = np.zeros(8)
    want[0], want[1] = _dV(cfg), -_dV(cfg)
    assert np.abs(gU[sl] - want[:, None, None, None]).max() <= 1e-9 * _dV(cfg)
    assert np.abs(gPB[sl]).max() <= 1e-9 * _dV(cfg) and abs(gg) <= 1e-9
    assert checked == 2


def test_c5_torus_128x64_20_steps(kh, torch, orc):
    """The FMKS torus with its floors, fixups, polar axis and outflow
    boundaries: E and the horizon mass flux against the dual tangent."""
    cfg, P0, dt, i_face = _torus(orc)
    _check_case(kh, torch, orc, cfg, P0, dt, i_face, seeds=(50, 51, 52), fd=False)


def test_c5_torus_mixed_forward(kh, torch, orc):
    """The mixed-precision forward with the FP64 adjoint (adj_ctx): the
    gradient of the FP64 step along the mixed trajectory. Its directional
    derivatives equal the FP64 trajectory's within 1e-3 of the sum of the
    terms' magnitudes (the trajectories differ at the FP32 flux level; 1.1e-4
    measured on the energy)."""
    cfg, P0, dt, i_face = _torus(orc)
    U0 = orc.prim_to_cons(cfg, P0)
    g64 = _rollout(kh, torch, cfg, U0, P0, dt, i_face)
    gmx = _rollout(kh, torch, cfg, U0, P0, dt, i_face, precision="mixed")
    for seed in (60, 61):
        vU, vP, dgam_unit = _direction(cfg, U0, P0, seed)
        dgam = dgam_unit * cfg["gam"]
        for name in ("energy", "mdot"):
            a, sa = _pair(g64[name], vU, vP, dgam)
            b, _ = _pair(gmx[name], vU, vP, dgam)
            assert abs(a - b) <= 1e-3 * sa, (name, seed, a, b, sa)
    for name in ("energy", "mdot"):
        assert abs(g64[name][0] - gmx[name][0]) <= 1e-4 * abs(g64[name][0]), (name, g64[name][0], gmx[name][0])
