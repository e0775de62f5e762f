"""Pins for the oracle's face-centred constrained transport (the paper's
"Algorithm" section: the face-centred CT of Stone & Gardiner 2009 with edge
EMFs after Gardiner & Stone 2005), by what the scheme fixes independently of
its code:
  * the face divergence of every cell is unchanged by a step (to rounding),
    for either EMF scheme, on a periodic box and on FMKS tori with polar and
    outflow boundaries;
  * with plain averaged EMFs the scheme is Toth's Flux-CT written on faces:
    starting from a cell field equal to the face means, the step equals the
    oracle's Flux-CT step (separate code) to rounding;
  * with the upwinded EMFs a flow that varies along x1 only evolves B^2 by
    the 1-D Riemann fluxes, so swapping (u~2, B^2) with (u~3, B^3), whose
    x1-x2 grid moves B^3 by plain finite volumes, commutes with the step;
    the averaged EMFs fail that (the test has teeth);
  * on a polar axis the faces carry no field: sqrt(-g) B^2 there stays 0.
The upwind side taken by the derivative terms is a reading of the paper's
reference (the mass flux through the attached face) that none of these
fixes: it changes results at second order only."""
import numpy as np
import pytest

from paper_2408_01361_gb300 import inputs


def _box(n=8, ndim=3, recon="weno5", seed=3, bscale=0.5):
    cfg = inputs.linear_mode_cfg(n, ndim=ndim, recon=recon)
    rng = np.random.default_rng(seed)
    P = np.zeros(inputs.shape(cfg))
    P[0] = 1.0 + 0.1 * rng.random(P[0].shape)
    P[1] = 1.0 + 0.1 * rng.random(P[1].shape)
    P[2:5] = 0.1 * rng.normal(size=P[2:5].shape)
    fB = inputs.random_face_field(cfg, seed + 2, bscale)
    P = inputs.cell_field_from_faces(cfg, fB, P)
    return cfg, P, fB


def _torus(n3, recon="weno5"):
    cfg = inputs.torus_cfg(48, 32, n3, r_out=60.0, recon=recon)
    P = inputs.torus_state(cfg, seed=2)
    fB = inputs.torus_face_field(cfg)
    return cfg, P, fB


def _interior_div_scale(orc, cfg, fB):
    """|fB| / dx: the size of one face difference."""
    dx = min((cfg[k][1] - cfg[k][0]) / cfg[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3")))
    return np.abs(fB).max() / dx


@pytest.mark.parametrize("case", ["box3d", "box2d", "torus2d", "torus3d"])
@pytest.mark.parametrize("emf", ["average", "gs05"])
def test_face_divergence_is_preserved(orc, case, emf):
    if case.startswith("box"):
        cfg, P, fB = _box(ndim=int(case[3]), recon="mc" if case == "box2d" else "weno5")
    else:
        cfg, P, fB = _torus(1 if case == "torus2d" else 8)
    cf = dict(cfg, bfield="face", emf=emf)
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    scale = _interior_div_scale(orc, cfg, fB)
    _, _, d0 = orc.face_divb(cf, fB, field=True)
    assert np.abs(d0).max() < 1e-13 * scale
    dt = 0.5 * orc.cfl_dt(cfg, P)
    for _ in range(3):
        U, P, fB, dtn, st = orc.step_face(cf, U, P, fB, dt)
    _, _, d1 = orc.face_divb(cf, fB, field=True)
    assert np.abs(d1 - d0).max() < 1e-13 * scale
    assert np.isfinite(U).all()


@pytest.mark.parametrize("ndim,recon", [(3, "weno5"), (2, "mc")])
def test_averaged_emfs_are_flux_ct(orc, ndim, recon):
    cfg, P, fB = _box(n=10, ndim=ndim, recon=recon)
    P = orc.apply_bc(cfg, P)
    U = orc.prim_to_cons(cfg, P)
    cf = dict(cfg, bfield="face", emf="average")
    dt = 0.5 * orc.cfl_dt(cfg, P)
    Ua, Pa, Uf, Pf, f = U, P, U, P, fB
    for _ in range(2):
        Ua, Pa, _, _ = orc.step(cfg, Ua, Pa, dt)
        Uf, Pf, f, _, _ = orc.step_face(cf, Uf, Pf, f, dt)
    sl = (slice(None),) + inputs.interior(cfg)
    for v in range(8):
        sc = np.abs(Ua[v][sl[1:]]).max() + 1e-300
        assert np.abs(Ua[v][sl[1:]] - Uf[v][sl[1:]]).max() < 1e-13 * sc, v
        sc = np.abs(Pa[v][sl[1:]]).max() + 1e-300
        assert np.abs(Pa[v][sl[1:]] - Pf[v][sl[1:]]).max() < 1e-13 * sc, v
    # and the upwinded EMFs give a different (second-order-close) result
    Ug, _, _, _, _ = orc.step_face(dict(cf, emf="gs05"), U, P, fB, dt)
    Uc = orc.step(cfg, U, P, dt)[0]
    assert not np.allclose(Ug[5:][sl], Uc[5:][sl], rtol=1e-10, atol=0)


def _plane_parallel(swap: bool):
    """2-D Minkowski box; state varying along x1 only, with transverse
    velocity and field in (u~2, B^2) and (u~3, B^3); swap exchanges them."""
    cfg = inputs.linear_mode_cfg(16, ndim=2, recon="weno5")
    cfg["n2"] = 6
    N = inputs.shape(cfg)
    x1 = inputs.centers(cfg, 0)
    prof = lambda a, b, c: a + b * np.sin(2 * np.pi * x1 + c)  # noqa: E731
    P = np.zeros(N)
    P[0] = prof(1.0, 0.2, 0.3)
    P[1] = prof(1.0, 0.3, 1.1)
    P[2] = prof(0.1, 0.2, 2.0)
    t2, t3 = prof(0.05, 0.2, 0.7), prof(-0.1, 0.15, 2.9)
    b2, b3 = prof(0.2, 0.4, 1.7), prof(-0.3, 0.3, 0.4)
    if swap:
        t2, t3, b2, b3 = t3, t2, b3, b2
    P[3], P[4] = t2, t3
    fB = np.zeros((3,) + N[1:])
    fB[0] = 0.7                          # uniform B^1: the field is divergence-free
    fB[1] = b2                           # x2 faces: uniform along x2
    fB[2] = b3
    P[5] = 0.7
    P[6], P[7] = b2, b3
    return cfg, P, fB


def test_upwinded_emfs_reduce_to_the_1d_riemann_emf(orc):
    out = {}
    for emf in ("gs05", "average"):
        res = []
        for swap in (False, True):
            cfg, P, fB = _plane_parallel(swap)
            cf = dict(cfg, bfield="face", emf=emf)
            P = orc.apply_bc(cfg, P)
            U = orc.prim_to_cons(cfg, P)
            dt = 0.3 / 16  # the same for both (the x2 signal speeds differ)
            for _ in range(3):
                U, P, fB, _, _ = orc.step_face(cf, U, P, fB, dt)
            res.append((P, fB))
        sl = inputs.interior(cfg)
        (Pa, fa), (Pb, fb) = res
        # B^2 of the plain problem is B^3 of the swapped one, and vice versa
        d_b = max(np.abs(fa[1][sl] - fb[2][sl]).max(), np.abs(fa[2][sl] - fb[1][sl]).max())
        d_u = max(np.abs(Pa[3][sl] - Pb[4][sl]).max(), np.abs(Pa[0][sl] - Pb[0][sl]).max())
        out[emf] = (d_b, d_u)
    assert out["gs05"][0] < 1e-13 and out["gs05"][1] < 1e-13, out
    assert out["average"][0] > 1e-6, out


def test_polar_faces_carry_no_field(orc):
    for n3 in (1, 8):
        cfg, P, fB = _torus(n3)
        cf = dict(cfg, bfield="face", emf="gs05")
        P = orc.apply_bc(cfg, P)
        U = orc.prim_to_cons(cfg, P)
        ng = 3
        jp = [ng, ng + cfg["n2"]]  # the axis faces
        fB[1][:, jp, :] = 0.0
        dt = 0.5 * orc.cfl_dt(cfg, P)
        U2, P2, f2, _, _ = orc.step_face(cf, U, P, fB, dt)
        sl3, _, sl1 = inputs.interior(cfg)
        assert np.all(f2[1][sl3, jp, sl1] == 0.0)
        # and the torus field matches the cell field the torus state carries
        Pc = inputs.cell_field_from_faces(cfg, fB, P)
        sl = inputs.interior(cfg)
        for b in (5, 6):
            assert np.abs(Pc[b][sl] - P[b][sl]).max() <= 1e-12 * np.abs(P[b][sl]).max()
