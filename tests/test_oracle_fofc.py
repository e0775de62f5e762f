"""Pins for the oracle's first-order flux correction (the paper's "Algorithm"
section; Beckwith & Stone 2011): a trial update with the high-order fluxes
flags the zones whose inversion fails or whose floors act; the faces of the
flagged zones take the donor-cell LLF flux; polar zeroing and Flux-CT run
again. Pinned by what the scheme fixes independently of its code:
  * no zone flagged -> the stage is the plain stage, bit for bit;
  * every zone flagged -> every face is first order: the stage is the plain
    stage with donor-cell reconstruction, bit for bit;
  * the flagged zones are the zones the plain stage floors or fails to invert
    (the trial is that stage's update);
  * the correction is local: zones farther than two (face-adjacent) steps
    from a flagged zone are untouched;
  * Flux-CT still holds on the corrected fluxes: the corner divergence of B
    is unchanged by the stage, zone by zone.
"""
import numpy as np
from scipy.ndimage import binary_dilation

from paper_2408_01361_gb300 import inputs


def _box(recon="weno5", n=8, seed=3, rho_min=1e-20):
    cfg = inputs.linear_mode_cfg(n, ndim=3, recon=recon)
    cfg = dict(cfg, floors=dict(rho_min=rho_min, u_min=1e-20))
    rng = np.random.default_rng(seed)
    P = np.zeros(inputs.shape(cfg))
    P[0] = 1.0 + 0.1 * rng.random(P[0].shape)
    P[1] = 1.0 + 0.1 * rng.random(P[1].shape)
    P[2:5] = 0.1 * rng.normal(size=P[2:5].shape)
    P[5:] = 0.5 * rng.normal(size=P[5:].shape)
    return cfg, P


def _stage(orc, cfg, U, P, cdt):
    Uo, Po = U.copy(), P.copy()
    _, st = orc.stage(cfg, U, P, cdt, Uo, Po)
    return Uo, Po, st, orc.last_nfofc


def _prepared(orc, cfg, P):
    P = orc.apply_bc(cfg, P)
    return orc.prim_to_cons(cfg, P), P


def test_no_flag_is_the_plain_stage(orc):
    cfg, P = _box()
    U, P = _prepared(orc, cfg, P)
    cdt = 0.5 * 0.3 / 8
    Ua, Pa, sa, _ = _stage(orc, cfg, U, P, cdt)
    Ub, Pb, sb, nf = _stage(orc, dict(cfg, fofc=True), U, P, cdt)
    assert nf == 0 and sa == sb
    assert np.array_equal(Ua, Ub) and np.array_equal(Pa, Pb)


def test_all_flagged_is_the_donor_cell_stage(orc):
    # rho_min above every density: every trial zone floors
    cfg, P = _box(rho_min=10.0)
    U, P = _prepared(orc, cfg, P)
    cdt = 0.5 * 0.3 / 8
    Ub, Pb, sb, nf = _stage(orc, dict(cfg, fofc=True), U, P, cdt)
    assert nf == 8**3
    Ud, Pd, sd, _ = _stage(orc, dict(cfg, recon="donor"), U, P, cdt)
    assert sb == sd
    assert np.array_equal(Ub, Ud) and np.array_equal(Pb, Pd)
    # and differs from the high-order stage
    Uh, _, _, _ = _stage(orc, cfg, U, P, cdt)
    assert not np.array_equal(Uh, Ub)


def test_flags_are_the_plain_stage_interventions_and_correction_is_local(orc):
    cfg, P = _box(rho_min=1.05)
    U, P = _prepared(orc, cfg, P)
    cdt = 0.5 * 0.3 / 8
    cf = dict(cfg, fofc=True)
    flags = orc.fofc_flags(cf, U, P, cdt)
    Ua, Pa, sa, _ = _stage(orc, cfg, U, P, cdt)
    Ub, Pb, sb, nf = _stage(orc, cf, U, P, cdt)
    n = int(flags.sum())
    # every zone the plain stage fails to invert or floors is flagged, nothing else
    assert 0 < n < 8**3
    assert nf == n == sa[0] + sa[1]
    # the plain stage's floored zones are the zones its floors changed: their
    # density sits at rho_min exactly
    sl = inputs.interior(cfg)
    assert np.array_equal(flags[sl] > 0, Pa[0][sl] == 1.05)
    changed = (Ua != Ub).any(axis=0)[sl] | (Pa != Pb).any(axis=0)[sl]
    # the box is periodic: distances wrap
    near = binary_dilation(np.pad(flags[sl] > 0, 2, mode="wrap"), iterations=2)[2:-2, 2:-2, 2:-2]
    assert changed.any()
    assert not (changed & ~near).any()


def test_flux_ct_holds_on_the_corrected_fluxes(orc):
    for rho_min in (1.05, 10.0):
        cfg, P = _box(rho_min=rho_min)
        U, P = _prepared(orc, cfg, P)
        cf = dict(cfg, fofc=True)
        _, _, d0 = orc.divb(cf, P, field=True)
        _, Pb, _, nf = _stage(orc, cf, U, P, 0.5 * 0.3 / 8)
        assert nf > 0
        _, _, d1 = orc.divb(cf, orc.apply_bc(cf, Pb), field=True)
        sl = inputs.interior(cfg)
        assert np.abs(d1[sl] - d0[sl]).max() < 1e-12 * np.abs(d0[sl]).max()


def test_fofc_step_on_a_torus_flags_the_atmosphere(orc):
    cfg = inputs.torus_cfg(48, 32, 1, r_out=60.0, recon="weno5")
    P = orc.apply_bc(cfg, inputs.torus_state(cfg, seed=2))
    U = orc.prim_to_cons(cfg, P)
    a = orc.step(cfg, U, P, 1e-2)
    b = orc.step(dict(cfg, fofc=True), U, P, 1e-2)
    # the atmosphere sits at its floors: both stages flag zones there
    assert orc.last_nfofc > 0 and a[3][1] > 0
    assert np.isfinite(b[0]).all() and np.isfinite(b[1]).all()
    assert not np.array_equal(a[1], b[1])
