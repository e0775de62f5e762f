"""Pins for the oracle's geometry (metric, inverse, determinant, connection).

The Kerr metric is pinned by the vacuum field equations: the Ricci tensor
built from the oracle's connection (derivatives of Gamma by central
differences) must vanish, in Kerr-Schild and in the MKS/FMKS native
coordinates. A wrong sign, a dropped term or a transposed Jacobian in the
metric or in the connection breaks Ricci-flatness.
"""
import math

import numpy as np
import pytest

from paper_2408_01361_gb300 import inputs

A = 0.9375


def _cfg(kind, a=A):
    c = inputs.torus_cfg(16, 16, 1, a=a)
    c["coords"] = kind
    if kind == "ks":
        c["x1"] = (1.5, 30.0)
        c["x2"] = (0.05, math.pi - 0.05)
    return c


def test_minkowski_flat(orc):
    cfg = inputs.linear_mode_cfg(8)
    gcov, gcon, gdet, alpha = orc.geometry(cfg, 0)
    assert np.array_equal(gcov[3, 3], np.diag([-1.0, 1.0, 1.0, 1.0]))
    assert np.all(gdet == 1.0) and np.all(alpha == 1.0)
    assert np.all(orc.connection(cfg) == 0.0)


@pytest.mark.parametrize("kind", ["ks", "mks", "fmks"])
def test_inverse_and_symmetry(orc, kind):
    cfg = _cfg(kind)
    for loc in range(5):
        gcov, gcon, gdet, alpha = orc.geometry(cfg, loc)
        prod = np.einsum("jiab,jibc->jiac", gcov, gcon)
        # rounding bound of a 4x4 product, relative to the entries' magnitudes
        scale = np.abs(gcov).max(axis=(2, 3)) * np.abs(gcon).max(axis=(2, 3))
        err = np.abs(prod - np.eye(4)).max(axis=(2, 3)) / scale
        assert err.max() < 1e-14
        assert np.abs(gcov - np.swapaxes(gcov, -1, -2)).max() == 0.0
    conn = orc.connection(cfg)
    assert np.abs(conn - np.swapaxes(conn, -1, -2)).max() < 1e-12 * np.abs(conn).max()


def test_ks_closed_forms(orc):
    """Kerr-Schild: sqrt(-g) = Sigma sin(theta), lapse = (1 + 2r/Sigma)^-1/2,
    g^rr = Delta/Sigma (zero on the horizon r+ = 1 + sqrt(1 - a^2))."""
    cfg = _cfg("ks")
    r = np.array([1.0 + math.sqrt(1 - A * A), 2.5, 7.0, 20.0])
    th = np.array([0.3, 1.1, 1.9, 2.8])
    gcov, gcon, gdet, _ = orc.metric_points(cfg, r, th)
    sig = r ** 2 + A ** 2 * np.cos(th) ** 2
    dl = r ** 2 - 2 * r + A ** 2
    assert np.allclose(gdet, sig * np.sin(th), rtol=1e-13)
    assert np.allclose(gcon[:, 1, 1], dl / sig, rtol=1e-12, atol=1e-14)
    assert abs(gcon[0, 1, 1]) < 1e-14
    assert np.allclose(1.0 / np.sqrt(-gcon[:, 0, 0]), 1.0 / np.sqrt(1 + 2 * r / sig), rtol=1e-13)


def test_mks_gdet_closed_form(orc):
    """MKS: sqrt(-g) = Sigma sin(theta) * r * dtheta/dx2, dtheta/dx2 = pi (1 + (1-h) cos 2 pi x2)."""
    cfg = _cfg("mks")
    h = cfg["hslope"]
    x1 = np.array([0.4, 1.2, 2.5, 5.0])
    x2 = np.array([0.1, 0.37, 0.5, 0.93])
    _, _, gdet, _ = orc.metric_points(cfg, x1, x2)
    r = np.exp(x1)
    th = np.pi * x2 + 0.5 * (1 - h) * np.sin(2 * np.pi * x2)
    sig = r ** 2 + A ** 2 * np.cos(th) ** 2
    want = sig * np.sin(th) * r * np.pi * (1 + (1 - h) * np.cos(2 * np.pi * x2))
    assert np.allclose(gdet, want, rtol=1e-13)


def test_fmks_map_endpoints(orc):
    """FMKS: theta(x2=0) = 0, theta(x2=1) = pi and theta(1/2) = pi/2 for any x1."""
    cfg = _cfg("fmks")
    x1 = np.array([0.3, 1.0, 4.0])
    r, th = orc.native_to_ks(cfg, x1, np.zeros(3))
    assert np.allclose(th, 0.0, atol=1e-14)
    r, th = orc.native_to_ks(cfg, x1, np.ones(3))
    assert np.allclose(th, np.pi, atol=1e-13)
    r, th = orc.native_to_ks(cfg, x1, np.full(3, 0.5))
    assert np.allclose(th, np.pi / 2, atol=1e-14)
    assert np.allclose(r, np.exp(x1), rtol=1e-15)


def _ricci(orc, cfg, x1, x2, h=1e-4):
    """R_mn = d_l G^l_mn - d_n G^l_ml + G^l_ls G^s_mn - G^l_ns G^s_ml (4th-order central differences)."""
    def conn(a, b):
        return orc.metric_points(cfg, np.array([a]), np.array([b]))[3][0]

    G = conn(x1, x2)
    dG = np.zeros((4, 4, 4, 4))  # dG[k] = d_k Gamma
    for k, (e1, e2) in ((1, (1, 0)), (2, (0, 1))):
        fp1 = conn(x1 + h * e1, x2 + h * e2); fm1 = conn(x1 - h * e1, x2 - h * e2)
        fp2 = conn(x1 + 2 * h * e1, x2 + 2 * h * e2); fm2 = conn(x1 - 2 * h * e1, x2 - 2 * h * e2)
        dG[k] = (8 * (fp1 - fm1) - (fp2 - fm2)) / (12 * h)
    R = np.zeros((4, 4))
    for m in range(4):
        for n in range(4):
            s = 0.0
            for l in range(4):
                s += dG[l][l, m, n] - dG[n][l, m, l]
                for q in range(4):
                    s += G[l, l, q] * G[q, m, n] - G[l, n, q] * G[q, m, l]
            R[m, n] = s
    return R, np.abs(G).max()


@pytest.mark.parametrize("kind,pts", [
    ("ks", [(3.0, 0.7), (8.0, 1.9), (1.9, 1.3)]),
    ("mks", [(1.0, 0.3), (2.2, 0.55), (0.6, 0.8)]),
    ("fmks", [(1.0, 0.3), (2.2, 0.55), (0.6, 0.08)]),
])
def test_ricci_flat(orc, kind, pts):
    cfg = _cfg(kind)
    for x1, x2 in pts:
        R, scale = _ricci(orc, cfg, x1, x2)
        assert np.abs(R).max() < 1e-7 * max(scale, 1.0) ** 2, (kind, x1, x2, np.abs(R).max())


def test_connection_matches_metric_derivatives(orc):
    """Gamma^l_mn vs 1/2 g^lk (d_m g_kn + d_n g_km - d_k g_mn) with the metric
    differentiated by central differences (independent of the oracle's duals)."""
    cfg = _cfg("fmks")
    x1, x2, h = 1.3, 0.41, 1e-5
    gcov, gcon, _, conn = orc.metric_points(cfg, np.array([x1]), np.array([x2]))
    dg = np.zeros((4, 4, 4))
    gp = orc.metric_points(cfg, np.array([x1 + h]), np.array([x2]))[0][0]
    gm = orc.metric_points(cfg, np.array([x1 - h]), np.array([x2]))[0][0]
    dg[1] = (gp - gm) / (2 * h)
    gp = orc.metric_points(cfg, np.array([x1]), np.array([x2 + h]))[0][0]
    gm = orc.metric_points(cfg, np.array([x1]), np.array([x2 - h]))[0][0]
    dg[2] = (gp - gm) / (2 * h)
    want = 0.5 * (np.einsum("lk,mkn->lmn", gcon[0], dg) + np.einsum("lk,nkm->lmn", gcon[0], dg)
                  - np.einsum("lk,kmn->lmn", gcon[0], dg))
    assert np.abs(conn[0] - want).max() < 1e-7 * np.abs(want).max()
