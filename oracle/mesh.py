"""Statically refined mesh on the oracle (test infrastructure only).

A mesh is a base configuration (its n1, n2, n3 the level-0 grid) plus blocks
(level, first interior cell i0, j0, k0 in level indices, sizes n1, n2, n3);
level l is 2^l times finer (x3 only when the problem is 3-D). Each block is a
grid of its own, stepped by the oracle's single-stage routine after its
ghost zones are filled here, cell by cell, from the block that owns the
ghost cell's centre:

* the centre is first carried through the physical boundaries: outflow in x1
  moves it to the centre of the first (last) interior cell of its level and
  forbids inflow through u~1; polar x2 reflects it across the axis and flips
  u~2 and B2; periodic directions wrap;
* the owner at the same level gives its cell's value; a coarser owner gives
  its cell's value plus MC-limited slopes times the +-1/4 offset of the fine
  centre; a finer owner gives the mean of its 2x2(x2) cells covering the
  ghost cell;
* a slope in one direction takes the coarse-level values at the centres one
  coarse cell below and above: the value of the cell there if a block at the
  coarse level owns it, the mean of the covering cells if a block one level
  finer owns it; the slope is zero if either centre lies past a non-periodic
  edge of the domain or inside a still coarser block.

Every block takes the same dt; there is no flux correction at level
interfaces. step advances every block with the predictor-corrector, step_rk
with a Runge-Kutta integrator (each stage's input ghost-filled across blocks
before the blocks' stages). With the first-order flux correction each stage
first runs every block's trial, then fills the flags' ghost cells across
blocks by the same map (a copied or prolonged ghost takes its source cell's
flag, a restricted one the largest of the fine cells'), and corrects the
faces of the flagged zones of every block from those flags. Written from positions in floating point, independently of the
CUDA library's integer map.

With face-centred constrained transport (step_face) every block also
carries its face field; after each block's edge EMFs are computed, an edge
of a coarse block that lies on the surface of a block one level finer takes
the fine block's EMF there (the mean of the two fine edges along it where
the edge's own direction is refined), so that the coarse face on the
interface moves exactly as the mean of the fine faces covering it and the
face divergence stays zero on both sides. (Interfaces across a periodic
domain edge are not matched; the layouts here have none.)
"""
from __future__ import annotations

import math

import numpy as np

from . import face_emfs, fofc_flags, rk_table, stage, stage_face

NV = 8


def _mc(qm, q0, qp):
    dm, dp = q0 - qm, qp - q0
    if dm * dp <= 0.0:
        return 0.0
    cand = (2.0 * dm, 2.0 * dp, 0.5 * (dm + dp))
    s = cand[0]
    for c in cand[1:]:
        if abs(c) < abs(s):
            s = c
    return s


class OracleMesh:
    def __init__(self, base: dict, blocks: list, block_cfg):
        self.base = base
        self.blocks = blocks
        self.cfgs = [block_cfg(base, b) for b in blocks]
        self.ng = base.get("ng", 3)
        self.ndim = 3 if base["n3"] > 1 else 2
        self.dom = [base["x1"], base["x2"], base["x3"]]

    # ---- geometry of a block ----
    def _dx(self, b):
        c = self.cfgs[b]
        return [(c[k][1] - c[k][0]) / c[n] for k, n in (("x1", "n1"), ("x2", "n2"), ("x3", "n3"))]

    def _origin(self, b):
        c = self.cfgs[b]
        return [c["x1"][0], c["x2"][0], c["x3"][0]]

    def _ng(self, d):
        return self.ng if (d < 2 or self.ndim == 3) else 0

    def _owner(self, x):
        for b, c in enumerate(self.cfgs):
            ok = True
            for d, key in enumerate(("x1", "x2", "x3")):
                if d == 2 and self.ndim == 2:
                    continue
                lo, hi = c[key]
                if not (lo < x[d] < hi):
                    ok = False
                    break
            if ok:
                return b
        raise ValueError(f"no block owns {x}")

    def _cell(self, b, x):
        """(local array index per direction) of block b's cell containing x."""
        o, dx = self._origin(b), self._dx(b)
        return [int(math.floor((x[d] - o[d]) / dx[d])) + self._ng(d) if (d < 2 or self.ndim == 3) else 0
                for d in range(3)]

    def _transform(self, b, x):
        bc = self.base["bc"]
        dx = self._dx(b)
        flip = False
        clamp = 0
        (a1, b1), (a2, b2), (a3, b3) = self.dom
        if x[0] < a1:
            if bc[0] == "periodic":
                x[0] += b1 - a1
            else:
                x[0], clamp = a1 + 0.5 * dx[0], 1
        elif x[0] > b1:
            if bc[1] == "periodic":
                x[0] -= b1 - a1
            else:
                x[0], clamp = b1 - 0.5 * dx[0], 2
        if x[1] < a2:
            if bc[2] == "polar":
                x[1], flip = 2 * a2 - x[1], not flip
            elif bc[2] == "periodic":
                x[1] += b2 - a2
            else:
                x[1] = a2 + 0.5 * dx[1]
        elif x[1] > b2:
            if bc[3] == "polar":
                x[1], flip = 2 * b2 - x[1], not flip
            elif bc[3] == "periodic":
                x[1] -= b2 - a2
            else:
                x[1] = b2 - 0.5 * dx[1]
        if self.ndim == 3:
            if x[2] < a3:
                x[2] = x[2] + (b3 - a3) if bc[4] == "periodic" else a3 + 0.5 * dx[2]
            elif x[2] > b3:
                x[2] = x[2] - (b3 - a3) if bc[5] == "periodic" else b3 - 0.5 * dx[2]
        return x, flip, clamp

    def _mean_fine(self, s, x, Ps):
        """Mean of block s's cells covering the cell twice their size centred at x."""
        dxs = self._dx(s)
        acc = np.zeros(NV)
        cnt = 0
        for a3 in ((-0.5, 0.5) if self.ndim == 3 else (0.0,)):
            for a2 in (-0.5, 0.5):
                for a1 in (-0.5, 0.5):
                    y = [x[0] + a1 * dxs[0], x[1] + a2 * dxs[1], x[2] + a3 * dxs[2]]
                    ci = self._cell(s, y)
                    acc += Ps[s][:, ci[2], ci[1], ci[0]]
                    cnt += 1
        return acc / cnt

    def _coarse_value(self, level, cc, d, step, Ps):
        """Level-`level` value at the centre cc shifted by `step` along d, or None."""
        y = list(cc)
        y[d] += step
        lo, hi = self.dom[d]
        if not (lo < y[d] < hi):
            if self.base["bc"][2 * d + (0 if y[d] < lo else 1)] != "periodic":
                return None
            y[d] += (hi - lo) if y[d] < lo else -(hi - lo)
        w = self._owner(y)
        lw = self.blocks[w]["level"]
        if lw == level:
            ci = self._cell(w, y)
            return Ps[w][:, ci[2], ci[1], ci[0]]
        if lw == level + 1:
            return self._mean_fine(w, y, Ps)
        return None

    def fill_ghosts(self, Ps):
        """Fill every block's ghost cells in place (Ps: list of (8, N3, N2, N1))."""
        lev = [blk["level"] for blk in self.blocks]
        for b, P in enumerate(Ps):
            N3, N2, N1 = P.shape[1:]
            o, dx = self._origin(b), self._dx(b)
            g = [self._ng(0), self._ng(1), self._ng(2)]
            n = [self.cfgs[b]["n1"], self.cfgs[b]["n2"], self.cfgs[b]["n3"]]
            for k in range(N3):
                for j in range(N2):
                    for i in range(N1):
                        idx = (i, j, k)
                        if all(g[d] <= idx[d] < g[d] + n[d] for d in range(3)):
                            continue
                        x = [o[d] + (idx[d] - g[d] + 0.5) * dx[d] for d in range(3)]
                        if self.ndim == 2:
                            x[2] = 0.5 * sum(self.dom[2])
                        x, flip, clamp = self._transform(b, x)
                        s = self._owner(x)
                        Q = Ps[s]
                        dl = lev[s] - lev[b]
                        if dl == 0:
                            ci = self._cell(s, x)
                            val = Q[:, ci[2], ci[1], ci[0]].copy()
                        elif dl == -1:
                            ci = self._cell(s, x)
                            os_, dxs = self._origin(s), self._dx(s)
                            gs = [self._ng(0), self._ng(1), self._ng(2)]
                            q0 = Q[:, ci[2], ci[1], ci[0]]
                            val = q0.copy()
                            cc = [os_[d] + (ci[d] - gs[d] + 0.5) * dxs[d] for d in range(3)]
                            for d in range(self.ndim):
                                sgn = 1.0 if x[d] > cc[d] else -1.0
                                qm = self._coarse_value(lev[s], cc, d, -dxs[d], Ps)
                                qp = self._coarse_value(lev[s], cc, d, +dxs[d], Ps)
                                if qm is None or qp is None:
                                    continue
                                for v in range(NV):
                                    val[v] += 0.25 * sgn * _mc(qm[v], q0[v], qp[v])
                        elif dl == 1:
                            val = self._mean_fine(s, x, Ps)
                        else:
                            raise ValueError("blocks more than one level apart")
                        if flip:
                            val[3] = -val[3]
                            val[6] = -val[6]
                        if clamp == 1 and val[2] > 0.0:
                            val[2] = 0.0
                        if clamp == 2 and val[2] < 0.0:
                            val[2] = 0.0
                        P[:, k, j, i] = val

    def fill_flag_ghosts(self, Fs):
        """The flux correction's flags in every block's ghost cells (Fs: list
        of int (N3, N2, N1), interior flags set), by the ghost map of the
        state: a ghost cell takes the flag of the cell whose value it copies,
        of the coarse cell it is prolonged from, or the largest flag of the
        fine cells whose mean it takes."""
        lev = [blk["level"] for blk in self.blocks]
        for b, F in enumerate(Fs):
            N3, N2, N1 = F.shape
            o, dx = self._origin(b), self._dx(b)
            g = [self._ng(0), self._ng(1), self._ng(2)]
            n = [self.cfgs[b]["n1"], self.cfgs[b]["n2"], self.cfgs[b]["n3"]]
            for k in range(N3):
                for j in range(N2):
                    for i in range(N1):
                        idx = (i, j, k)
                        if all(g[d] <= idx[d] < g[d] + n[d] for d in range(3)):
                            continue
                        x = [o[d] + (idx[d] - g[d] + 0.5) * dx[d] for d in range(3)]
                        if self.ndim == 2:
                            x[2] = 0.5 * sum(self.dom[2])
                        x, _, _ = self._transform(b, x)
                        s = self._owner(x)
                        dl = lev[s] - lev[b]
                        if dl in (0, -1):
                            ci = self._cell(s, x)
                            F[k, j, i] = Fs[s][ci[2], ci[1], ci[0]]
                        elif dl == 1:
                            dxs = self._dx(s)
                            f = 0
                            for a3 in ((-0.5, 0.5) if self.ndim == 3 else (0.0,)):
                                for a2 in (-0.5, 0.5):
                                    for a1 in (-0.5, 0.5):
                                        ci = self._cell(s, [x[0] + a1 * dxs[0], x[1] + a2 * dxs[1],
                                                            x[2] + a3 * dxs[2]])
                                        f = max(f, int(Fs[s][ci[2], ci[1], ci[0]]))
                            F[k, j, i] = f
                        else:
                            raise ValueError("blocks more than one level apart")

    def _stage_all(self, U0s, Pins, cdt, Uouts, Pouts, dUs=None):
        """One stage of every block (Pins ghost-filled); with the flux
        correction (base "fofc") the flags of all blocks' trials first, their
        ghosts filled across blocks. Returns (ctops, summed stats)."""
        flags = [None] * len(Pins)
        if self.base.get("fofc"):
            flags = [fofc_flags(self.cfgs[b], U0s[b], Pins[b], cdt) for b in range(len(Pins))]
            self.fill_flag_ghosts(flags)
        tot, cts = [0, 0, 0], []
        for b in range(len(Pins)):
            ct, st = stage(self.cfgs[b], U0s[b], Pins[b], cdt, Uouts[b], Pouts[b],
                           dU=None if dUs is None else dUs[b], fofc_flags=flags[b])
            cts.append(ct)
            tot = [x + y for x, y in zip(tot, st)]
        return cts, tot

    def cfl_dt(self, cts):
        """cfl / max over all blocks' zones of sum_d max(ctop faces)/dx_d."""
        mx = 0.0
        for b, ct in enumerate(cts):
            c = self.cfgs[b]
            g = [self._ng(0), self._ng(1), self._ng(2)]
            n = [c["n1"], c["n2"], c["n3"]]
            dx = self._dx(b)
            sl = (slice(g[2], g[2] + n[2]), slice(g[1], g[1] + n[1]), slice(g[0], g[0] + n[0]))
            inv = np.zeros((n[2], n[1], n[0]))
            for d in range(self.ndim):
                lo = ct[d][sl]
                shift = [0, 0, 0]
                shift[d] = 1
                sh = tuple(slice(s_.start + shift[2 - q], s_.stop + shift[2 - q]) for q, s_ in enumerate(sl))
                hi = ct[d][sh]
                inv += np.maximum(lo, hi) / dx[d]
            mx = max(mx, inv.max())
        return self.base.get("cfl", 0.9) / mx

    def step(self, Us, Ps, dt):
        """One two-stage step of every block; returns (Us, Ps, dt_cfl, stats)."""
        Pn = [np.array(P, copy=True) for P in Ps]
        U0 = [np.array(U, copy=True) for U in Us]
        self.fill_ghosts(Pn)
        Ps_ = [np.array(P, copy=True) for P in Pn]
        Us_ = [np.array(U, copy=True) for U in U0]
        _, tot = self._stage_all(U0, Pn, 0.5 * dt, Us_, Ps_)
        self.fill_ghosts(Ps_)
        Pout = [np.array(P, copy=True) for P in Pn]
        Uout = [np.array(U, copy=True) for U in U0]
        cts, t2 = self._stage_all(U0, Ps_, dt, Uout, Pout)
        tot = [a + c for a, c in zip(tot, t2)]
        return Uout, Pout, self.cfl_dt(cts), tot

    def step_rk(self, Us, Ps, dt, integrator):
        """One Runge-Kutta step ("rk1", "rk2" or "ssprk54") of every block:
        the stages of the oracle's single-grid Runge-Kutta step (its table,
        rk_table), each stage input's ghost zones filled across blocks before
        the blocks' stages; returns (Us, Ps, dt_cfl, stats)."""
        table = rk_table(integrator)
        nb = len(Us)
        Ust = [[np.array(U, copy=True) for U in Us]]
        Pst = [[np.array(P, copy=True) for P in Ps]]
        dU4 = [np.zeros_like(U) for U in Us]
        tot = [0, 0, 0]
        cts = []
        for s, (src, w, c, w4) in enumerate(table):
            Pin = Pst[s]
            self.fill_ghosts(Pin)
            keep = integrator == "ssprk54" and s == 3
            bases = []
            for b in range(nb):
                base = 0.0
                for t, a in zip(src, w):
                    base = base + a * Ust[t][b]
                if w4 != 0.0:
                    base = base + w4 * dU4[b]
                bases.append(base)
            Uout = [np.array(x, copy=True) for x in bases]
            Pout = [np.array(P, copy=True) for P in Pin]
            cts, st = self._stage_all(bases, Pin, c * dt, Uout, Pout, dU4 if keep else None)
            tot = [x + y for x, y in zip(tot, st)]
            Ust.append(Uout)
            Pst.append(Pout)
        return Ust[-1], Pst[-1], self.cfl_dt(cts), tot

    # ---- face-centred constrained transport ----
    def _edge_ranges(self, b, c):
        """Local index ranges (lo, hi inclusive) per direction of block b's
        edges along x^(c+1) that its interior faces need."""
        cfg = self.cfgs[b]
        n = (cfg["n1"], cfg["n2"], cfg["n3"])
        out = []
        for q in range(3):
            active = q < 2 or self.ndim == 3
            if not active:
                out.append((0, 0))
                continue
            g = self.ng
            out.append((g, g + n[q] - 1) if q == c else (g, g + n[q]))
        return out

    def _global(self, b, q, i):
        blk = self.blocks[b]
        o = (blk["i0"], blk["j0"], blk["k0"])[q]
        active = q < 2 or self.ndim == 3
        return o + i - self.ng if active else 0

    def _local(self, f, q, G):
        blk = self.blocks[f]
        o = (blk["i0"], blk["j0"], blk["k0"])[q]
        active = q < 2 or self.ndim == 3
        return G - o + self.ng if active else 0

    def emf_matches(self):
        """[(b, c, (k, j, i), f, [(k, j, i), ...])]: the coarse edges of block b
        on the surface of a block f one level finer, with the fine edges whose
        mean replaces them."""
        out = []
        for b, bb in enumerate(self.blocks):
            for f, fb in enumerate(self.blocks):
                if fb["level"] != bb["level"] + 1:
                    continue
                for c in range(3):
                    rb = self._edge_ranges(b, c)
                    rf = self._edge_ranges(f, c)
                    for k in range(rb[2][0], rb[2][1] + 1):
                        for j in range(rb[1][0], rb[1][1] + 1):
                            for i in range(rb[0][0], rb[0][1] + 1):
                                loc = (i, j, k)
                                fine = []
                                ok = True
                                for q in range(3):
                                    active = q < 2 or self.ndim == 3
                                    G = self._global(b, q, loc[q])
                                    if not active:
                                        fine.append([0])
                                    elif q == c:
                                        fine.append([self._local(f, q, 2 * G), self._local(f, q, 2 * G + 1)])
                                    else:
                                        fine.append([self._local(f, q, 2 * G)])
                                    for x in fine[-1]:
                                        if not (rf[q][0] <= x <= rf[q][1]):
                                            ok = False
                                if not ok:
                                    continue
                                cells = [(kk, jj, ii) for kk in fine[2] for jj in fine[1] for ii in fine[0]]
                                out.append((b, c, (k, j, i), f, cells))
        return out

    def _correct(self, Es, matches):
        for b, c, (k, j, i), f, cells in matches:
            Es[b][c][k, j, i] = sum(Es[f][c][kk, jj, ii] for kk, jj, ii in cells) / len(cells)

    def step_face(self, Us, Ps, fBs, dt):
        """One two-stage step with face-centred CT (every block's cfg has bfield
        "face"): returns (Us, Ps, fBs, dt_cfl, stats)."""
        matches = self.emf_matches()
        Pn = [np.array(P, copy=True) for P in Ps]
        U0 = [np.array(U, copy=True) for U in Us]
        f0 = [np.array(f, copy=True) for f in fBs]
        tot = [0, 0, 0]
        self.fill_ghosts(Pn)
        Ps_ = [np.array(P, copy=True) for P in Pn]
        Us_ = [np.array(U, copy=True) for U in U0]
        fs_ = [np.array(f, copy=True) for f in f0]
        Es = [face_emfs(self.cfgs[b], Pn[b]) for b in range(len(Pn))]
        self._correct(Es, matches)
        for b in range(len(Pn)):
            _, st = stage_face(self.cfgs[b], U0[b], Pn[b], 0.5 * dt, Es[b], f0[b], fs_[b], Us_[b], Ps_[b])
            tot = [a + c for a, c in zip(tot, st)]
        self.fill_ghosts(Ps_)
        Pout = [np.array(P, copy=True) for P in Pn]
        Uout = [np.array(U, copy=True) for U in U0]
        fout = [np.array(f, copy=True) for f in f0]
        Es = [face_emfs(self.cfgs[b], Ps_[b]) for b in range(len(Pn))]
        self._correct(Es, matches)
        cts = []
        for b in range(len(Pn)):
            ct, st = stage_face(self.cfgs[b], U0[b], Ps_[b], dt, Es[b], f0[b], fout[b], Uout[b], Pout[b])
            cts.append(ct)
            tot = [a + c for a, c in zip(tot, st)]
        return Uout, Pout, fout, self.cfl_dt(cts), tot
