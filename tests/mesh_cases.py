"""Refined-mesh layouts and states shared by the mesh tests. A block is
{level, i0, j0, k0, n1, n2, n3} in level-``level`` indices (level l is 2^l
times finer than the base grid)."""
import os

import numpy as np

from conftest import GOLDEN
from paper_2408_01361_gb300 import inputs


def blk(level, i0, j0, k0, n1, n2, n3):
    return dict(level=level, i0=i0, j0=j0, k0=k0, n1=n1, n2=n2, n3=n3)


def uneven_split(cfg, cuts1, cuts2, cuts3=None):
    """Level-0 blocks cutting the base grid at the given interior indices."""
    def segs(cuts, n):
        e = [0] + list(cuts) + [n]
        return list(zip(e[:-1], e[1:]))
    out = []
    s3 = segs(cuts3 or [], cfg["n3"]) if cfg["n3"] > 1 else [(0, 1)]
    for k0, k1 in s3:
        for j0, j1 in segs(cuts2, cfg["n2"]):
            for i0, i1 in segs(cuts1, cfg["n1"]):
                out.append(blk(0, i0, j0, k0, i1 - i0, j1 - j0, k1 - k0))
    return out


def slice_blocks(cfg, A, blocks):
    """Per-block arrays (ghosts included) cut from a single-grid array A whose
    ghosts already hold the boundary values (level-0 blocks only)."""
    ng = cfg.get("ng", 3)
    out = []
    for b in blocks:
        assert b["level"] == 0
        if cfg["n3"] > 1:
            ks = slice(b["k0"], b["k0"] + b["n3"] + 2 * ng)
        else:
            ks = slice(0, 1)
        out.append(np.ascontiguousarray(A[:, ks, b["j0"]:b["j0"] + b["n2"] + 2 * ng,
                                          b["i0"]:b["i0"] + b["n1"] + 2 * ng]))
    return out


def block_interior(base, b, A):
    return A[(slice(None),) + inputs.interior(inputs.block_cfg(base, b))]


def torus_base(n1=32, n2=24, recon="mc"):
    cfg = inputs.torus_cfg(n1, n2, 1, r_out=60.0, recon=recon)
    return cfg


def torus_two_level(recon="mc"):
    """2-D torus: level-0 polar caps, level-1 midplane band, uneven blocks."""
    base = torus_base(32, 24, recon)
    blocks = [blk(0, 0, 0, 0, 12, 6, 1), blk(0, 12, 0, 0, 20, 6, 1), blk(0, 0, 18, 0, 32, 6, 1),
              blk(1, 0, 12, 0, 24, 24, 1), blk(1, 24, 12, 0, 40, 24, 1)]
    return base, blocks


def torus_three_level(recon="weno5"):
    """2-D torus: level 0 at the poles, level 1 between, level 2 at the midplane."""
    base = torus_base(32, 32, recon)
    blocks = [blk(0, 0, 0, 0, 32, 4, 1), blk(0, 0, 28, 0, 32, 4, 1),
              blk(1, 0, 8, 0, 40, 12, 1), blk(1, 40, 8, 0, 24, 12, 1), blk(1, 0, 44, 0, 64, 12, 1),
              blk(2, 0, 40, 0, 56, 48, 1), blk(2, 56, 40, 0, 72, 48, 1)]
    return base, blocks


def box_two_level(n=16, recon="mc"):
    """3-D periodic Minkowski box, centre cube refined once, 6 level-0 slabs."""
    base = inputs.linear_mode_cfg(n, ndim=3, recon=recon)
    q, h = n // 4, n // 2
    blocks = [blk(0, 0, 0, 0, q, n, n), blk(0, n - q, 0, 0, q, n, n),
              blk(0, q, 0, 0, h, q, n), blk(0, q, n - q, 0, h, q, n),
              blk(0, q, q, 0, h, h, q), blk(0, q, q, n - q, h, h, q),
              blk(1, 2 * q, 2 * q, 2 * q, 2 * h, 2 * h, 2 * h)]
    return base, blocks


def torus_states(base, blocks, seed=2):
    norms = inputs.torus_norms(base)
    return [inputs.torus_state(inputs.block_cfg(base, b), seed=seed, norms=norms) for b in blocks]


def mode_states(base, blocks, amp=0.05):
    dP, om = inputs.load_eigvec(os.path.join(GOLDEN, "linear_slow_mode.txt"))
    return [inputs.linear_mode_state(inputs.block_cfg(base, b), dP, om, amp=amp) for b in blocks]
