"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare with the oracle on the same seeded inputs."""
import numpy as np

from paper_2408_01361_gb300 import inputs

TOL = 1e-10  # relative L1 per variable (FP64 path vs FP64 oracle)


def rel_l1(a, b):
    """Per-variable relative L1 over the given arrays (shape (nvar, ...))."""
    out = []
    for v in range(a.shape[0]):
        num = np.abs(a[v] - b[v]).sum()
        den = np.abs(b[v]).sum()
        out.append(num / den if den > 0 else num)
    return np.array(out)


# Element-wise bound of the FP64 path: |a - b| <= ELEM_TOL * max(|b|, 1e-3 max|b_v|)
# at every interior cell (see elem_err). The FP64 path's element-wise
# differences from the oracle are set by the conditioning of tenuous,
# magnetised zones (the inversion there amplifies rounding ~100-fold) and by
# WENO5 weights on near-flat data: ~1e-8 at most after 10 torus steps.
ELEM_TOL = 5e-8
ELEM_SCALE = 1e-3


def elem_err(a, b, frac=ELEM_SCALE):
    """Per-variable max over cells of |a - b| / max(|b|, frac * max|b_v|): the
    relative error of each cell, measured against a thousandth of the
    variable's largest magnitude where the variable itself is smaller (momenta,
    velocities and field components cross zero, where a relative error has no
    meaning). A single cell off by 1e-4 of itself fails a 5e-8 bound unless
    it is below 5e-7 of the variable's largest magnitude."""
    out = []
    for v in range(a.shape[0]):
        s = frac * np.abs(b[v]).max()
        den = np.maximum(np.abs(b[v]), s if s > 0 else np.finfo(np.float64).tiny)
        out.append(float((np.abs(a[v] - b[v]) / den).max()))
    return np.array(out)


def assert_fp64_parity(a, b, what=""):
    """The FP64 bar: relative L1 per variable <= TOL and the element-wise
    bound ELEM_TOL."""
    e1, ee = rel_l1(a, b), elem_err(a, b)
    assert e1.max() < TOL, (what, "rel L1", e1)
    assert ee.max() < ELEM_TOL, (what, "element-wise", ee)


def interior(cfg, A):
    return A[(slice(None),) + inputs.interior(cfg)]


class GpuRun:
    """Device copies of a state for one context."""

    def __init__(self, ctx, cfg, P, U=None, dirichlet=None):
        self.ctx, self.cfg = ctx, cfg
        self.N1 = P.shape[3]
        self.PB = ctx.to_device(P)
        self.P, self.B = ctx.split(self.PB)
        self.U = ctx.empty(8)
        if U is None:
            ctx.prim_to_cons(self.P, self.B, self.U)
        else:
            self.U.copy_(ctx.to_device(U))
        if dirichlet is not None:
            for face, D in enumerate(dirichlet):
                if D is not None:
                    ctx.set_dirichlet(face, ctx.torch.from_numpy(np.ascontiguousarray(D)).to(ctx.device))

    def host(self):
        return self.ctx.to_host(self.U, self.N1), self.ctx.to_host(self.PB, self.N1)
