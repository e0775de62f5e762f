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
