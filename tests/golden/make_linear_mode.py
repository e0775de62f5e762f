"""Write linear_slow_mode.txt, linear_alfven_mode.txt and linear_fast_mode.txt:
the eigenvectors of the linear mode tests, derived from the oracle's flux
Jacobians.

Background (Minkowski, at rest): rho = 1, u = 1, B = (1, 0, 0), gamma = 4/3;
wave vector k = (2 pi, 2 pi, 0). The primitive-form system
dP/dt + (dU/dP)^-1 (k1 dF1/dP + k2 dF2/dP)/|k| dP/dx_k = 0 has real
eigenvalues (phase speeds): with the positive ones sorted, slow < Alfven <
fast. The slow and fast eigenvectors are normalised to d rho = 1, the
Alfven one (no density perturbation) to d B^3 = 1; omega = speed * |k|.

Calls only oracle/ (run: python tests/golden/make_linear_mode.py).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

P0 = np.array([1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0])
K = np.array([2.0 * np.pi, 2.0 * np.pi, 0.0])
GAM = 4.0 / 3.0


def primitive_matrix():
    eta = np.diag([-1.0, 1.0, 1.0, 1.0])
    dF1, dU = oracle.point_jacobians(GAM, eta, P0, 1)
    dF2, _ = oracle.point_jacobians(GAM, eta, P0, 2)
    kn = K / np.linalg.norm(K)
    return np.linalg.solve(dU, kn[0] * dF1 + kn[1] * dF2)


def mode(rank: int, norm_slot: int):
    """The eigenvector of the rank-th smallest positive speed (0 slow, 1
    Alfven, 2 fast), normalised to 1 in slot norm_slot."""
    A = primitive_matrix()
    lam, vec = np.linalg.eig(A)
    lam = lam.real
    pos = sorted((q for q in range(8) if lam[q] > 1e-8), key=lambda i: lam[i])
    q = pos[rank]
    v = vec[:, q].real
    v = v / v[norm_slot]
    v[(np.abs(v) > 0.0) & (np.abs(v) < 1e-12)] = 0.0  # round-off in slots the mode leaves at rest
    return v, lam[q] * np.linalg.norm(K), np.sort(lam)


def slow_mode():
    return mode(0, 0)


NAMES = {"slow": ("Slow magnetosonic", 0, 0, "drho=1"), "alfven": ("Alfven", 1, 7, "dB3=1"),
         "fast": ("Fast magnetosonic", 2, 0, "drho=1")}

if __name__ == "__main__":
    for key, (title, rank, slot, normtxt) in NAMES.items():
        v, omega, lam = mode(rank, slot)
        out = os.path.join(HERE, f"linear_{key}_mode.txt")
        with open(out, "w") as f:
            f.write(f"# {title} eigenvector of the linear-mode test (written by make_linear_mode.py,\n")
            f.write("# from the oracle's flux Jacobians). Background rho=1 u=1 B=(1,0,0), gamma=4/3,\n")
            f.write(f"# Minkowski, k=(2pi,2pi,0); dP normalised to {normtxt}; "
                    "P = P0 + amp dP cos(k.x - omega t).\n")
            f.write("dP = " + " ".join(f"{x:.17e}" for x in v) + "\n")
            f.write(f"omega = {omega:.17e}\n")
            f.write("speeds = " + " ".join(f"{x:.17e}" for x in lam) + "\n")
        print(open(out).read())
