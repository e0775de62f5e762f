"""Write linear_slow_mode.txt: the slow magnetosonic eigenvector of the linear
mode test, derived from the oracle's flux Jacobians.

Background (Minkowski, at rest): rho = 1, u = 1, B = (1, 0, 0), gamma = 4/3;
wave vector k = (2 pi, 2 pi, 0). The primitive-form system
dP/dt + (dU/dP)^-1 (k1 dF1/dP + k2 dF2/dP)/|k| dP/dx_k = 0 has real
eigenvalues (phase speeds); the slow mode is the smallest positive one. Its
eigenvector is normalised to d rho = 1, and omega = speed * |k|.

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


def slow_mode():
    A = primitive_matrix()
    lam, vec = np.linalg.eig(A)
    lam = lam.real
    pos = [q for q in range(8) if lam[q] > 1e-8]
    q = min(pos, key=lambda i: lam[i])
    v = vec[:, q].real
    v = v / v[0]
    return v, lam[q] * np.linalg.norm(K), np.sort(lam)


if __name__ == "__main__":
    v, omega, lam = slow_mode()
    out = os.path.join(HERE, "linear_slow_mode.txt")
    with open(out, "w") as f:
        f.write("# Slow magnetosonic eigenvector of the linear-mode test (written by make_linear_mode.py,\n")
        f.write("# from the oracle's flux Jacobians). Background rho=1 u=1 B=(1,0,0), gamma=4/3,\n")
        f.write("# Minkowski, k=(2pi,2pi,0); dP normalised to drho=1; P = P0 + amp dP cos(k.x - omega t).\n")
        f.write("dP = " + " ".join(f"{x:.17e}" for x in v) + "\n")
        f.write(f"omega = {omega:.17e}\n")
        f.write("speeds = " + " ".join(f"{x:.17e}" for x in lam) + "\n")
    print(open(out).read())
