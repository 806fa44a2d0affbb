"""Writes homogeneous.json: closed-form macroscopic stresses of the void-free
(f = 0) lattice, where every field is uniform and the augmented-Lagrangian
iteration is exact after one step.  Two material sets:

  baseline : lambda = 1.5, mu = 1 (nu = 0.3), Y = 1
  paper    : K = 1, mu = 0.4, Y = 0.5 (arXiv:0802.2488, Sec. 2, the values
             used for all computations of the paper), lambda = K - 2 mu / 3.

Derivation (3D deviator, plane strain E33 = 0, K = lambda + 2 mu / 3):
  equibiaxial E11 = E22 = e: tr = 2e, dev = e (1/3, 1/3, -2/3, 0),
    |dev| = e sqrt(6) / 3; first yield where 2 mu |dev| = sqrt(2/3) Y,
    i.e. e_y = Y / (2 mu).
    elastic: s11 = s22 = 2 (lambda + mu) e,  s33 = 2 lambda e
    plastic: s11 = s22 = 2 K e + Y / 3,      s33 = 2 K e - 2 Y / 3
  shear E12 = g: tr = 0, |dev| = sqrt(2) g; g_y = Y / (2 sqrt(3) mu).
    elastic: s12 = 2 mu g;  plastic: s12 = Y / sqrt(3); other components 0.
Nothing here calls the oracle or the CUDA path.
"""
import json
import math
import os


def cases(lam, mu, Y):
    K = lam + 2 * mu / 3
    ey, gy = Y / (2 * mu), Y / (2 * math.sqrt(3) * mu)
    out = {"lambda": lam, "mu": mu, "Y": Y, "equibiaxial_yield": ey, "shear_yield": gy,
           "equibiaxial": [], "shear": []}
    for r in (0.5, 1 - 1e-9, 1 + 1e-9, 1.5, 2.0):
        e = r * ey
        if r < 1:
            s = [2 * (lam + mu) * e, 2 * (lam + mu) * e, 2 * lam * e, 0.0]
        else:
            s = [2 * K * e + Y / 3, 2 * K * e + Y / 3, 2 * K * e - 2 * Y / 3, 0.0]
        out["equibiaxial"].append({"E": [e, e, 0.0, 0.0], "sigma": s, "plastic": r > 1})
        g = r * gy
        s = [0.0, 0.0, 0.0, 2 * mu * g if r < 1 else Y / math.sqrt(3)]
        out["shear"].append({"E": [0.0, 0.0, 0.0, g], "sigma": s, "plastic": r > 1})
    return out


if __name__ == "__main__":
    data = {
        "source": "closed forms derived in make_homogeneous.py; paper constants from "
                  "arXiv:0802.2488 Sec. 2 (K = 1, mu = 0.4, Y = 0.5)",
        "baseline": cases(1.5, 1.0, 1.0),
        "paper": cases(1.0 - 2 * 0.4 / 3, 0.4, 0.5),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "homogeneous.json"), "w") as fh:
        json.dump(data, fh, indent=1)
