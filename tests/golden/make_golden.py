"""Writes the stored expected values under tests/golden/ by calling only the
CPU oracle (and the seeded input generator). Run from the repo root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import hamiltonian, twist  # noqa: E402
from paper_2203_09732_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def l12():
    L, h, seed, K = 12, 3.0, 0, 10
    hv = inputs.disorder(L, h, seed)
    H, diag, st = hamiltonian.build(L, hv)
    w, V = np.linalg.eigh(H.toarray())
    sigma = 0.5 * (w[0] + w[-1])
    order = np.lexsort((w, np.abs(w - sigma)))[:K]
    z = twist.overlap(V[:, order], st, L)
    with open(os.path.join(HERE, "l12_config.txt"), "w") as f:
        f.write("# L=12, h=3, seed 0 (numpy default_rng(0).uniform(-3,3,12)); dense eigh (oracle)\n")
        f.write("h " + " ".join(repr(float(x)) for x in hv) + "\n")
        f.write(f"sigma {float(sigma)!r}\n")
        f.write(f"emin {float(w[0])!r}\nemax {float(w[-1])!r}\n")
        for i, k in enumerate(order):
            f.write(f"eig {float(w[k])!r} zabs2 {float(abs(z[i])**2)!r}\n")


if __name__ == "__main__":
    l12()
