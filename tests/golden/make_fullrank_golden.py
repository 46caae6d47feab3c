"""Writes the expected values of the paper's dense-limit Gaussian rows (Sec. 5: the
three-dimensional column of the Gaussian table, C_ij = 2 delta_ij + exp(-|r_i - r_j|^2),
points uniform in [-3, 3]^3, n = 10 000; the d-dimensional table, points uniform in
[-3, 3]^4, n = 5000) from the oracle alone: log det C, y^T C^-1 y and the largest ACA rank
of every level, for leaf size 128 and eps = 1e-12. The oracle needs several minutes (d = 4)
to about an hour (d = 3) of host time, too long for a test, so the GPU tests read these
files. Run from the repository root:

    python tests/golden/make_fullrank_golden.py d4
    python tests/golden/make_fullrank_golden.py d3
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1403_6015_gb300 import inputs as I  # noqa: E402

# exp(-r^2) is the squared-exponential exp(-r^2 / (2 ell^2)) with ell = 1 / sqrt(2)
ELL = 1.0 / np.sqrt(2.0)
S2 = 2.0
LEAF = 128
EPS = 1e-12
CASES = {
    # name: (n, d, seed, source)
    "d4": (5000, 4, 2004, "Sec. 5, d-dimensional Gaussian table (unscaled cube), row d = 4"),
    "d3": (10000, 3, 2003, "Sec. 5, Gaussian table, three-dimensional data, row n = 10,000"),
}


def main(name):
    n, d, seed, src = CASES[name]
    x = I.uniform_points(n, d, -3.0, 3.0, seed)
    y = I.normal(n, seed + 1)
    t0 = time.time()
    o = O.Hodlr(x, "se", [ELL, 1.0], S2, LEAF, EPS, max_rank=n // 2)
    sol = o.factor_solve(y)
    ld = o.logdet()
    ranks = o.ranks()
    lv = [int(ranks[(1 << j) - 1:(1 << (j + 1)) - 1].max()) for j in range(o.kappa)]
    out = {
        "source": src,
        "n": n, "d": d, "seed_points": seed, "seed_y": seed + 1,
        "box": [-3.0, 3.0], "kernel": "se", "ell": ELL, "amp": 1.0, "sigma2": S2,
        "leaf": LEAF, "eps": EPS, "kappa": int(o.kappa),
        "logdet": float(ld), "quad": float(y @ sol), "level_max_rank": lv,
        "oracle_seconds": round(time.time() - t0, 1),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"fullrank_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path, out)


if __name__ == "__main__":
    main(sys.argv[1])
