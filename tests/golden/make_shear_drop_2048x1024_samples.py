"""Write shear_drop_2048x1024_10000_samples.txt: the FP64 oracle's fields after 10000 steps of the
2048 x 1024 sheared drop (Sec. 4.4 set-up: drop between walls moving at +/-U, R = 160, Re = 1,
Ca = 0.2, Langmuir EOS E0 = 0.2, psi0 = 0.3), at seeded sample cells, plus the FP64 totals of phi
and psi.  Calls only the oracle and the input generators.  The unit normal is taken where
|grad phi| > 1e-4 (N_EPS): with n wherever grad phi is not zero, the far-bulk normal of a
single-precision run is set by rounding and 10000 steps would compare rounding histories, not
implementations.

    python tests/golden/make_shear_drop_2048x1024_samples.py [threads]

About 2.5 hours on 6 cores of a desktop CPU, 16 minutes on 16 Grace cores."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2408_15654_gb300 import workloads as W  # noqa: E402

STEPS = 10000
N_EPS = 1e-4
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "shear_drop_2048x1024_10000_samples.txt")


def sample_cells(phi0, seed=2408):
    """1024 cells uniform over the grid and 512 in the initial interface band 0.02 < phi < 0.98."""
    ny, nx = phi0.shape
    rng = np.random.default_rng(seed)
    flat = rng.choice(nx * ny, size=1024, replace=False)
    band = np.flatnonzero((phi0.ravel() > 0.02) & (phi0.ravel() < 0.98))
    band = rng.choice(band, size=512, replace=False)
    cells = np.unique(np.concatenate([flat, band]))
    return cells % nx, cells // nx


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    oracle.build()
    oracle.set_threads(threads)
    p, f = W.shear_drop_large()
    p = dict(p, n_eps=N_EPS)
    xs, ys = sample_cells(f["phi"])
    s = oracle.Sim(p)
    s.init(**f)
    t0 = time.time()
    for k in range(0, STEPS, 500):
        s.step(500)
        print(f"{k + 500} steps, {time.time() - t0:.0f} s", flush=True)
    m = s.moments()
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle, 2048 x 1024 sheared drop (workloads.shear_drop_large: Sec. 4.4 set-up), "
                 f"after {STEPS} steps\n")
        fh.write("# written by tests/golden/make_shear_drop_2048x1024_samples.py (oracle only)\n")
        fh.write(f"# steps {STEPS}\n")
        fh.write(f"# n_eps {N_EPS}\n")
        fh.write(f"# total_phi {s.total('phi'):.17g}\n")
        fh.write(f"# total_psi {s.total('psi'):.17g}\n")
        fh.write("# x y phi psi ux uy P\n")
        for x, y in zip(xs, ys):
            fh.write(f"{x} {y} " + " ".join(f"{m[k][y, x]:.17g}" for k in ("phi", "psi", "ux", "uy", "P")) + "\n")
    s.close()
    print("wrote", OUT, len(xs), "cells")


if __name__ == "__main__":
    main()
