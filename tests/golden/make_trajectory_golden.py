"""Write the FP64 oracle's 100-step trajectory of the broadband vacuum
workload (256^3 periodic grid, 4 x 4 x 4 subdomains of 64^3 with 16 guards,
order 64) at sampled cells, for the full-size FP32 trajectory test.

Calls only oracle/ (the local-FFT push of Sec. 3.2 with Eq. 1 of Sec. 3.1,
guards refilled from their owners every step as in Fig. 3) and the shared
seeded input generator.  The samples are the same pseudo-random cells for
every component (numpy PCG64, seed 1707).  Usage:
    python tests/golden/make_trajectory_golden.py [steps]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import psatd_oracle as O  # noqa: E402
from paper_1707_08500_gb300 import inputs as I  # noqa: E402

NSAMPLE = 2048
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "broadband256_trajectory.txt")


def sample_cells(shape_zyx, n, seed=1707):
    rng = np.random.default_rng(seed)
    flat = rng.choice(int(np.prod(shape_zyx)), size=n, replace=False)
    return np.stack(np.unravel_index(np.sort(flat), shape_zyx), axis=1)


def main(steps=100):
    wl = I.workload("broadband256")
    g = {k: v.numpy() for k, v in I.global_fields(wl).items()}
    nx, ny, nz = wl.global_n
    cells = sample_cells((nz, ny, nx), NSAMPLE)
    t0 = time.time()
    for s in range(steps):
        g = O.step(g, wl)
        print(f"step {s + 1}/{steps}  {time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle (Sec. 3.2 local-FFT push with Eq. 1 of Sec. 3.1; guard refill of Fig. 3)\n")
        f.write(f"# workload broadband256 after {steps} steps; {NSAMPLE} sampled cells (numpy PCG64 seed 1707)\n")
        f.write("# columns: z y x Ex Ey Ez Bx By Bz\n")
        f.write(f"steps {steps}\n")
        for z, y, x in cells:
            vals = " ".join(f"{g[n][z, y, x]:.17e}" for n in O.EB)
            f.write(f"{z} {y} {x} {vals}\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 100)
