"""Write config3_oracle_<route>_500.txt: the CPU FP64 oracle's field after the
full 500-step run of the 3D workload (n = 256 per axis, alpha = (1.2, 1.5, 1.8),
eps = 0.08, tau = 2e-3, [-1, 1]^3, u0 ~ U[-1, 1] from seed 2), sampled at 4096
fixed points, with the full field's max |u|.

The oracle needs about 10 minutes (dense route) or an hour (spectral route) on
a CPU for this run, too long for a test, so the test suite compares the GPU
paths with these stored samples. Calls only the oracle and the seeded input
generator. Run from the repo root:
    python tests/golden/make_config3_reference.py dense
    python tests/golden/make_config3_reference.py spectral
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import sfac_inputs as I  # noqa: E402
from oracle import sfac_oracle as O  # noqa: E402

STEPS = 500
SAMPLES = 4096
INDEX_SEED = 33


def sample_indices(points):
    """4096 distinct flat indices (memory order, axis 1 fastest), drawn from
    SplitMix64 stream 33 and sorted; the first and last points are included."""
    raw = I.splitmix64(INDEX_SEED, 3 * SAMPLES) % np.uint64(points)
    idx = sorted({0, points - 1} | {int(v) for v in raw})
    return np.array(idx[:SAMPLES], dtype=np.int64)


def main():
    route = sys.argv[1] if len(sys.argv) > 1 else "dense"
    p = I.CONFIG3
    sch = O.Scheme.for_problem(p, route=route)
    u = np.array(I.config3_u0(), dtype=np.float64)
    t0 = time.time()
    for s in range(STEPS):
        u = sch.step(u)
        if (s + 1) % 50 == 0:
            print(f"{route}: step {s + 1} ({time.time() - t0:.0f} s)", flush=True)
    idx = sample_indices(p.points)
    flat = u.reshape(-1)
    path = os.path.join(HERE, f"config3_oracle_{route}_{STEPS}.txt")
    with open(path, "w") as f:
        f.write(f"# The oracle's FP64 field after {STEPS} steps of eq. (finalstrang) (Sec. 2.2) on the 3D\n")
        f.write("# workload n=(256,256,256), alpha=(1.2,1.5,1.8), eps=0.08, tau=2e-3, [-1,1]^3,\n")
        f.write("# u0 = sfac_inputs.config3_u0() (U[-1,1] from seed 2), sampled at 4096 flat indices\n")
        f.write(f"# (memory order, axis 1 fastest; tests/golden/make_config3_reference.py, route {route}).\n")
        f.write(f"# max_abs {float(np.abs(u).max()):.17e}\n")
        for i in idx:
            f.write(f"{int(i)} {float(flat[i]):.17e}\n")
    print("wrote", path, f"({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
