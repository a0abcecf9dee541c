"""Write mp_axis_factor_*.txt: one axis factor e^{tau/2 C} e^{tau S} e^{tau/2 C}
applied to a seeded vector, evaluated in 30 digits by oracle/sfac_oracle_mp.py.

Calls only the oracle and the seeded input generator. Run from the repo root:
    python tests/golden/make_mp_reference.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import sfac_inputs as I  # noqa: E402
from oracle.sfac_oracle_mp import mp_axis_apply  # noqa: E402

CASES = [  # (n, alpha, eps, tau, seed); domain [-1, 1], h = 2 / (n + 1)
    (256, 1.7, 0.05, 1e-3, 21),
    (1024, 1.3, 0.05, 1e-3, 22),
]


def main():
    for n, alpha, eps, tau, seed in CASES:
        x = I.uniform(seed, n, -1.0, 1.0)
        h = 2.0 / (n + 1)
        y = mp_axis_apply(alpha, eps, h, n, tau, x, dps=30)
        path = os.path.join(HERE, f"mp_axis_factor_n{n}.txt")
        with open(path, "w") as f:
            f.write("# e^{tau/2 C} e^{tau S} e^{tau/2 C} x for one axis (eqs. (C), (S), (hatv); Remark 1),\n")
            f.write("# evaluated in 30 digits from the FP64 first columns of C and S by\n")
            f.write("# oracle/sfac_oracle_mp.py; written by tests/golden/make_mp_reference.py.\n")
            f.write(f"# n={n} alpha={alpha} eps={eps} tau={tau} a=-1 b=1 x=sfac_inputs.uniform({seed}, n, -1, 1)\n")
            for v in y:
                f.write(f"{float(v):.17e}\n")
        print("wrote", path)


if __name__ == "__main__":
    main()
