"""High-precision (mpmath) evaluation of one axis factor e^{tau/2 C} e^{tau S} e^{tau/2 C}
applied to a vector: the yardstick for the FP64 routes of sfac_oracle.

TEST INFRASTRUCTURE ONLY (see sfac_oracle). Used by tests/golden/make_mp_reference.py
to write stored reference values, and by the CPU tests that pin the oracle.

Starting from the FP64 first columns c_k, s_k of C and S (eqs. (C), (S), built by
sfac_oracle.split_CS), everything is carried in `dps` decimal digits:
  lambda_j = sum_k c_k cos(2 pi j k / n),      mu_j = sum_k s_k cos(pi k (2j - 1) / n)
(the real spectra of Remark 1), then the Toeplitz first columns of the factors
  e^{t C}[a, b] = (1/n) sum_j e^{t lambda_j} cos(2 pi j (a-b) / n),
  e^{t S}[a, b] = (1/n) sum_j e^{t mu_j} cos(pi (a-b)(2j - 1) / n),
which follow from C = F^* Lambda_C F and S = Theta^{-1} F^* Lambda_S F Theta with
Theta = diag(e^{i pi k/n}), and finally three Toeplitz matrix-vector products.
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

from . import sfac_oracle as O


def mp_axis_apply(alpha: float, eps: float, h: float, n: int, tau: float, x, dps: int = 30):
    """e^{tau/2 C} e^{tau S} e^{tau/2 C} x in `dps` digits; returns an mp list."""
    with mp.workdps(dps):
        C, S = O.split_CS(O.matrix_B(alpha, eps, h, n))
        c = [mp.mpf(float(v)) for v in C[:, 0]]
        s = [mp.mpf(float(v)) for v in S[:, 0]]
        cosv = [mp.cos(mp.pi * m / n) for m in range(2 * n)]
        lam = [mp.fsum(c[k] * cosv[(2 * j * k) % (2 * n)] for k in range(n)) for j in range(n)]
        mu = [mp.fsum(s[k] * cosv[(k * (2 * j - 1)) % (2 * n)] for k in range(n)) for j in range(n)]
        half, full = mp.mpf(tau) / 2, mp.mpf(tau)
        eC = [mp.exp(half * v) for v in lam]
        eS = [mp.exp(full * v) for v in mu]
        gC = [mp.fsum(eC[j] * cosv[(2 * j * d) % (2 * n)] for j in range(n)) / n for d in range(n)]
        gS = {d: mp.fsum(eS[j] * cosv[(d * (2 * j - 1)) % (2 * n)] for j in range(n)) / n
              for d in range(-n + 1, n)}

        def toeplitz(col, v, symmetric):
            return [mp.fsum((col[abs(a - b)] if symmetric else col[a - b]) * v[b] for b in range(n))
                    for a in range(n)]

        y = [mp.mpf(float(v)) for v in x]
        y = toeplitz(gC, y, True)
        y = toeplitz(gS, y, False)
        y = toeplitz(gC, y, True)
        return y


def mp_axis_apply_f64(alpha, eps, h, n, tau, x, dps: int = 30) -> np.ndarray:
    return np.array([float(v) for v in mp_axis_apply(alpha, eps, h, n, tau, x, dps)])
