"""CPU FP64 oracle for the two-level Strang splitting scheme of the spatial
fractional Allen-Cahn (SFAC) equation (Cai, Fang, Chen, Sun, arXiv 2209.08437).

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module. The product path (the
CUDA library and its Python binding) never calls it and shares no code with it.

Everything here is plain, dense and slow on purpose so that it can be checked
against the paper by eye:

* weights g_k and omega_k by their recursions (Sec. 2.1, eqs. (g_coe), (omega_coe));
* the dense lower-Hessenberg Toeplitz matrix D_alpha and B_alpha (eq. (B), first
  display of that label, Sec. 2.1);
* the circulant and skew-circulant parts C and S of B entry by entry (eqs. (C),
  (S), Sec. 2.2);
* matrix exponentials of the symmetric matrices C and S by scaling and squaring
  (scipy.linalg.expm, a library primitive); a second evaluation from a symmetric
  eigendecomposition, exp(tM) = V diag(exp(t w)) V^T, serves as a cross-check;
* the per-axis linear factor P = e^{tau/2 C} e^{tau S} e^{tau/2 C} (eq. (hatv)); by
  the Kronecker-sum form of C_alpha and S_alpha (eq. (newlinear)) the d-dimensional
  operator is the tensor product of the per-axis factors, applied line by line;
* the exact nonlinear flow J^Q (eq. (nonlinear_operator)) and the two-level step
  u <- J^Q_{tau/2} J^P_hat J^Q_{tau/2} u (eq. (finalstrang)), with no merging of the
  half flows between steps;
* the one-level Strang step with the exact e^{tau B} per axis (eq. (strang)) and
  the splitting-ADI step of Sec. 5, which the paper compares against.

Two evaluation routes of the same two-level factors exist. The "dense" route
multiplies every line by the dense n x n matrix P (the definition). The
"spectral" route applies e^{tau/2 C}, e^{tau S}, e^{tau/2 C} one after another
through the diagonalisations of Remark 1 (C = F^* Lambda_C F and
S = Theta^{-1} F^* Lambda_S F Theta) with numpy's FFT as the library primitive.
The two agree to about 1e-13 per application (pinned). The spectral route
exists because a dense FP64 matrix carries a fixed rounding error of a few
1e-15 per application at n = 1024 (checked against a 30-digit evaluation);
repeated for 1000 steps that error alone exceeds a 1e-12 comparison, whereas
the spectral route stays near 1e-15 per application.

Memory layout: a field is a numpy array of shape (n_d, ..., n_2, n_1), axis 1
(x^(1)) fastest, which is the paper's lexicographic ordering (Sec. 2.1).
Axis l of the paper is numpy axis d - l.

Every function is pinned by a test in tests/test_oracle_pins.py against
something the paper or mathematics fixes (Proposition 1, the stencil of
eq. (disFAC), the alpha = 2 Laplacian, library expm, the Bernoulli ODE, the
printed numbers of Tables 1, 2 and 4, the maximum principle, order 2, and for the
energy of Example 5 the alpha = 2 Ginzburg-Landau edge sum).
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np


# --------------------------------------------------------------------------
# Spatial discretisation (Sec. 2.1)
# --------------------------------------------------------------------------

def grunwald_g(alpha: float, K: int) -> np.ndarray:
    """g_0 .. g_K: g_0 = 1, g_{k+1} = (1 - (alpha+1)/(k+1)) g_k (eq. (g_coe))."""
    g = np.empty(K + 1)
    g[0] = 1.0
    for k in range(K):
        g[k + 1] = (1.0 - (alpha + 1.0) / (k + 1)) * g[k]
    return g


def omega_weights(alpha: float, K: int) -> np.ndarray:
    """omega_0 .. omega_K: omega_0 = (alpha/2) g_0,
    omega_{k+1} = (alpha/2) g_{k+1} + ((2-alpha)/2) g_k (eq. (omega_coe))."""
    g = grunwald_g(alpha, K)
    w = np.empty(K + 1)
    w[0] = 0.5 * alpha * g[0]
    for k in range(K):
        w[k + 1] = 0.5 * alpha * g[k + 1] + 0.5 * (2.0 - alpha) * g[k]
    return w


def riesz_factor(alpha: float, eps: float, h: float) -> float:
    """-eps^2 / (2 h^alpha cos(alpha pi / 2)), the scalar in front of D + D^T (eq. (B))."""
    return -eps * eps / (2.0 * h ** alpha * math.cos(alpha * math.pi / 2.0))


def matrix_D(alpha: float, n: int) -> np.ndarray:
    """The n x n lower Hessenberg Toeplitz matrix D_alpha of eq. (B): omega_1 on the
    diagonal, omega_0 on the first superdiagonal and omega_{i-j+1} below."""
    w = omega_weights(alpha, n + 1)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i - j + 1 >= 0:
                D[i, j] = w[i - j + 1]
    return D


def matrix_B(alpha: float, eps: float, h: float, n: int) -> np.ndarray:
    """B_alpha = -eps^2/(2 h^alpha cos(alpha pi/2)) (D_alpha + D_alpha^T) (eq. (B))."""
    D = matrix_D(alpha, n)
    return riesz_factor(alpha, eps, h) * (D + D.T)


def split_CS(B: np.ndarray):
    """C and S with B = C + S, entry by entry from eqs. (C) and (S).

    B = [b_{i-j}] is Toeplitz of size n = m - 1; for k = 1 .. m-2,
    c_k = (b_k + b_{k-m+1}) / 2 and s_k = (b_k - b_{k-m+1}) / 2; c_0 = s_0 = b_0 / 2;
    for k = -1 .. 2-m, c_k = (b_k + b_{k+m-1}) / 2 and s_k = (b_k - b_{k+m-1}) / 2.
    """
    n = B.shape[0]
    m = n + 1

    def b(k):  # the k-th diagonal of B: b_k = B[i, j] with i - j = k
        return B[k, 0] if k >= 0 else B[0, -k]

    c = {0: 0.5 * b(0)}
    s = {0: 0.5 * b(0)}
    for k in range(1, m - 1):
        c[k] = 0.5 * (b(k) + b(k - m + 1))
        s[k] = 0.5 * (b(k) - b(k - m + 1))
    for k in range(-1, 1 - m, -1):
        c[k] = 0.5 * (b(k) + b(k + m - 1))
        s[k] = 0.5 * (b(k) - b(k + m - 1))
    C = np.empty((n, n))
    S = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            C[i, j] = c[i - j]
            S[i, j] = s[i - j]
    return C, S


# --------------------------------------------------------------------------
# Flows (Sec. 2.2)
# --------------------------------------------------------------------------

def expm_dense(M: np.ndarray, t: float) -> np.ndarray:
    """exp(t M) by scaling and squaring with Pade approximants (scipy.linalg.expm)."""
    import scipy.linalg
    return scipy.linalg.expm(t * M)


def expm_symmetric(M: np.ndarray, t: float) -> np.ndarray:
    """exp(t M) for symmetric M from its eigendecomposition M = V diag(w) V^T
    (cross-check of expm_dense)."""
    w, V = np.linalg.eigh(M)
    return (V * np.exp(t * w)) @ V.T


def nonlinear_flow(v: np.ndarray, s: float) -> np.ndarray:
    """Exact flow J^Q_s of v' = v - v^3 (eq. (nonlinear_operator)):
    v / sqrt(v^2 + (1 - v^2) e^{-2s})."""
    return v / np.sqrt(v * v + (1.0 - v * v) * math.exp(-2.0 * s))


def axis_two_level_factor(alpha: float, eps: float, h: float, n: int, tau: float) -> np.ndarray:
    """P = e^{tau/2 C} e^{tau S} e^{tau/2 C} for one axis (eq. (hatv))."""
    C, S = split_CS(matrix_B(alpha, eps, h, n))
    EC = expm_dense(C, 0.5 * tau)
    ES = expm_dense(S, tau)
    return EC @ ES @ EC


def axis_one_level_factor(alpha: float, eps: float, h: float, n: int, tau: float) -> np.ndarray:
    """e^{tau B} for one axis; the d-dim e^{tau A} is their tensor product (eqs. (2DA),
    (3DA), (linear_operator))."""
    return expm_dense(matrix_B(alpha, eps, h, n), tau)


def axis_adi_factor(alpha: float, eps: float, h: float, n: int, tau: float) -> np.ndarray:
    """(I - tau/2 B)^{-1} (I + tau/2 B), the per-axis factor of the splitting-ADI
    scheme that Sec. 5 compares against."""
    B = matrix_B(alpha, eps, h, n)
    I = np.eye(n)
    return np.linalg.solve(I - 0.5 * tau * B, I + 0.5 * tau * B)


def apply_axis(u: np.ndarray, P: np.ndarray, axis: int) -> np.ndarray:
    """Multiply every line of u along paper axis `axis` (1-based) by P."""
    ax = u.ndim - axis
    return np.moveaxis(np.tensordot(P, u, axes=([1], [ax])), 0, ax)


class SpectralFactor:
    """e^{tau/2 C} e^{tau S} e^{tau/2 C} of one axis applied through Remark 1:
    e^{t C} = F^{-1} diag(e^{t lambda}) F with lambda = F c (first column of C), and
    e^{t S} = Theta^{-1} F^{-1} diag(e^{t mu}) F Theta with Theta = diag(e^{i pi k/n})
    and mu = F (Theta s). F is numpy's forward FFT (e^{-2 pi i jk/n})."""

    def __init__(self, alpha: float, eps: float, h: float, n: int, tau: float):
        C, S = split_CS(matrix_B(alpha, eps, h, n))
        self.theta = np.exp(1j * np.pi * np.arange(n) / n)
        self.lam = np.fft.fft(C[:, 0]).real      # C symmetric: real spectrum
        self.mu = np.fft.fft(self.theta * S[:, 0]).real
        self.eC = np.exp(0.5 * tau * self.lam)
        self.eS = np.exp(tau * self.mu)

    def apply(self, u: np.ndarray, axis: int) -> np.ndarray:
        """Multiply every line of u along paper axis `axis` (1-based)."""
        ax = u.ndim - axis
        shp = [1] * u.ndim
        shp[ax] = -1
        eC, eS, th = self.eC.reshape(shp), self.eS.reshape(shp), self.theta.reshape(shp)
        z = np.fft.ifft(eC * np.fft.fft(u, axis=ax), axis=ax)
        z = np.conj(th) * np.fft.ifft(eS * np.fft.fft(th * z, axis=ax), axis=ax)
        z = np.fft.ifft(eC * np.fft.fft(z, axis=ax), axis=ax)
        return z.real


class Scheme:
    """Per-axis factors for one problem (alpha per axis, eps, tau, [a, b]).

    kind = "two_level" (eq. (finalstrang)), "one_level" (eq. (strang)) or "adi"
    (the splitting-ADI scheme of Sec. 5). route = "dense" multiplies lines by the
    dense factor; route = "spectral" (two-level only) applies the factor through
    Remark 1 (SpectralFactor).
    """

    def __init__(self, n: Sequence[int], alpha: Sequence[float], eps: float, tau: float,
                 a: float = -1.0, b: float = 1.0, kind: str = "two_level", route: str = "dense"):
        self.n = tuple(int(v) for v in n)
        self.alpha = tuple(float(v) for v in alpha)
        self.eps, self.tau, self.a, self.b = float(eps), float(tau), float(a), float(b)
        self.route = route
        if route == "spectral":
            if kind != "two_level":
                raise ValueError("the spectral route evaluates the two-level factors only")
            build = SpectralFactor
        else:
            build = {"two_level": axis_two_level_factor, "one_level": axis_one_level_factor,
                     "adi": axis_adi_factor}[kind]
        self.P = []
        for ax, nn in enumerate(self.n):
            h = (self.b - self.a) / (nn + 1)
            self.P.append(build(self.alpha[ax], self.eps, h, nn, self.tau))

    @classmethod
    def for_problem(cls, problem, kind: str = "two_level", route: str = "dense") -> "Scheme":
        return cls(problem.n, problem.alpha, problem.eps, problem.tau, problem.a, problem.b, kind, route)

    def apply_linear(self, u: np.ndarray, axis: int) -> np.ndarray:
        P = self.P[axis - 1]
        return P.apply(u, axis) if self.route == "spectral" else apply_axis(u, P, axis)

    def step(self, u: np.ndarray) -> np.ndarray:
        """One step u <- J^Q_{tau/2} (prod_l P_l) J^Q_{tau/2} u (eqs. (strang), (finalstrang))."""
        u = nonlinear_flow(u, 0.5 * self.tau)
        for ax in range(len(self.P)):
            u = self.apply_linear(u, ax + 1)
        return nonlinear_flow(u, 0.5 * self.tau)

    def run(self, u0: np.ndarray, nsteps: int) -> np.ndarray:
        u = np.array(u0, dtype=np.float64, copy=True)
        assert u.shape == tuple(reversed(self.n))
        for _ in range(nsteps):
            u = self.step(u)
        return u


def solve(problem, u0: np.ndarray, nsteps: int | None = None, kind: str = "two_level",
          route: str = "dense") -> np.ndarray:
    """Run `nsteps` (default problem.steps) steps of the chosen scheme from u0."""
    sch = Scheme.for_problem(problem, kind, route)
    return sch.run(u0, problem.steps if nsteps is None else nsteps)


# --------------------------------------------------------------------------
# Remark 1: the same factors through Fourier diagonalisation (direct DFTs)
# --------------------------------------------------------------------------

def dft_matrix(n: int) -> np.ndarray:
    """F_jk = exp(-2 pi i j k / n) (unnormalised forward DFT), built entry by entry."""
    j = np.arange(n).reshape(-1, 1)
    k = np.arange(n).reshape(1, -1)
    return np.exp(-2j * np.pi * ((j * k) % n) / n)


def circulant_eigenvalues(first_col: np.ndarray) -> np.ndarray:
    """lambda_j = sum_k c_k e^{-2 pi i j k / n} (Remark 1: F C e_1 gives the spectrum)."""
    return dft_matrix(len(first_col)) @ first_col


def skew_circulant_eigenvalues(first_col: np.ndarray) -> np.ndarray:
    """mu_j = sum_k s_k e^{i pi k / n} e^{-2 pi i j k / n}: the skew-circulant S equals
    Theta^{-1} circ(s_k e^{i pi k/n}) Theta with Theta = diag(e^{i pi k / n}) (Remark 1)."""
    n = len(first_col)
    twist = np.exp(1j * np.pi * np.arange(n) / n)
    return dft_matrix(n) @ (twist * first_col)


def axis_factor_by_dft(alpha: float, eps: float, h: float, n: int, tau: float) -> np.ndarray:
    """P of eq. (hatv) assembled from O(n^2) DFT matrices and the spectra of Remark 1
    (complex arithmetic, real part returned)."""
    C, S = split_CS(matrix_B(alpha, eps, h, n))
    lam = circulant_eigenvalues(C[:, 0])
    mu = skew_circulant_eigenvalues(S[:, 0])
    F = dft_matrix(n)
    Finv = F.conj().T / n
    theta = np.diag(np.exp(1j * np.pi * np.arange(n) / n))
    EC = Finv @ np.diag(np.exp(0.5 * tau * lam)) @ F
    ES = theta.conj() @ Finv @ np.diag(np.exp(tau * mu)) @ F @ theta
    return (EC @ ES @ EC).real


# --------------------------------------------------------------------------
# Diagnostics (Sec. 5)
# --------------------------------------------------------------------------

def time_error(u_tau: np.ndarray, u_half: np.ndarray) -> float:
    """Max-norm difference of two runs with steps tau and tau/2 (the E_t of Sec. 5)."""
    return float(np.max(np.abs(u_tau - u_half)))


def discrete_energy(u: np.ndarray, scheme: Scheme) -> float:
    """E(u) = h^d ((1/4)(u^2-1)^T (u^2-1) - (1/2) u^T A u) (Example 5), with the
    operator A = sum_l I x .. x B_l x .. x I applied axis by axis."""
    d = u.ndim
    Au = np.zeros_like(u)
    hprod = 1.0
    for ax in range(d):
        nn = scheme.n[ax]
        h = (scheme.b - scheme.a) / (nn + 1)
        hprod *= h
        B = matrix_B(scheme.alpha[ax], scheme.eps, h, nn)
        Au += apply_axis(u, B, ax + 1)
    w = u * u - 1.0
    return hprod * (0.25 * float(np.sum(w * w)) - 0.5 * float(np.sum(u * Au)))
