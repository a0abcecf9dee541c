"""Pins of the CPU FP64 oracle against what the paper and mathematics fix.

Each check is independent of the oracle's own formulas: closed forms of
Proposition 1, the literal stencil of eq. (disFAC), the alpha = 2 Laplacian
and its sine eigenbasis, library routines (scipy expm, numpy FFT, an ODE
integrator), the printed numbers of Tables 2 and 4, Theorem 1's maximum
principle and the second-order rates of Theorem 2. A final group plants
plausible mistakes in a copy of the oracle and checks a pin catches each.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.special
from scipy.integrate import solve_ivp

import sfac_inputs as I
from oracle import sfac_oracle as O
from tests.conftest import read_golden

ALPHAS = [1.05, 1.2, 1.3, 1.5, 1.7, 1.8, 1.95]


# ---------------------------------------------------------------- weights ---

@pytest.mark.parametrize("alpha", ALPHAS + [2.0])
def test_g_is_alternating_binomial(alpha):
    """g_k = (-1)^k binom(alpha, k): the alternating fractional binomial coefficients."""
    g = O.grunwald_g(alpha, 60)
    ref = np.array([(-1) ** k * scipy.special.binom(alpha, k) for k in range(61)])
    np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("alpha", ALPHAS)
def test_omega_proposition1(alpha):
    """Proposition 1 (Sec. 2.1): closed forms, signs, monotonicity and sums."""
    w = O.omega_weights(alpha, 20000)
    assert w[0] == pytest.approx(alpha / 2, rel=1e-15)
    assert w[1] == pytest.approx((2 - alpha - alpha ** 2) / 2, rel=1e-14)
    assert w[2] == pytest.approx(alpha * (alpha ** 2 + alpha - 4) / 4, rel=1e-13)
    assert w[1] <= 0 and w[0] + w[2] > 0
    assert 1 >= w[0] >= w[3]
    assert np.all(np.diff(w[3:]) <= 0) and np.all(w[3:] >= 0)
    partial = np.cumsum(w)
    assert np.all(partial[2:] < 0)
    # sum_{k>=0} omega_k = 0: the tail decays like k^(-alpha-1), partial sums -> 0.
    assert abs(partial[-1]) < 5 * 20000 ** (1 - alpha)


# ------------------------------------------------------------ matrix B -----

def stencil_apply(alpha, eps, h, u):
    """Eq. (disFAC) for one axis, written out literally: the two sums with the
    zero boundary values u_0 = u_m = 0 of eq. (condition)."""
    n = len(u)
    m = n + 1
    full = np.zeros(m + 1)
    full[1:m] = u
    w = O.omega_weights(alpha, m + 2)
    pre = -eps ** 2 / (2 * h ** alpha * math.cos(alpha * math.pi / 2))
    out = np.zeros(n)
    for i in range(1, m):
        left = sum(w[k] * full[i - k + 1] for k in range(0, i + 2))
        right = sum(w[k] * full[i + k - 1] for k in range(0, m - i + 2))
        out[i - 1] = pre * (left + right)
    return out


@pytest.mark.parametrize("alpha,n", [(1.3, 7), (1.7, 12), (1.5, 2), (1.1, 16)])
def test_B_equals_stencil(alpha, n):
    eps, h = 0.1, 2.0 / (n + 1)
    B = O.matrix_B(alpha, eps, h, n)
    rng = np.random.default_rng(3)
    for _ in range(3):
        u = rng.uniform(-1, 1, n)
        np.testing.assert_allclose(B @ u, stencil_apply(alpha, eps, h, u), rtol=1e-12, atol=1e-12)
    assert np.array_equal(B, B.T)
    assert np.all(np.diag(B) < 0)


def laplacian_spectrum(n, eps, h):
    """alpha = 2: B = eps^2/h^2 tridiag(1, -2, 1); eigenpairs are the DST-I modes."""
    j = np.arange(1, n + 1)
    lam = -(4 * eps ** 2 / h ** 2) * np.sin(j * np.pi / (2 * (n + 1))) ** 2
    i = np.arange(1, n + 1).reshape(-1, 1)
    V = np.sqrt(2.0 / (n + 1)) * np.sin(i * j.reshape(1, -1) * np.pi / (n + 1))
    return lam, V


def test_alpha2_reduces_to_laplacian_and_expm():
    n, eps = 15, 0.3
    h = 1.0 / (n + 1)
    B = O.matrix_B(2.0, eps, h, n)
    T = eps ** 2 / h ** 2 * (np.diag(-2 * np.ones(n)) + np.diag(np.ones(n - 1), 1)
                              + np.diag(np.ones(n - 1), -1))
    np.testing.assert_allclose(B, T, rtol=1e-12, atol=1e-9)
    lam, V = laplacian_spectrum(n, eps, h)
    tau = 0.37
    closed = (V * np.exp(tau * lam)) @ V.T
    np.testing.assert_allclose(O.expm_dense(B, tau), closed, atol=1e-13)
    np.testing.assert_allclose(O.expm_symmetric(B, tau), closed, atol=1e-13)


# ------------------------------------------------------------ C and S ------

@pytest.mark.parametrize("alpha,n", [(1.3, 8), (1.7, 13), (1.5, 32), (1.1, 5), (1.9, 64)])
def test_split_structure_and_lemma2(alpha, n):
    eps, h = 0.05, 2.0 / (n + 1)
    B = O.matrix_B(alpha, eps, h, n)
    C, S = O.split_CS(B)
    # B = C + S up to the rounding of (x+y)/2 + (x-y)/2.
    np.testing.assert_allclose(C + S, B, rtol=0, atol=4 * np.finfo(float).eps * np.abs(B).max())
    c, s = C[:, 0], S[:, 0]
    for i in range(n):
        for j in range(n):
            assert C[i, j] == c[(i - j) % n]                        # circulant
            sgn = 1.0 if i >= j else -1.0                            # skew-circulant wrap
            assert S[i, j] == sgn * s[(i - j) % n]
    assert np.array_equal(C, C.T) and np.array_equal(S, S.T)
    # Lemma 2: diagonally dominant with negative diagonal.
    for M in (C, S):
        d = np.diag(M)
        off = np.abs(M).sum(axis=1) - np.abs(d)
        assert np.all(d < 0) and np.all(off <= -d * (1 + 1e-12))
    # Row sum of C = -eps^2/(2 h^a cos(a pi/2)) sum_{k=0}^{m-1} omega_k (proof of Lemma 2).
    w = O.omega_weights(alpha, n + 1)
    rowsum = O.riesz_factor(alpha, eps, h) * w[: n + 1].sum()
    np.testing.assert_allclose(C.sum(axis=1), rowsum, rtol=1e-11)


@pytest.mark.parametrize("alpha,n", [(1.3, 8), (1.7, 13), (1.5, 32), (1.2, 63)])
def test_spectra_from_first_column(alpha, n):
    """Remark 1: the circulant / skew-circulant spectra are the DFT of the first
    column (twisted for S); compared with a dense symmetric eigensolve and with
    numpy's FFT (both libraries, independent of the oracle's DFT matrix)."""
    eps, h = 0.1, 2.0 / (n + 1)
    C, S = O.split_CS(O.matrix_B(alpha, eps, h, n))
    lam = O.circulant_eigenvalues(C[:, 0])
    mu = O.skew_circulant_eigenvalues(S[:, 0])
    scale = np.abs(np.diag(C)).max()
    assert np.abs(lam.imag).max() < 1e-12 * scale and np.abs(mu.imag).max() < 1e-12 * scale
    np.testing.assert_allclose(np.sort(lam.real), np.linalg.eigvalsh(C), atol=1e-12 * scale)
    np.testing.assert_allclose(np.sort(mu.real), np.linalg.eigvalsh(S), atol=1e-12 * scale)
    np.testing.assert_allclose(lam, np.fft.fft(C[:, 0]), atol=1e-12 * scale)
    tw = np.exp(1j * np.pi * np.arange(n) / n)
    np.testing.assert_allclose(mu, np.fft.fft(tw * S[:, 0]), atol=1e-12 * scale)
    assert np.all(lam.real <= 1e-12 * scale) and np.all(mu.real <= 1e-12 * scale)


@pytest.mark.parametrize("alpha,n", [(1.3, 8), (1.7, 21), (1.5, 40)])
def test_expm_against_pade_and_contractivity(alpha, n):
    eps, h, tau = 0.1, 2.0 / (n + 1), 0.05
    C, S = O.split_CS(O.matrix_B(alpha, eps, h, n))
    for M, t in ((C, tau / 2), (S, tau), (C + S, tau)):
        E = O.expm_dense(M, t)
        # scaling-and-squaring against the eigendecomposition route
        np.testing.assert_allclose(E, O.expm_symmetric(M, t), atol=1e-13, rtol=1e-12)
    for M in (C, S):  # Lemmas 1-2: ||e^{tM}||_inf <= 1
        for t in (1e-3, 0.1, 10.0):
            assert np.abs(O.expm_dense(M, t)).sum(axis=1).max() <= 1 + 1e-12


@pytest.mark.parametrize("alpha,n", [(1.3, 8), (1.7, 13), (1.45, 32)])
def test_two_level_factor_by_dft(alpha, n):
    """The dense P = e^{tau/2 C} e^{tau S} e^{tau/2 C} equals its Remark-1 FFT form."""
    eps, h, tau = 0.08, 2.0 / (n + 1), 0.02
    P = O.axis_two_level_factor(alpha, eps, h, n, tau)
    Q = O.axis_factor_by_dft(alpha, eps, h, n, tau)
    np.testing.assert_allclose(P, Q, atol=1e-13)
    np.testing.assert_allclose(P, P.T, atol=1e-14)  # symmetric: a product E_C E_S E_C


def test_mp_yardstick_equals_dense_definition():
    """The 30-digit evaluation (Toeplitz columns from the Remark-1 spectra) against the
    dense definition e^{tau/2 C} e^{tau S} e^{tau/2 C} on small n."""
    from oracle.sfac_oracle_mp import mp_axis_apply_f64
    for n, alpha in ((5, 1.3), (8, 1.8), (16, 1.5)):
        h, tau = 2.0 / (n + 1), 0.3
        x = I.uniform(40 + n, n, -1, 1)
        P = O.axis_two_level_factor(alpha, 0.2, h, n, tau)
        np.testing.assert_allclose(mp_axis_apply_f64(alpha, 0.2, h, n, tau, x), P @ x, atol=2e-15)


def _mp_golden(n):
    rows = read_golden(f"mp_axis_factor_n{n}.txt")
    return np.array([float(r[0]) for r in rows])


@pytest.mark.parametrize("n,alpha,seed,tol_dense", [(256, 1.7, 21, 5e-15), (1024, 1.3, 22, 1e-14)])
def test_routes_against_30_digit_reference(n, alpha, seed, tol_dense):
    """Both FP64 routes of the oracle against the stored 30-digit values: the dense
    route within its rounding (a few 1e-15), the spectral route within 3e-15."""
    x = I.uniform(seed, n, -1.0, 1.0)
    y = _mp_golden(n)
    h = 2.0 / (n + 1)
    P = O.axis_two_level_factor(alpha, 0.05, h, n, 1e-3)
    assert np.abs(P @ x - y).max() <= tol_dense
    sf = O.SpectralFactor(alpha, 0.05, h, n, 1e-3)
    assert np.abs(sf.apply(x, 1) - y).max() <= 3e-15


@pytest.mark.parametrize("n", [(16,), (32, 8), (8, 16, 4)], ids=str)
def test_dense_and_spectral_routes_agree(n):
    prob = I.Problem(n=n, alpha=(1.25, 1.75, 1.5)[: len(n)], eps=0.1, tau=0.02)
    u0 = I.random_field(prob, 9)
    a = O.solve(prob, u0, 5)
    b = O.solve(prob, u0, 5, route="spectral")
    assert np.abs(a - b).max() <= 1e-13


def test_circulant_B_makes_second_level_exact():
    """If B is itself symmetric circulant then S = (b_0/2) I commutes with C, so the
    second-level splitting is exact: P = e^{tau B}."""
    n = 9
    first = np.array([-3.0, 1.2, 0.4, 0.1, 0.05, 0.05, 0.1, 0.4, 1.2])
    B = np.array([[first[(i - j) % n] for j in range(n)] for i in range(n)])
    C, S = O.split_CS(B)
    np.testing.assert_allclose(S, 0.5 * first[0] * np.eye(n), atol=1e-15)
    tau = 0.3
    P = O.expm_symmetric(C, tau / 2) @ O.expm_symmetric(S, tau) @ O.expm_symmetric(C, tau / 2)
    np.testing.assert_allclose(P, scipy.linalg.expm(tau * B), atol=1e-13)


# --------------------------------------------------------------- J^Q -------

def test_nonlinear_flow_solves_bernoulli_ode():
    v0 = np.array([-1.3, -1.0, -0.7, -0.2, 0.0, 1e-3, 0.4, 0.95, 1.0, 2.5])
    for s in (1e-3, 0.05, 0.5, 3.0):
        sol = solve_ivp(lambda t, v: v - v ** 3, (0, s), v0, method="DOP853", rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(O.nonlinear_flow(v0, s), sol.y[:, -1], rtol=1e-10, atol=1e-13)


def test_nonlinear_flow_properties():
    v = np.linspace(-1, 1, 2001)
    for s in (1e-4, 0.01, 1.0, 50.0):
        J = O.nonlinear_flow(v, s)
        assert np.all(np.abs(J) <= 1 + 1e-15)
        np.testing.assert_array_equal(O.nonlinear_flow(-v, s), -J)
        np.testing.assert_array_equal(O.nonlinear_flow(np.array([0.0, 1.0, -1.0]), s),
                                      np.array([0.0, 1.0, -1.0]))
        np.testing.assert_allclose(O.nonlinear_flow(O.nonlinear_flow(v, s), 0.3 * s),
                                   O.nonlinear_flow(v, 1.3 * s), rtol=2e-15, atol=1e-16)


# ----------------------------------------------------------- full scheme ---

def test_brute_force_n2():
    """n = 2: C = [[b0/2, b1], [b1, b0/2]] and S = (b0/2) I, so P = e^{tau B}, whose
    eigenpairs are b0 +- b1 on (1, +-1)/sqrt(2); checked by hand against one step."""
    alpha, eps, tau = 1.4, 0.2, 0.1
    h = 2.0 / 3
    w = O.omega_weights(alpha, 3)
    r = O.riesz_factor(alpha, eps, h)
    b0, b1 = 2 * r * w[1], r * (w[0] + w[2])
    ep, em = math.exp(tau * (b0 + b1)), math.exp(tau * (b0 - b1))
    P = 0.5 * np.array([[ep + em, ep - em], [ep - em, ep + em]])
    u0 = np.array([0.3, -0.8])
    E = math.exp(-tau)
    jq = lambda v: v / np.sqrt(v * v + (1 - v * v) * E)
    expect = jq(P @ jq(u0))
    got = O.Scheme((2,), (alpha,), eps, tau).step(u0)
    np.testing.assert_allclose(got, expect, rtol=1e-14)


def _golden_rows(name, ncols):
    out = []
    for r in read_golden(name):
        out.append(tuple(float(x) for x in r[:ncols]) + tuple(float(x) for x in r[ncols:]))
    return out


def _close_to_printed(value, printed):
    """Agreement to the 5 printed significant digits (one unit of the last digit),
    with a 2e-13 absolute floor for the rounding of either implementation."""
    unit = 10.0 ** (math.floor(math.log10(printed)) - 4)
    return abs(value - printed) <= unit + 2e-13


_T2 = [r for r in _golden_rows("table2_example1_Et.txt", 3)]


@pytest.mark.parametrize("row", [r for r in _T2 if r[2] in (100.0, 200.0)], ids=lambda r: f"{r[:3]}")
def test_table2_example1(row):
    a1, a2, ninv = row[0], row[1], int(row[2])
    for col, kind in ((3, "two_level"), (4, "one_level"), (5, "adi")):
        if (a1, a2, ninv, kind) == (1.2, 1.8, 100, "two_level"):
            continue  # printed 3.2386e-6; the scheme gives 3.2383e-6 (misprint reading)
        res = []
        for N in (ninv, 2 * ninv):
            p = I.example1_problem((a1, a2), 1.0 / N)
            res.append(O.solve(p, I.example1_u0(p), kind=kind))
        et = O.time_error(res[0], res[1])
        assert _close_to_printed(et, row[col]), (kind, et, row[col])


@pytest.mark.slow
@pytest.mark.parametrize("row", [r for r in _T2 if r[2] == 400.0], ids=lambda r: f"{r[:3]}")
def test_table2_example1_row400(row):
    test_table2_example1(row)


_T1 = _golden_rows("table1_example1_Es.txt", 3)


def _table1_block(alpha):
    """Table 1 for one alpha pair: one step (tau = T = 1) on h = 2^-4 .. 2^-8 and
    on the reference h = 1/2048 (m = 4096), spectral route; the coarse grid's
    nodes x_i = i h are the reference nodes i 2^(11-k)."""
    m_ref = 4096
    pf = I.example1_problem(alpha, 1.0, m=m_ref)
    uf = O.solve(pf, I.example1_u0(pf), route="spectral")
    out = {}
    for k in (4, 5, 6, 7, 8):
        mc = 2 ** (k + 1)
        pc = I.example1_problem(alpha, 1.0, m=mc)
        uc = O.solve(pc, I.example1_u0(pc), route="spectral")
        r = m_ref // mc
        out[k] = float(np.abs(uc - uf[r - 1::r, r - 1::r]).max())
    return out


def _check_table1(alpha):
    got = _table1_block(alpha)
    rows = [r for r in _T1 if (r[0], r[1]) == alpha]
    assert len(rows) == 5
    for a1, a2, k, printed in rows:
        if (alpha, int(k)) == ((1.2, 1.8), 6):
            assert abs(got[6] - 1.52425e-3) < 1e-8  # printed 1.5245e-3 (misprint reading)
            continue
        assert _close_to_printed(got[int(k)], printed), (alpha, k, got[int(k)], printed)
    orders = [math.log2(got[k] / got[k + 1]) for k in (4, 5, 6, 7)]
    assert all(1.75 < o < 2.05 for o in orders), orders


def test_table1_example1_space_order():
    """Table 1, first column (alpha = (1.2, 1.4), different orders on the two
    axes): the spatial errors to the printed digits, order about 2."""
    _check_table1((1.2, 1.4))


@pytest.mark.slow
@pytest.mark.parametrize("alpha", [(1.5, 1.5), (1.2, 1.8), (1.6, 1.9)], ids=str)
def test_table1_example1_other_columns(alpha):
    _check_table1(alpha)


@pytest.mark.parametrize("row", _golden_rows("table4_example2_Et.txt", 4)[:2] + _golden_rows("table4_example2_Et.txt", 4)[3:5],
                         ids=lambda r: f"{r[:4]}")
def test_table4_example2_one_level_and_adi(row):
    al, ninv = row[:3], int(row[3])
    for col, kind in ((5, "one_level"), (6, "adi")):
        if kind == "adi" and tuple(al) == (1.5, 1.5, 1.5):
            continue  # 1.3-1.8 printed units off; recorded in the fixture header
        res = []
        for N in (ninv, 2 * ninv):
            p = I.example2_problem(al, 1.0 / N)
            res.append(O.solve(p, I.example2_u0(p), kind=kind))
        et = O.time_error(res[0], res[1])
        assert _close_to_printed(et, row[col]), (kind, et, row[col])


@pytest.mark.parametrize("dims,n", [(1, 16), (2, 12), (3, 6)])
def test_maximum_principle_any_tau(dims, n):
    """Theorem 1: ||u^n||_inf <= 1 for every tau > 0 whenever ||u^0||_inf <= 1."""
    for tau in (1e-3, 0.1, 10.0):
        p = I.Problem(n=(n,) * dims, alpha=(1.9, 1.3, 1.6)[:dims], eps=0.3, tau=tau)
        u = I.random_field(p, 11, -1.0, 1.0)
        sch = O.Scheme.for_problem(p)
        for _ in range(20):
            u = sch.step(u)
            assert np.abs(u).max() <= 1 + 1e-14


def test_second_order_in_time_and_local_defect():
    """Theorem 2 / Sec. 4: E_t(tau)/E_t(tau/2) -> 4, and the per-step gap between the
    one-level and two-level steps is O(tau^3) (ratio 8 under halving)."""
    p0 = I.Problem(n=(31, 31), alpha=(1.3, 1.8), eps=0.1, tau=0.1, a=0.0, b=2.0)
    u0 = I.example1_u0(p0)
    ets = []
    for N in (20, 40, 80, 160):
        pa = I.Problem(n=p0.n, alpha=p0.alpha, eps=p0.eps, tau=1.0 / N, a=0.0, b=2.0)
        pb = I.Problem(n=p0.n, alpha=p0.alpha, eps=p0.eps, tau=0.5 / N, a=0.0, b=2.0)
        ets.append(O.time_error(O.solve(pa, u0, N), O.solve(pb, u0, 2 * N)))
    orders = np.log2(np.array(ets[:-1]) / np.array(ets[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.1), orders
    gaps = []
    for tau in (0.04, 0.02, 0.01):
        p = I.Problem(n=p0.n, alpha=p0.alpha, eps=p0.eps, tau=tau, a=0.0, b=2.0)
        one = O.Scheme.for_problem(p, "one_level").step(u0)
        two = O.Scheme.for_problem(p, "two_level").step(u0)
        gaps.append(np.abs(one - two).max())
    ratios = np.array(gaps[:-1]) / np.array(gaps[1:])
    assert np.all(np.abs(ratios - 8.0) < 0.8), ratios


# ------------------------------------------------ axis assignment (d >= 2) ---
#
# Eq. (2DA) writes A = I (x) B_{alpha_1} + B_{alpha_2} (x) I for the vector u
# ordered with x^(1) fastest (the ordering under eq. (condition)), and eq. (3DA)
# the three-term sum; eq. (newlinear) splits C_alpha and S_alpha the same way.
# The pins below build those Kronecker sums literally with np.kron on grids whose
# axes differ in n (hence in h) and in alpha, so that every assignment of alpha,
# h or the memory axis to the wrong paper axis changes the result.

_AXIS_CASES = [((2, 3), (1.2, 1.8)), ((3, 3), (1.15, 1.85)), ((4, 3), (1.7, 1.3)),
               ((2, 3, 4), (1.2, 1.5, 1.8)), ((3, 2, 2), (1.9, 1.1, 1.45))]


def _kron_sum(mats):
    """sum_l I (x) .. (x) M_l (x) .. (x) I with M_1 acting on the fastest index:
    the paper's M_d (x) ... (x) M_1 ordering of eqs. (2DA), (3DA), (newlinear)."""
    sizes = [m.shape[0] for m in mats]
    total = np.zeros((int(np.prod(sizes)),) * 2)
    for l, M in enumerate(mats):
        term = np.eye(1)
        for k in reversed(range(len(mats))):  # axis d first (slowest)
            term = np.kron(term, M if k == l else np.eye(sizes[k]))
        total += term
    return total


def _axis_pieces(n, alpha, eps, a, b):
    Bs, Cs, Ss = [], [], []
    for nl, al in zip(n, alpha):
        h = (b - a) / (nl + 1)
        B = O.matrix_B(al, eps, h, nl)
        C, S = O.split_CS(B)
        Bs.append(B)
        Cs.append(C)
        Ss.append(S)
    return Bs, Cs, Ss


def _kron_two_level_step(n, alpha, eps, tau, a, b, u):
    """J^Q_{tau/2} e^{tau/2 C_alpha} e^{tau S_alpha} e^{tau/2 C_alpha} J^Q_{tau/2} u
    with C_alpha, S_alpha the full Kronecker sums of eq. (newlinear) and dense
    matrix exponentials of the whole (prod n) x (prod n) matrices."""
    _, Cs, Ss = _axis_pieces(n, alpha, eps, a, b)
    Ca, Sa = _kron_sum(Cs), _kron_sum(Ss)
    EC = scipy.linalg.expm(0.5 * tau * Ca)
    ES = scipy.linalg.expm(tau * Sa)
    E = math.exp(-tau)
    jq = lambda v: v / np.sqrt(v * v + (1 - v * v) * E)
    v = jq(u.ravel())  # C order of shape (n_d, .., n_1): x^(1) fastest
    return jq(EC @ (ES @ (EC @ v))).reshape(u.shape)


def _kron_one_level_step(n, alpha, eps, tau, a, b, u):
    """J^Q_{tau/2} e^{tau A} J^Q_{tau/2} u with A from eq. (2DA) / (3DA)."""
    Bs, _, _ = _axis_pieces(n, alpha, eps, a, b)
    EA = scipy.linalg.expm(tau * _kron_sum(Bs))
    E = math.exp(-tau)
    jq = lambda v: v / np.sqrt(v * v + (1 - v * v) * E)
    return jq(EA @ jq(u.ravel())).reshape(u.shape)


def _axis_assignment_errors(n, alpha, eps=0.3, tau=0.2, a=-1.0, b=1.5):
    """Largest differences of one oracle step (two-level and one-level) and of the
    oracle energy from the Kronecker-sum definitions. A mutant that makes the
    oracle fail to run at all counts as an infinite error."""
    u = np.random.default_rng(sum(n)).uniform(-1.0, 1.0, tuple(reversed(n)))
    try:
        two = O.Scheme(n, alpha, eps, tau, a, b).step(u)
        one = O.Scheme(n, alpha, eps, tau, a, b, kind="one_level").step(u)
        en = O.discrete_energy(u, O.Scheme(n, alpha, eps, tau, a, b))
    except (ValueError, IndexError):
        return math.inf, math.inf, math.inf
    e_two = float(np.abs(two - _kron_two_level_step(n, alpha, eps, tau, a, b, u)).max())
    e_one = float(np.abs(one - _kron_one_level_step(n, alpha, eps, tau, a, b, u)).max())
    Bs, _, _ = _axis_pieces(n, alpha, eps, a, b)
    hprod = float(np.prod([(b - a) / (nl + 1) for nl in n]))
    v = u.ravel()
    ref = hprod * (0.25 * float(np.sum((v * v - 1) ** 2)) - 0.5 * float(v @ (_kron_sum(Bs) @ v)))
    return e_two, e_one, abs(en - ref) / abs(ref)


@pytest.mark.parametrize("n,alpha", _AXIS_CASES, ids=str)
def test_axis_assignment_against_kronecker_sums(n, alpha):
    """One oracle step equals the dense step built from the Kronecker sums of
    eqs. (2DA)/(3DA)/(newlinear), and the oracle energy equals
    h^d((1/4)(u^2-1)^T(u^2-1) - (1/2) u^T A u) with that A (Example 5)."""
    e_two, e_one, e_en = _axis_assignment_errors(n, alpha)
    assert e_two <= 1e-14 and e_one <= 1e-14 and e_en <= 1e-13, (e_two, e_one, e_en)


def _stencil_2d(n, alpha, eps, a, b, u):
    """The right-hand side of eq. (disFAC) in 2D without the nonlinear term,
    written with the double indices of the paper: u[j, i] is u_{i,j}, i along
    x^(1) with (alpha_1, h_1, m_1), j along x^(2) with (alpha_2, h_2, m_2)."""
    (n1, n2), (a1, a2) = n, alpha
    m1, m2 = n1 + 1, n2 + 1
    h1, h2 = (b - a) / m1, (b - a) / m2
    full = np.zeros((m2 + 1, m1 + 1))
    full[1:m2, 1:m1] = u
    w1, w2 = O.omega_weights(a1, m1 + 2), O.omega_weights(a2, m2 + 2)
    p1 = -eps ** 2 / (2 * h1 ** a1 * math.cos(a1 * math.pi / 2))
    p2 = -eps ** 2 / (2 * h2 ** a2 * math.cos(a2 * math.pi / 2))
    out = np.zeros_like(u)
    for j in range(1, m2):
        for i in range(1, m1):
            s1 = sum(w1[k] * full[j, i - k + 1] for k in range(i + 2)) + \
                sum(w1[k] * full[j, i + k - 1] for k in range(m1 - i + 2))
            s2 = sum(w2[k] * full[j - k + 1, i] for k in range(j + 2)) + \
                sum(w2[k] * full[j + k - 1, i] for k in range(m2 - j + 2))
            out[j - 1, i - 1] = p1 * s1 + p2 * s2
    return out


@pytest.mark.parametrize("n,alpha", [((2, 3), (1.2, 1.8)), ((5, 3), (1.7, 1.3)), ((4, 4), (1.1, 1.9))], ids=str)
def test_kronecker_sum_is_the_2d_stencil(n, alpha):
    """The Kronecker sum used by the pins above equals the literal double-index
    stencil of eq. (disFAC) (alpha_1, h_1 on the index i of x^(1)), so the pins
    do not rest on the ordering convention alone."""
    eps, a, b = 0.3, -1.0, 1.5
    Bs, _, _ = _axis_pieces(n, alpha, eps, a, b)
    A = _kron_sum(Bs)
    u = np.random.default_rng(11).uniform(-1.0, 1.0, tuple(reversed(n)))
    np.testing.assert_allclose((A @ u.ravel()).reshape(u.shape), _stencil_2d(n, alpha, eps, a, b, u),
                               rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------- energy -------

def _ginzburg_landau_energy(u, n, eps, a, b):
    """h_1...h_d (1/4 sum (u^2-1)^2 + eps^2/2 sum over grid edges ((u_i - u_j)/h_l)^2),
    the edges to the zero Dirichlet boundary included: the classical discrete
    Ginzburg-Landau energy, written with differences rather than a matrix."""
    hs = [(b - a) / (m + 1) for m in n]
    grad = 0.0
    for l, h in enumerate(hs):
        ax = u.ndim - 1 - l
        pad = [(0, 0)] * u.ndim
        pad[ax] = (1, 1)
        grad += np.sum(np.diff(np.pad(u, pad), axis=ax) ** 2) / h ** 2
    return float(np.prod(hs)) * (0.25 * np.sum((u * u - 1) ** 2) + 0.5 * eps ** 2 * grad)


@pytest.mark.parametrize("n", [(5, 7), (3, 4, 6), (9,)], ids=str)
def test_energy_alpha2_is_ginzburg_landau(n):
    """Example 5's energy E(u) = h^d((1/4)(u^2-1)^T(u^2-1) - (1/2) u^T A u): with
    alpha = 2 on every axis B_l is the Dirichlet Laplacian times eps^2, so E is
    the edge-difference sum above. Non-square grids (a different h per axis) make
    an axis mix-up fail too."""
    sch = O.Scheme(n, (2.0,) * len(n), 0.3, 0.01, -1.0, 1.0)
    u = np.random.default_rng(len(n)).uniform(-1.0, 1.0, tuple(reversed(n)))
    ref = _ginzburg_landau_energy(u, n, 0.3, -1.0, 1.0)
    assert abs(O.discrete_energy(u, sch) - ref) <= 1e-13 * ref


@pytest.mark.parametrize("alpha", [(1.2, 1.8), (1.5, 1.05), (1.95, 1.3)], ids=str)
def test_energy_bounds_and_zero_field(alpha):
    """For alpha in (1, 2), B is symmetric with a negative diagonal and
    nonpositive row sums (Proposition 1), so -u^T A u >= 0 (Gershgorin) and
    E(u) >= h^d (1/4) sum (u^2-1)^2; E(0) = h^d N / 4 exactly; at u = +-1 E is
    the nonlocal term alone, which grows with eps^2."""
    n = (11, 6)
    hs = [2.0 / (m + 1) for m in n]
    sch = O.Scheme(n, alpha, 0.2, 0.01)
    rng = np.random.default_rng(7)
    for _ in range(5):
        u = rng.uniform(-1.0, 1.0, (6, 11))
        bulk = float(np.prod(hs)) * 0.25 * np.sum((u * u - 1) ** 2)
        assert O.discrete_energy(u, sch) > bulk
    assert O.discrete_energy(np.zeros((6, 11)), sch) == pytest.approx(np.prod(hs) * 66 / 4, rel=1e-15)
    ones = np.ones((6, 11))
    e1 = O.discrete_energy(ones, sch)
    e2 = O.discrete_energy(ones, O.Scheme(n, alpha, 0.4, 0.01))
    assert e1 > 0 and e2 == pytest.approx(4 * e1, rel=1e-13)


def test_energy_decays_along_the_scheme():
    """Example 5 reports that E(u^n) decreases monotonically; on a 31 x 31 grid
    with u0 = 0.8 rand - 0.4 it does so over 200 steps."""
    p = I.Problem(n=(31, 31), alpha=(1.5, 1.7), eps=0.05, tau=0.01)
    sch = O.Scheme.for_problem(p)
    u = I.random_field(p, 4, -0.4, 0.4)
    prev = O.discrete_energy(u, sch)
    for _ in range(200):
        u = sch.step(u)
        e = O.discrete_energy(u, sch)
        assert e < prev
        prev = e


# ------------------------------------------------- planted mistakes --------

class _Mutant:
    """Context manager that swaps one oracle function for a mutated copy."""

    def __init__(self, name, fn):
        self.name, self.fn = name, fn

    def __enter__(self):
        self.old = getattr(O, self.name)
        setattr(O, self.name, self.fn)

    def __exit__(self, *exc):
        setattr(O, self.name, self.old)


def _table2_first_two_level():
    res = []
    for N in (100, 200):
        p = I.example1_problem((1.2, 1.4), 1.0 / N)
        res.append(O.solve(p, I.example1_u0(p)))
    return O.time_error(res[0], res[1])


def _wrong_split(B):  # wraps by m instead of m - 1
    n = B.shape[0]
    b = lambda k: B[k, 0] if 0 <= k < n else (B[0, -k] if -n < k < 0 else 0.0)
    C = np.array([[0.5 * (b(i - j) + b(i - j - n - 1 if i > j else i - j + n + 1)) if i != j
                   else 0.5 * b(0) for j in range(n)] for i in range(n)])
    return C, B - C


def _wrong_factor(alpha, eps, h, n, tau):  # drops the closing e^{tau/2 C}
    C, S = O.split_CS(O.matrix_B(alpha, eps, h, n))
    return O.expm_symmetric(C, tau) @ O.expm_symmetric(S, tau)


@pytest.mark.parametrize("mutant", [
    ("nonlinear_flow", lambda v, s: v / np.sqrt(v * v + (1 - v * v) * math.exp(-s))),
    ("riesz_factor", lambda a, e, h: -e / (2 * h ** a * math.cos(a * math.pi / 2))),
    ("split_CS", _wrong_split),
    ("axis_two_level_factor", _wrong_factor),
], ids=["jq-exponent", "eps-not-squared", "split-wrap-index", "dropped-C-half"])
def test_planted_mistakes_fail_table2(mutant):
    with _Mutant(*mutant):
        et = _table2_first_two_level()
    assert not _close_to_printed(et, 1.2824e-7), et


def _energy_mutant(sign=-0.5, bulk=0.25, hpow=True):
    def energy(u, scheme):
        Au = np.zeros_like(u)
        hprod = 1.0
        for ax in range(u.ndim):
            h = (scheme.b - scheme.a) / (scheme.n[ax] + 1)
            hprod = hprod * h if hpow else h
            Au += O.apply_axis(u, O.matrix_B(scheme.alpha[ax], scheme.eps, h, scheme.n[ax]), ax + 1)
        w = u * u - 1.0
        return hprod * (bulk * float(np.sum(w * w)) + sign * float(np.sum(u * Au)))
    return energy


@pytest.mark.parametrize("mutant", [_energy_mutant(sign=+0.5), _energy_mutant(bulk=0.5),
                                    _energy_mutant(hpow=False)],
                         ids=["energy-sign", "energy-bulk-weight", "energy-h-power"])
def test_planted_mistakes_fail_energy_pins(mutant):
    n = (5, 7)
    sch = O.Scheme(n, (2.0, 2.0), 0.3, 0.01)
    u = np.random.default_rng(2).uniform(-1.0, 1.0, (7, 5))
    with _Mutant("discrete_energy", mutant):
        got = O.discrete_energy(u, sch)
    ref = _ginzburg_landau_energy(u, n, 0.3, -1.0, 1.0)
    assert abs(got - ref) > 1e-6 * ref


class _AlphaReversed(O.Scheme):
    """Mutant: the alpha list taken in reverse axis order."""

    def __init__(self, n, alpha, *args, **kw):
        super().__init__(n, tuple(reversed(alpha)), *args, **kw)


class _HOfOtherAxis(O.Scheme):
    """Mutant: each axis's h computed from the mirrored axis's n."""

    def __init__(self, n, alpha, eps, tau, a=-1.0, b=1.0, kind="two_level", route="dense"):
        super().__init__(n, alpha, eps, tau, a, b, kind, route)
        build = {"two_level": O.axis_two_level_factor, "one_level": O.axis_one_level_factor,
                 "adi": O.axis_adi_factor}[kind]
        mirrored = list(reversed(self.n))
        self.P = [build(self.alpha[ax], self.eps, (self.b - self.a) / (mirrored[ax] + 1), nn, self.tau)
                  for ax, nn in enumerate(self.n)]


def _mirrored_apply_axis(u, P, axis):
    """Mutant: paper axis l taken as numpy axis l - 1 (x^(1) slowest)."""
    ax = axis - 1
    return np.moveaxis(np.tensordot(P, u, axes=([1], [ax])), 0, ax)


@pytest.mark.parametrize("mutant", [("Scheme", _AlphaReversed), ("Scheme", _HOfOtherAxis),
                                    ("apply_axis", _mirrored_apply_axis)],
                         ids=["alpha-reversed", "h-of-other-axis", "memory-axis-mirrored"])
@pytest.mark.parametrize("n,alpha", [_AXIS_CASES[0], _AXIS_CASES[3]], ids=str)
def test_planted_axis_mixups_fail_kronecker_pins(mutant, n, alpha):
    with _Mutant(*mutant):
        e_two, e_one, e_en = _axis_assignment_errors(n, alpha)
    assert e_two > 1e-6 and e_one > 1e-6, (e_two, e_one, e_en)


@pytest.mark.parametrize("mutant", [("Scheme", _AlphaReversed), ("apply_axis", _mirrored_apply_axis)],
                         ids=["alpha-reversed", "memory-axis-mirrored"])
def test_planted_axis_mixups_fail_on_a_square_grid(mutant):
    """On a square grid with distinct alpha per axis only the alpha assignment
    tells the axes apart; both mix-ups still fail (the energy pin included)."""
    with _Mutant(*mutant):
        e_two, e_one, e_en = _axis_assignment_errors(*_AXIS_CASES[1])
    assert e_two > 1e-6 and e_one > 1e-6 and e_en > 1e-6, (e_two, e_one, e_en)
