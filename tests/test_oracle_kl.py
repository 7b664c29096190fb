"""Pins of the oracle's KL mode table (1D exponential covariance eigenpairs)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import kl


@pytest.mark.parametrize("lc", [0.1, 0.2, 0.3])
def test_transcendental_conditions(lc):
    c = 1.0 / lc
    omega, lam, parity, norm = kl.modes_1d(lc, 12)
    for n in range(12):
        w = omega[n]
        assert n * np.pi < w < (n + 1) * np.pi
        if parity[n] == 0:
            assert abs(w * np.tan(w / 2) - c) < 1e-9 * max(1.0, c)
        else:
            assert abs(np.tan(w / 2) + w / c) < 1e-9 * max(1.0, w / c)
    assert np.all(np.diff(lam) < 0)


@pytest.mark.parametrize("lc", [0.1, 0.3])
def test_orthonormal(lc):
    omega, lam, parity, norm = kl.modes_1d(lc, 10)
    x, w = np.polynomial.legendre.leggauss(200)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    P = kl.eval_1d(omega, parity, norm, x)
    G = (P * w[None, :]) @ P.T
    assert np.abs(G - np.eye(10)).max() < 1e-12


@pytest.mark.parametrize("lc", [0.2, 0.3])
def test_integral_equation(lc):
    """int_0^1 exp(-|x-s|/lc) phi(s) ds = lambda phi(x) at a few points."""
    omega, lam, parity, norm = kl.modes_1d(lc, 6)
    for n in range(6):
        for x0 in (0.0, 0.13, 0.5, 0.91):
            f = lambda s: np.exp(-abs(x0 - s) / lc) * kl.eval_1d(omega[n:n + 1], parity[n:n + 1],
                                                                   norm[n:n + 1], [s])[0, 0]
            val, _ = integrate.quad(f, 0.0, 1.0, points=[x0], epsabs=1e-13, epsrel=1e-12, limit=200)
            phi = kl.eval_1d(omega[n:n + 1], parity[n:n + 1], norm[n:n + 1], [x0])[0, 0]
            assert abs(val - lam[n] * phi) < 1e-10


def test_trace_is_one():
    """sum_n lambda_n = int_0^1 C(x, x) dx = 1; the tail beyond n modes is
    bounded by sum 2c/(omega^2) with omega > n pi."""
    lc = 0.2
    c = 1.0 / lc
    n = 2000
    _, lam, _, _ = kl.modes_1d(lc, n)
    tail_upper = 2.0 * c / np.pi ** 2 * (1.0 / (n - 1))  # sum_{m>=n} 1/(m^2) <= 1/(n-1)
    s = lam.sum()
    assert s < 1.0
    assert 1.0 - s <= tail_upper * 1.01


def test_3d_selection_and_variance():
    T = kl.KLTable(0.2, 128)
    assert T.idx.shape == (128, 3)
    assert np.all(np.diff(T.lam3) <= 0)
    # permutation groups have identical keys
    key = {tuple(r): v for r, v in zip(T.idx, T.lam3)}
    for r, v in key.items():
        for p in [(r[1], r[0], r[2]), (r[2], r[1], r[0])]:
            if p in key:
                assert key[p] == v
    # no unselected triple beats the smallest selected one
    n = T.lam1.shape[0]
    sel = set(map(tuple, T.idx))
    for i in range(n):
        for j in range(n):
            for k in range(n):
                if (i, j, k) not in sel:
                    a, b, d = sorted((T.lam1[i], T.lam1[j], T.lam1[k]))
                    assert (a * b) * d <= T.lam3[-1]
    # Mercer: truncated pointwise variance sum_k lam_k phi_k(x)^2 <= C(x, x) = 1
    Phi = T.cell_modes(8)
    var = (T.lam3[:, None] * Phi ** 2).sum(0)
    assert var.max() <= 1.0 and var.min() > 0.2


def test_log_coefficient_is_the_kl_sum():
    T = kl.KLTable(0.3, 64)
    rng = np.random.default_rng(1)
    xi = rng.standard_normal((2, 64))
    la = T.log_coefficient(xi, 1.5, 8)
    # brute force at one cell from the 1D functions
    ix, iy, iz = 3, 5, 6
    x, y, z = (ix + 0.5) / 8, (iy + 0.5) / 8, (iz + 0.5) / 8
    p = lambda n, t: kl.eval_1d(T.omega[n:n + 1], T.parity[n:n + 1], T.norm[n:n + 1], [t])[0, 0]
    ref = sum(1.5 * np.sqrt(T.lam3[k]) * xi[1, k] * p(T.idx[k, 0], x) * p(T.idx[k, 1], y) * p(T.idx[k, 2], z)
              for k in range(64))
    assert abs(la[1, ix + 8 * (iy + 8 * iz)] - ref) < 1e-13
