"""Karhunen-Loeve modes of the exponential covariance and the log-normal field.

Oracle (test infrastructure only).  The paper builds its random coefficient
as exp of a truncated KL expansion a~ = mu0 + sum sqrt(lambda) phi xi
(Sec. 5, field model of the numerical experiments); the workload built here
keeps that structure with the covariance C(x, x') = exp(-|x - x'| / l_c) in
each coordinate, tensorised over x, y, z, mean 0, sigma multiplying the sum,
and xi ~ N(0, 1).

1D eigenpairs on [0, 1] (t = x - 1/2, c = 1/l_c); the integral equation
int C(t, s) phi(s) ds = lambda phi(t) reduces to phi'' = -omega^2 phi with
lambda = 2c / (omega^2 + c^2) and Robin conditions at t = +-1/2:
  even modes phi = cos(omega t) / sqrt(1/2 + sin(omega)/(2 omega)),
            omega tan(omega/2) = c,
  odd modes  phi = sin(omega t) / sqrt(1/2 - sin(omega)/(2 omega)),
            tan(omega/2) = -omega / c.
1D mode n has omega in (n pi, (n+1) pi): even for even n, odd for odd n.
Roots: bisection on a pole-free form of each condition, to the last bit.

3D modes: products phi_i(x) phi_j(y) phi_k(z) with eigenvalue
lambda_i lambda_j lambda_k.  The K largest are kept; the sort key is the
product of the three sorted factors ((smallest*middle)*largest), so that
permutations of (i, j, k) get bit-identical keys; ties are ordered by the
tuple (i, j, k) ascending.

Pins (tests/test_oracle_kl.py): orthonormality by quadrature, the integral
equation residual, the trace identity sum(lambda) = 1 with a closed-form tail
bound, and pointwise variance <= sigma^2.
"""
import numpy as np


def _bisect(f, lo, hi):
    flo = f(lo)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        fm = f(mid)
        if fm == 0.0:
            return mid
        if (fm < 0.0) == (flo < 0.0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def modes_1d(corr_len, n):
    """First n 1D eigenpairs: returns (omega[n], lam[n], parity[n], norm[n]).

    parity 0 = even (cos), 1 = odd (sin); norm is the L2 normalisation factor.
    """
    c = 1.0 / corr_len
    omega = np.empty(n)
    for m in range(n):
        # s = omega / 2 lies in (m pi/2, (m+1) pi/2)
        lo, hi = m * np.pi / 2, (m + 1) * np.pi / 2
        if m % 2 == 0:  # tan(s) = c / (2 s)  <=>  2 s sin s - c cos s = 0
            f = lambda s: 2.0 * s * np.sin(s) - c * np.cos(s)
        else:  # tan(s) = -2 s / c  <=>  c sin s + 2 s cos s = 0
            f = lambda s: c * np.sin(s) + 2.0 * s * np.cos(s)
        omega[m] = 2.0 * _bisect(f, lo, hi)
    lam = 2.0 * c / (omega ** 2 + c ** 2)
    parity = np.arange(n) % 2
    norm = np.where(parity == 0,
                    1.0 / np.sqrt(0.5 + np.sin(omega) / (2.0 * omega)),
                    1.0 / np.sqrt(0.5 - np.sin(omega) / (2.0 * omega)))
    return omega, lam, parity, norm


def eval_1d(omega, parity, norm, x):
    """phi_n(x) for all modes n at points x: returns [n, len(x)]."""
    t = np.asarray(x, dtype=np.float64)[None, :] - 0.5
    w = omega[:, None]
    val = np.where(parity[:, None] == 0, np.cos(w * t), np.sin(w * t))
    return norm[:, None] * val


def select_3d(lam1, K):
    """K largest tensor-product eigenvalues: returns (idx[K, 3], lam3[K])."""
    n = lam1.shape[0]
    cand = []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                a, b, d = sorted((lam1[i], lam1[j], lam1[k]))
                cand.append((-(a * b) * d, i, j, k))
    cand.sort()
    sel = cand[:K]
    idx = np.array([[s[1], s[2], s[3]] for s in sel], dtype=np.int64)
    lam3 = np.array([-s[0] for s in sel])
    return idx, lam3


class PaperKLTable:
    """The random field of the paper's numerical experiments (Sec. 5):
    a~(x) = sum_{j,k,l=1}^{m} sqrt(lambda_jkl) phi_jkl(x) xi_jkl with
    phi_jkl(x) = cos(j pi x2) cos(k pi x3) cos(l pi x1) (not normalised),
    lambda_jkl = exp(-pi (j + k + l) rho), mean 0; xi ~ U(-4, 4) is drawn elsewhere.
    Modes are ordered (j, k, l) with l fastest; idx holds the 1D indices along
    (x, y, z) = (l - 1, j - 1, k - 1)."""

    def __init__(self, rho, m):
        self.rho, self.m, self.n_modes = rho, m, m ** 3
        jkl = np.array([(j, k, l) for j in range(1, m + 1) for k in range(1, m + 1) for l in range(1, m + 1)])
        self.jkl = jkl
        self.idx = np.stack([jkl[:, 2] - 1, jkl[:, 0] - 1, jkl[:, 1] - 1], axis=1)
        self.lam3 = np.exp(-np.pi * jkl.sum(axis=1) * rho)
        self.sqrt_lam3 = np.sqrt(self.lam3)

    def cell_modes(self, N):
        """Phi[mode, cell] at the N^3 cell centres, cell index ix + N (iy + N iz)."""
        xc = (np.arange(N) + 0.5) / N
        cz, cy, cx = np.meshgrid(xc, xc, xc, indexing="ij")
        j, k, l = self.jkl[:, 0], self.jkl[:, 1], self.jkl[:, 2]
        phi = (np.cos(j[:, None, None, None] * np.pi * cy[None]) * np.cos(k[:, None, None, None] * np.pi * cz[None]) *
               np.cos(l[:, None, None, None] * np.pi * cx[None]))
        return phi.reshape(self.n_modes, N ** 3)


class KLTable:
    """Mode table for a workload: 1D eigenpairs plus the K selected 3D modes."""

    def __init__(self, corr_len, n_modes, n1d=None):
        n1d = 4 if n1d is None else n1d
        while True:
            self.omega, self.lam1, self.parity, self.norm = modes_1d(corr_len, n1d)
            self.idx, self.lam3 = select_3d(self.lam1, n_modes)
            # enough 1D modes once the selection leaves the last one unused
            if self.idx.max() < n1d - 1:
                break
            n1d += 1
        self.corr_len = corr_len
        self.n_modes = n_modes
        self.sqrt_lam3 = np.sqrt(self.lam3)

    def cell_modes(self, N):
        """Phi[k, cell] = phi_i(x) phi_j(y) phi_l(z) at the N^3 cell centres.

        Cell index = ix + N*(iy + N*iz)."""
        xc = (np.arange(N) + 0.5) / N
        p1 = eval_1d(self.omega, self.parity, self.norm, xc)  # [n1d, N]
        i, j, k = self.idx[:, 0], self.idx[:, 1], self.idx[:, 2]
        phi = p1[k][:, :, None, None] * p1[j][:, None, :, None] * p1[i][:, None, None, :]
        return phi.reshape(self.n_modes, N ** 3)

    def log_coefficient(self, xi, sigma, N):
        """log a at cell centres of an N^3 grid for each row of xi: [S, N^3]."""
        coef = sigma * self.sqrt_lam3[None, :] * xi
        return coef @ self.cell_modes(N)
