"""Pins of the oracle's assembled Q1 operators, control operator and solvers."""
import numpy as np
import pytest

from oracle import fem, solve


def test_element_matrix_closed_form():
    """Q1 Laplace element matrix of a cube of side h is h * K_ref with
    diagonal 1/3, edge neighbours 0, face and body diagonals -1/12."""
    h = 0.25
    Ke, Me = fem.element_matrices(h)
    for a in range(8):
        for b in range(8):
            ham = bin(a ^ b).count("1")
            want = {0: 1.0 / 3.0, 1: 0.0, 2: -1.0 / 12.0, 3: -1.0 / 12.0}[ham]
            assert abs(Ke[a, b] - h * want) < 1e-15
            # mass: h^3 * (1/3)^(3-ham) * (1/6)^ham
            assert abs(Me[a, b] - h ** 3 * (1 / 3) ** (3 - ham) * (1 / 6) ** ham) < 1e-16


@pytest.mark.parametrize("N", [4, 8])
def test_discrete_eigenpairs(N):
    """For a = 1, v = sin(i pi x) sin(j pi y) sin(k pi z) at the nodes is an
    eigenvector of the stiffness with eigenvalue kmm + mkm + mmk and of the
    mass with mmm, k_j = (2/h)(1 - cos j pi h), m_j = (h/3)(2 + cos j pi h)."""
    lev = fem.Level(N)
    h = lev.h
    A = lev.restrict(lev.stiffness(np.ones(lev.nc)))
    M = lev.restrict(lev.mass())
    x, y, z = [c[lev.interior] for c in lev.node_coords()]
    k1 = lambda j: (2.0 / h) * (1.0 - np.cos(j * np.pi * h))
    m1 = lambda j: (h / 3.0) * (2.0 + np.cos(j * np.pi * h))
    for (i, j, k) in [(1, 1, 1), (1, 2, 3), (N - 1, 1, 2), (N - 1, N - 1, N - 1)]:
        v = np.sin(i * np.pi * x) * np.sin(j * np.pi * y) * np.sin(k * np.pi * z)
        lam = k1(i) * m1(j) * m1(k) + m1(i) * k1(j) * m1(k) + m1(i) * m1(j) * k1(k)
        assert np.abs(A @ v - lam * v).max() < 1e-12 * lam
        mu = m1(i) * m1(j) * m1(k)
        assert np.abs(M @ v - mu * v).max() < 1e-13 * mu


def test_one_dof_brute_force():
    """2^3 cells: the only interior node sees A = (h/3) sum_e a_e, h = 1/2."""
    lev = fem.Level(2)
    a = np.array([1.0, 2.0, 3.0, 4.0, 0.5, 0.25, 8.0, 1.5])
    A = lev.restrict(lev.stiffness(a))
    assert A.shape == (1, 1)
    assert abs(A[0, 0] - 0.5 / 3.0 * a.sum()) < 1e-15


def test_symmetry_and_row_sums():
    lev = fem.Level(8)
    rng = np.random.default_rng(0)
    a = np.exp(rng.standard_normal(lev.nc))
    Af = lev.stiffness(a)
    assert abs(Af - Af.T).max() < 1e-15 * abs(Af).max()
    # constants are in the kernel of the full (unrestricted) operator
    assert np.abs(Af @ np.ones(lev.nn)).max() < 1e-13
    A = lev.restrict(Af)
    u, v = rng.standard_normal((2, A.shape[0]))
    assert abs(u @ (A @ v) - v @ (A @ u)) < 1e-12 * np.abs(u @ (A @ v))
    # the variable-coefficient stencil: a node's coupling to a face-diagonal
    # neighbour is -h/12 times the sum of the two cells sharing that face diagonal
    N, n1, h = 8, 9, 1.0 / 8
    node = lambda i, j, k: i + n1 * (j + n1 * k)
    cell = lambda i, j, k: i + N * (j + N * k)
    i, j, k = 3, 4, 5
    want = -h / 12 * (a[cell(i, j, k - 1)] + a[cell(i, j, k)])
    assert abs(Af[node(i, j, k), node(i + 1, j + 1, k)] - want) < 1e-15
    assert abs(Af[node(i, j, k), node(i + 1, j + 1, k + 1)] + h / 12 * a[cell(i, j, k)]) < 1e-15
    assert abs(Af[node(i, j, k), node(i + 1, j, k)]) < 1e-15


def test_control_operator_adjoint_and_mass():
    lev = fem.Level(4)
    Nc = 8
    hc3 = (1.0 / Nc) ** 3
    I = lev.interpolation(Nc)
    rng = np.random.default_rng(2)
    z = rng.standard_normal(Nc ** 3)
    q = rng.standard_normal(lev.nn)
    Bz = hc3 * (I.T @ z)
    # <B z, q> = <z, B* q>_U
    assert abs(Bz @ q - hc3 * (z @ (I @ q))) < 1e-14
    # partition of unity: sum_n (B z)_n = int z
    assert abs(Bz.sum() - hc3 * z.sum()) < 1e-14
    # B 1 = M 1 (int phi_n = sum_m M_nm)
    assert np.abs(hc3 * (I.T @ np.ones(Nc ** 3)) - lev.mass() @ np.ones(lev.nn)).max() < 1e-15
    # B* of a trilinear function reproduces it at the cell centres
    x, y, zc = lev.node_coords()
    qlin = 1.0 + 2.0 * x - 3.0 * y + 0.5 * zc + x * y * zc
    c = np.arange(Nc ** 3)
    cx, cy, cz = (c % Nc + 0.5) / Nc, ((c // Nc) % Nc + 0.5) / Nc, (c // Nc ** 2 + 0.5) / Nc
    assert np.abs(I @ qlin - (1.0 + 2.0 * cx - 3.0 * cy + 0.5 * cz + cx * cy * cz)).max() < 1e-14


def test_manufactured_solution_second_order():
    """a = 1, z = 3 pi^2 prod sin(pi x_c): ||y_h - g_h||_M = O(h^2)."""
    errs = []
    for N in (8, 16, 32):
        lev = fem.Level(N)
        A = lev.restrict(lev.stiffness(np.ones(lev.nc)))
        c = np.arange(N ** 3)
        cx, cy, cz = (c % N + 0.5) / N, ((c // N) % N + 0.5) / N, (c // N ** 2 + 0.5) / N
        z = 3 * np.pi ** 2 * np.sin(np.pi * cx) * np.sin(np.pi * cy) * np.sin(np.pi * cz)
        b = (1.0 / N) ** 3 * (lev.interpolation(N).T @ z)
        y = np.zeros(lev.nn)
        y[lev.interior], _ = solve.solve(A, b[lev.interior], N)
        e = y - lev.nodal_target()
        errs.append(np.sqrt(e @ (lev.mass() @ e)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.8 < r2 < 4.2
    assert errs[2] < 2e-3


def test_solvers_agree():
    lev = fem.Level(16)
    rng = np.random.default_rng(3)
    A = lev.restrict(lev.stiffness(np.exp(1.5 * rng.standard_normal(lev.nc))))
    b = rng.standard_normal(A.shape[0])
    xd, _ = solve.solve(A, b, 16, method="direct")
    for m in ("jacobi", "mg"):
        x, it = solve.solve(A, b, 16, rtol=1e-13, method=m)
        assert it > 1
        assert np.linalg.norm(b - A @ x) <= 1e-13 * np.linalg.norm(b)
        assert np.abs(x - xd).max() <= 1e-10 * np.abs(xd).max()
    x0, it0 = solve.solve(A, np.zeros_like(b), 16, method="mg")
    assert it0 == 0 and not np.any(x0)


@pytest.mark.parametrize("N,Nc", [(8, 4), (8, 2), (4, 8), (4, 4), (4, 16), (2, 16)])
def test_control_cell_averages(N, Nc):
    """I[c, n] = average of phi_n over control cell c, both when the control grid is
    finer and when it is coarser than the level: partition of unity, exact averages
    of the Q1-represented functions x and x y z, the trapezoid identity for x^2
    (mean over the cell + h^2/6 for a coarse control), and B 1 = int phi_n = h^3."""
    lev = fem.Level(N)
    I = lev.interpolation(Nc)
    x, y, z = lev.node_coords()
    c = np.arange(Nc ** 3)
    xc, yc, zc = (c % Nc + 0.5) / Nc, ((c // Nc) % Nc + 0.5) / Nc, (c // Nc ** 2 + 0.5) / Nc
    assert np.abs(I @ np.ones(lev.nn) - 1).max() < 1e-14
    assert np.abs(I @ x - xc).max() < 1e-14
    assert np.abs(I @ (x * y * z) - xc * yc * zc).max() < 1e-14
    if N > Nc:
        H, h = 1.0 / Nc, 1.0 / N
        a0 = xc - H / 2
        mean_x2 = ((a0 + H) ** 3 - a0 ** 3) / (3 * H)
        assert np.abs(I @ (x * x) - (mean_x2 + h * h / 6)).max() < 1e-14
    b = (1.0 / Nc) ** 3 * (I.T @ np.ones(Nc ** 3))
    assert np.abs(b[lev.interior] - (1.0 / N) ** 3).max() < 1e-17


@pytest.mark.parametrize("N,Nc", [(4, 4), (4, 8), (4, 16), (4, 32), (2, 16)])
def test_rhs_closed_form_fine_control(N, Nc):
    """(B z)_n = h_c^3 sum_c z_c phi_n(x_c) for a control r = Nc / N times finer than
    the grid.  The hat weights of a node's 2r control cells per axis sum to r and are
    symmetric about the node, so for z_c = x_c y_c z_c (cell centres) every interior
    node gets exactly h^3 x_i y_j z_k, and for z_c = 1 exactly h^3."""
    lev = fem.Level(N)
    I = lev.interpolation(Nc)
    c = np.arange(Nc ** 3)
    xc, yc, zc = (c % Nc + 0.5) / Nc, ((c // Nc) % Nc + 0.5) / Nc, (c // Nc ** 2 + 0.5) / Nc
    x, y, z = lev.node_coords()
    hc3, h3 = (1.0 / Nc) ** 3, (1.0 / N) ** 3
    b = hc3 * (I.T @ (xc * yc * zc))
    assert np.abs(b[lev.interior] - h3 * (x * y * z)[lev.interior]).max() < 1e-16
    b1 = hc3 * (I.T @ np.ones(Nc ** 3))
    assert np.abs(b1[lev.interior] - h3).max() < 1e-17

