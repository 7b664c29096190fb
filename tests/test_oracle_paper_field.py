"""Pins of the oracle's paper-faithful workload (Sec. 5 field, uniform draws, 2 pi target)."""
import numpy as np

from oracle import fem, kl, philox, solve


def test_uniform_draws_range_and_moments():
    xi = philox.uniforms(0, 0, 1, np.arange(2000), 125, 4.0)
    assert xi.shape == (2000, 125)
    assert xi.min() > -4.0 and xi.max() <= 4.0
    n = xi.size
    assert abs(xi.mean()) < 5 * np.sqrt(16.0 / 3.0 / n)
    assert abs(xi.var() - 16.0 / 3.0) < 5 * np.sqrt((256.0 / 5.0 - (16.0 / 3.0) ** 2) / n)
    # the same counters as the normal draws: a sample's draw is independent of its batch
    assert np.array_equal(philox.uniforms(0, 0, 1, [7], 125, 4.0)[0], xi[7])


def test_paper_modes_orthogonal():
    """int_D phi_a phi_b dx = delta_ab / 8 for the cosine products (exact midpoint sums
    on a fine grid reproduce it to rounding)."""
    T = kl.PaperKLTable(0.15, 5)
    N = 40
    P = T.cell_modes(N)
    G = P @ P.T / N ** 3
    assert np.abs(G - np.eye(125) / 8).max() < 1e-12


def test_paper_field_variance_monte_carlo():
    """Var a~(x) = sum lambda phi(x)^2 Var(xi), Var(U(-4, 4)) = 16/3."""
    T = kl.PaperKLTable(0.15, 5)
    P = T.cell_modes(4)
    xi = philox.uniforms(3, 0, 0, np.arange(20000), 125, 4.0)
    field = (T.sqrt_lam3[None, :] * xi) @ P
    var_exact = (16.0 / 3.0) * (T.lam3[:, None] * P ** 2).sum(0)
    rel = np.abs(field.var(0) / var_exact - 1.0)
    assert rel.max() < 0.06  # 20000 samples: sampling error ~ sqrt(2/20000) * few


def test_manufactured_solution_2pi_target():
    """a = 1, z = 3 (2 pi)^2 prod sin(2 pi x_c): ||y_h - g_h||_M = O(h^2) with g = prod sin(2 pi x)."""
    errs = []
    for N in (8, 16, 32):
        lev = fem.Level(N)
        A = lev.restrict(lev.stiffness(np.ones(lev.nc)))
        c = np.arange(N ** 3)
        cx, cy, cz = (c % N + 0.5) / N, ((c // N) % N + 0.5) / N, (c // N ** 2 + 0.5) / N
        w = 2 * np.pi
        z = 3 * w ** 2 * np.sin(w * cx) * np.sin(w * cy) * np.sin(w * cz)
        b = (1.0 / N) ** 3 * (lev.interpolation(N).T @ z)
        y = np.zeros(lev.nn)
        y[lev.interior], _ = solve.solve(A, b[lev.interior], N)
        e = y - lev.nodal_target(2)
        errs.append(np.sqrt(e @ (lev.mass() @ e)))
    assert 3.3 < errs[1] / errs[2] < 4.3 and errs[0] / errs[1] > 2.5
